"""C-ABI checks that need no GPU: the library loads and exports every function
include/mcd.h declares; a host-only context validates its inputs and returns
the documented status codes; the library's threaded host sampler reproduces
the oracle's sampler bit for bit."""
import numpy as np
import pytest

import paper_2509_22975_gb300 as pkg
from oracle import fock, sampler as S
from workloads import configs as C, lattice as L


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    pkg.lib()


def host_ctx(w):
    ctx = pkg.Context(-1)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    return ctx


def test_exports_every_declared_symbol():
    L_ = pkg.lib()
    names = pkg.header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L_, n), n
    assert set(names) <= set(pkg._SIGS), set(names) - set(pkg._SIGS)


def test_status_strings_and_create_errors():
    L_ = pkg.lib()
    assert L_.mcd_status_string(0) == b"ok"
    assert L_.mcd_status_string(-6) == b"Lanczos breakdown"
    with pytest.raises(pkg.MCDError) as e:
        pkg.Context(-5)
    assert e.value.status == -1


def test_hamiltonian_validation():
    ctx = pkg.Context(-1)
    t = np.zeros((4, 4))
    t[0, 1] = 1.0                          # not symmetric
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_set_hamiltonian(t, None, [4.0], 2, 2)
    assert e.value.status == -1
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_hamiltonian(np.zeros((33, 33)), None, [1.0], 1, 1)   # n > 32
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_hamiltonian(np.zeros((4, 4)), None, [1.0, 2.0], 1, 1)  # bad U_len
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_hamiltonian(np.zeros((4, 4)), None, [1.0], 5, 1)  # N_up > n
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_set_basis([3])             # no Hamiltonian yet
    assert e.value.status == -8


def test_basis_validation_and_roundtrip():
    w = C.ring8_u4()
    ctx = host_ctx(w)
    full = fock.sector(8, 4, 4)
    ctx.mcd_set_basis(full[::7])
    assert np.array_equal(ctx.mcd_get_basis(), full[::7])
    for bad, code in [(full[[5, 3, 9]], -1), (full[[3, 3, 9]], -1),
                      (np.array([0b1111 << 8 | 0b111], dtype=np.uint64), -2),
                      (np.array([1 << 20 | (0b1111 << 8) | 0b1111], dtype=np.uint64), -2)]:
        with pytest.raises(pkg.MCDError) as e:
            ctx.mcd_set_basis(bad)
        assert e.value.status == code
    # a failed install keeps the previous basis
    assert np.array_equal(ctx.mcd_get_basis(), full[::7])


def test_device_calls_on_host_context():
    w = C.ring8_u4()
    ctx = host_ctx(w)
    ctx.mcd_set_basis(fock.sector(8, 4, 4)[:100])
    import ctypes
    E0, r = ctypes.c_double(), ctypes.c_double()
    it = ctypes.c_int()
    st = ctx.L.mcd_lanczos_ground(ctx.h, 10, 1e-10, 0, 0, ctypes.byref(E0), None, ctypes.byref(it),
                                  ctypes.byref(r))
    assert st == -9
    st = ctx.L.mcd_apply(ctx.h, 16, 1024, 1, 1, 0)
    assert st == -9


def oracle_basis(w, nf, seed=None, flags=0, beta=None, U=None, seeds=None):
    Uv = w.U_sites if U is None else np.asarray(U, float)
    return S.sample_basis(w.n_sites, w.lat.t, Uv, w.n_up, w.n_dn, nf,
                          w.beta if beta is None else beta,
                          [w.seed_word()] if seeds is None else seeds,
                          seed=w.seed if seed is None else seed, flags=flags)


@pytest.mark.parametrize("name,nf", [("ring8", 2000), ("ring8", 4900), ("tilted12", 1 << 18),
                                     ("square16", 200000)])
def test_sampler_bit_exact_vs_oracle(name, nf):
    w = C.WORKLOADS[name]()
    ctx = host_ctx(w)
    st, n = ctx.mcd_build_basis(w.seed, nf, w.beta, [w.seed_word()])
    got = ctx.mcd_get_basis()
    ref = oracle_basis(w, nf)
    assert n == len(ref) and st == (0 if len(ref) == nf else pkg.MCD_W_SHORT)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("threads", [1, 3, 16])
def test_sampler_thread_count_does_not_change_the_basis(threads):
    w = C.tilted12_u8()
    ctx = host_ctx(w)
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_THREADS, threads)
    ctx.mcd_build_basis(3, 20000, w.beta, [w.seed_word()])
    assert np.array_equal(ctx.mcd_get_basis(), oracle_basis(w, 20000, seed=3))


def test_sampler_new_only_flag_nonuniform_U_and_two_seeds():
    w = C.ring8_u4()
    rng = np.random.default_rng(11)
    U = rng.uniform(2.0, 8.0, size=8)
    ctx = pkg.Context(-1)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, U, 4, 4)
    other = (0b10101010 << 8) | 0b01010101
    seeds = [w.seed_word(), other]
    st, n = ctx.mcd_build_basis(5, 1500, 0.3, seeds, flags=pkg.MCD_SAMPLE_NEW_ONLY)
    ref = oracle_basis(w, 1500, seed=5, flags=S.NEW_ONLY, beta=0.3, U=U, seeds=seeds)
    assert np.array_equal(ctx.mcd_get_basis(), ref)
    assert len(ref) <= 1500


def test_sampler_short_return_on_disconnected_lattice():
    t = np.zeros((6, 6))
    for a, b in [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3)]:
        t[a, b] = t[b, a] = -1.0
    seed = (0b000011 << 6) | 0b011000
    ctx = pkg.Context(-1)
    ctx.mcd_set_hamiltonian(t, None, [4.0], 2, 2)
    st, n = ctx.mcd_build_basis(0, 225, 0.0, [seed])
    ref = S.sample_basis(6, t, np.full(6, 4.0), 2, 2, 225, 0.0, [seed], seed=0)
    assert st == pkg.MCD_W_SHORT
    assert np.array_equal(ctx.mcd_get_basis(), ref)


def test_sampler_argument_errors():
    w = C.ring8_u4()
    ctx = host_ctx(w)
    for args, code in [((0, 5000, 0.4, [w.seed_word()]), -1),        # > sector
                       ((0, 100, -1.0, [w.seed_word()]), -1),         # beta < 0
                       ((0, 100, 0.4, [0b111 << 8 | 0b1111]), -2),    # seed outside sector
                       ((0, 100, 0.4, [w.seed_word()], 8), -1)]:      # unknown flag
        with pytest.raises(pkg.MCDError) as e:
            ctx.mcd_build_basis(*args)
        assert e.value.status == code


def test_sampler_placement_option_on_host_context():
    # a host-only context samples on host threads under the default; asking
    # for the device is an error, not a silent change of placement
    w = C.ring8_u4()
    ctx = host_ctx(w)
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, pkg.SAMPLER_AUTO)
    ctx.mcd_build_basis(w.seed, 500, w.beta, [w.seed_word()])
    assert len(ctx.mcd_get_basis()) == 500
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, pkg.SAMPLER_DEVICE)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_build_basis(w.seed, 500, w.beta, [w.seed_word()])
    assert e.value.status == -1
    for bad in (-1, 3):
        with pytest.raises(pkg.MCDError):
            ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, bad)


def test_option_ranges():
    # every documented value is taken; values outside the documented range and
    # unknown options are MCD_E_INVALID
    ctx = pkg.Context(-1)
    ok = {pkg.MCD_OPT_HV_ALGO: [0, 1, 2, 3], pkg.MCD_OPT_KERNEL_TIMING: [0, 1],
          pkg.MCD_OPT_SAMPLER_THREADS: [0, 1, 16], pkg.MCD_OPT_SAMPLER_DEVICE: [0, 1, 2],
          pkg.MCD_OPT_HV_CACHE: [0, 1, 2], pkg.MCD_OPT_HASH_ITEM: [64, 128, 1024, 4096],
          pkg.MCD_OPT_APPLY_SYNC: [0, 1], pkg.MCD_OPT_WAIT_TEST: [-1, 0, 5], pkg.MCD_OPT_KRYLOV_STORE: [0, 1],
          pkg.MCD_OPT_HV_COLS: [0, 1, 2], pkg.MCD_OPT_BATCH_SPLIT: [0, 1, 2, 4],
          pkg.MCD_OPT_BATCH_MODE: [0, 1]}
    bad = {pkg.MCD_OPT_HV_ALGO: [-1, 4], pkg.MCD_OPT_SAMPLER_THREADS: [-1],
           pkg.MCD_OPT_SAMPLER_DEVICE: [-1, 3], pkg.MCD_OPT_HV_CACHE: [-1, 3],
           pkg.MCD_OPT_HASH_ITEM: [0, 32, 63, 100, 8192], pkg.MCD_OPT_APPLY_SYNC: [-1, 2],
           pkg.MCD_OPT_WAIT_TEST: [-2], pkg.MCD_OPT_KRYLOV_STORE: [-1, 2],
           pkg.MCD_OPT_HV_COLS: [-1, 3], pkg.MCD_OPT_BATCH_SPLIT: [-1, 3, 8],
           pkg.MCD_OPT_BATCH_MODE: [-1, 2], 999: [0]}
    for opt, vals in ok.items():
        for v in vals:
            ctx.mcd_set_option(opt, v)
    for opt, vals in bad.items():
        for v in vals:
            with pytest.raises(pkg.MCDError) as e:
                ctx.mcd_set_option(opt, v)
            assert e.value.status == -1, (opt, v)


def test_device_work_on_a_host_context():
    w = C.ring8_u4()
    ctx = host_ctx(w)
    ctx.mcd_set_basis(np.array([w.seed_word()], dtype=np.uint64))
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_lanczos_ground(10, 1e-6, 0, pkg.MCD_F64)
    assert e.value.status == -9
    assert ctx.mcd_hv_cache_info() == {"bytes": 0, "n_conn": 0, "rec_bytes": 0, "wait_errors": 0}


def test_every_status_code_has_its_own_string():
    import re
    text = open(pkg.HEADER).read()
    enum = text[text.index("typedef enum {"):text.index("} mcd_status;")]
    codes = {name: int(v) for name, v in re.findall(r"(MCD_[A-Z_]+)\s*=\s*(-?\d+)", enum)}
    assert codes["MCD_OK"] == 0 and len(codes) == 11
    L_ = pkg.lib()
    strings = {c: L_.mcd_status_string(c) for c in codes.values()}
    assert b"unknown status" not in strings.values()
    assert len(set(strings.values())) == len(codes)
    assert L_.mcd_status_string(min(codes.values()) - 1) == b"unknown status"
    assert L_.mcd_status_string(max(codes.values()) + 1) == b"unknown status"
