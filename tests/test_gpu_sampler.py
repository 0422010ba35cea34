"""Device Monte Carlo sampler through the C ABI: the same basis, word for word,
as the host sampler and the oracle, for every workload, both frontier rules,
an overshooting last step, a run that stops early, U on a subset of sites
(an impurity cluster), 32 sites; the option's errors; and the 6x4 basis of
5e7 states at full size."""
import numpy as np
import pytest

import paper_2509_22975_gb300 as pkg
from oracle import fock, sampler as S
from workloads import configs as C, lattice as L

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def sample(w, nf, where, flags=0, t=None, U=None, seeds=None, seed=None, beta=None):
    ctx = pkg.Context(0)
    t = w.lat.t if t is None else t
    U = w.U if U is None else U
    ctx.mcd_set_hamiltonian(t, w.eps, U, w.n_up, w.n_dn)
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, where)
    st, _ = ctx.mcd_build_basis(w.seed if seed is None else seed, nf, w.beta if beta is None else beta,
                                seeds or [w.seed_word()], flags=flags)
    return ctx.mcd_get_basis(), st


@pytest.mark.parametrize("name,nf", [("ring8_u4", 2000), ("tilted12_u8", 1 << 18), ("square16_u8", 300000),
                                     ("rect24_u8", 400000)])
@pytest.mark.parametrize("flags", [0, pkg.MCD_SAMPLE_NEW_ONLY])
def test_device_equals_host(name, nf, flags):
    w = getattr(C, name)()
    Bd, sd = sample(w, nf, pkg.SAMPLER_DEVICE, flags)
    Bh, sh = sample(w, nf, pkg.SAMPLER_HOST, flags)
    assert sd == sh
    assert np.array_equal(Bd, Bh)
    if sd == 0:
        assert len(Bd) == nf


def test_device_equals_oracle():
    w = C.ring8_u4()
    Bd, _ = sample(w, 2000, pkg.SAMPLER_DEVICE)
    Bo = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, 2000, w.beta, [w.seed_word()], seed=w.seed)
    assert np.array_equal(Bd, Bo)


@pytest.mark.parametrize("name,nf", [("rect24_u8", 30000), ("rect24_u8", 120000), ("square16_u8", 100000)])
@pytest.mark.parametrize("flags", [0, pkg.MCD_SAMPLE_NEW_ONLY])
def test_device_and_host_equal_oracle_beyond_16_sites(name, nf, flags):
    # the 24-site cluster (words above 32 bits, n > 16 sites) and the 4x4 one:
    # both library samplers against the oracle, word for word
    w = getattr(C, name)()
    Bo = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, nf, w.beta, [w.seed_word()], seed=w.seed,
                        flags=flags)
    for where in (pkg.SAMPLER_DEVICE, pkg.SAMPLER_HOST):
        B, st = sample(w, nf, where, flags)
        assert st == 0 and len(B) == nf
        assert np.array_equal(B, Bo)


def test_overshoot_and_nesting():
    # every size cuts some step short: the device keeps the same states of
    # smallest priority as the host, and smaller bases are prefixes in set terms
    w = C.tilted12_u8()
    prev = None
    for nf in (1000, 1001, 5003, 40000):
        Bd, _ = sample(w, nf, pkg.SAMPLER_DEVICE)
        Bh, _ = sample(w, nf, pkg.SAMPLER_HOST)
        assert np.array_equal(Bd, Bh) and len(Bd) == nf
        if prev is not None:
            assert np.all(np.isin(prev, Bd))
        prev = Bd


def test_short_run_on_disconnected_lattice():
    # two disconnected 3-site rings: the reachable set is smaller than asked
    n = 6
    t = np.zeros((n, n))
    for a, b in [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3)]:
        t[a, b] = t[b, a] = -1.0
    lat = L.Lattice("two_rings", n, t, np.zeros((n, 2), int), np.arange(n) % 2)
    w = C.Workload("two_rings", lat, 4.0, 2, 2, 0, 0.0)
    seedw = (np.uint64(0b000011) << np.uint64(n)) | np.uint64(0b000011)
    Bd, sd = sample(w, 200, pkg.SAMPLER_DEVICE, seeds=[int(seedw)])
    Bh, sh = sample(w, 200, pkg.SAMPLER_HOST, seeds=[int(seedw)])
    assert sd == sh == 1 and np.array_equal(Bd, Bh) and len(Bd) < 200


def test_u_on_cluster_sites_only():
    # impurity-like Hamiltonian: U on 4 of 12 sites, 0 elsewhere
    w = C.tilted12_u8()
    U = np.zeros(12)
    U[[0, 3, 5, 8]] = 6.0
    Bd, sd = sample(w, 30000, pkg.SAMPLER_DEVICE, U=U)
    Bh, sh = sample(w, 30000, pkg.SAMPLER_HOST, U=U)
    assert sd == sh and np.array_equal(Bd, Bh)
    Bo = S.sample_basis(12, w.lat.t, U, w.n_up, w.n_dn, 30000, w.beta, [w.seed_word()], seed=w.seed)
    assert np.array_equal(Bd, Bo)


def test_thirty_two_sites():
    n = 32
    rng = np.random.default_rng(8)
    t = np.zeros((n, n))
    for _ in range(60):
        i, j = rng.choice(n, 2, replace=False)
        t[i, j] = t[j, i] = rng.normal()
    lat = L.Lattice("rand32", n, t, np.zeros((n, 2), int), np.arange(n) % 2)
    w = C.Workload("rand32", lat, 3.0, 3, 2, 0, 0.5)
    seedw = (np.uint64(0b111 << 29) << np.uint64(32)) | np.uint64(0b11)
    Bd, _ = sample(w, 20000, pkg.SAMPLER_DEVICE, seeds=[int(seedw)], seed=1)
    Bh, _ = sample(w, 20000, pkg.SAMPLER_HOST, seeds=[int(seedw)], seed=1)
    assert np.array_equal(Bd, Bh)


def test_option_errors():
    w = C.ring8_u4()
    ctx = pkg.Context(0)
    U = np.linspace(1.0, 4.0, 8)      # two different nonzero U_i: host only
    ctx.mcd_set_hamiltonian(w.lat.t, np.zeros(8), U, 4, 4)
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, pkg.SAMPLER_DEVICE)
    with pytest.raises(pkg.MCDError):
        ctx.mcd_build_basis(0, 100, 0.4, [w.seed_word()])
    ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, pkg.SAMPLER_AUTO)   # falls to host threads
    ctx.mcd_build_basis(0, 100, 0.4, [w.seed_word()])
    assert len(ctx.mcd_get_basis()) == 100
    with pytest.raises(pkg.MCDError):
        ctx.mcd_set_option(pkg.MCD_OPT_SAMPLER_DEVICE, 3)


@pytest.mark.slow
def test_rect24_full_size():
    w = C.rect24_u8()
    Bd, sd = sample(w, w.n_f, pkg.SAMPLER_DEVICE)
    Bh, sh = sample(w, w.n_f, pkg.SAMPLER_HOST)
    assert sd == sh == 0 and len(Bd) == w.n_f
    assert np.array_equal(Bd, Bh)
