"""GPU band-Lanczos Green function through the C ABI against the oracle's
block-Krylov projection from the oracle's own ground state: same truncation
(w_t = 1, or w_t inside a gap between weights), excited spaces and Krylov
space, so G(z) agrees; the 12-site workload's 150 blocks on a nested prefix
of its basis against stored oracle values; fp32 vectors (and the fp32 ground
state) against the oracle; the anticommutator sum rule through the 1/z tail;
the dense Lehmann sum once the Krylov space is exhausted; argument and state
errors; the 12-site configuration at full size."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from oracle import fock, green as G, hamiltonian as H, lanczos as LZ, sampler as S
from workloads import configs as C, lattice as L

from gpu_common import device_ctx, model

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def ring8_half_filled(nf=2000):
    w = C.ring8_u4()
    w.mu = w.U / 2          # particle-hole symmetric point
    return w


def gpu_ground(ctx, n, dtype=pkg.MCD_F64):
    psi = torch.empty(n, dtype=torch.float64 if dtype == pkg.MCD_F64 else torch.float32, device=DEV)
    r = ctx.mcd_lanczos_ground(600, 1e-13 if dtype == pkg.MCD_F64 else 1e-7, 0, dtype, psi=psi,
                               allow_not_converged=True)
    return r, psi.double().cpu().numpy()


def gap_w_t(psi, near):
    """A target weight inside a gap between distinct weights of psi, at or
    above `near` (the kept set is then the same for the device's and the
    oracle's ground states, which agree far below the gap)."""
    p = np.sort((psi / np.linalg.norm(psi)) ** 2)[::-1]
    cum = np.cumsum(p)
    k0 = max(int(np.searchsorted(cum, near * cum[-1])), 1)
    k = next(k for k in range(k0, len(p) - 1) if p[k] > 1.001 * p[k + 1])
    return float((cum[k - 1] + 0.5 * p[k]) / cum[-1])


@pytest.mark.parametrize("w_t,n_blocks", [(1.0, 8), (1.0, 25), ("gap0.95", 12), ("gap0.999", 30)])
def test_matches_oracle_block_krylov(w_t, n_blocks):
    # the oracle works from its own dense ground state (not the device's):
    # truncation, F~+-, start vectors and the block Krylov space all follow
    # from an independently computed Omega~ (G is even in the sign of Omega~)
    w = ring8_half_filled()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    r, psi = gpu_ground(ctx, len(B))
    M = model(w)
    E_ref, v_ref, _ = LZ.dense_ground(H.build(M, B).dense())
    assert abs(r["E0"] - E_ref) < 1e-11 * abs(E_ref)
    if isinstance(w_t, str):
        w_t = gap_w_t(v_ref, float(w_t[3:]))
    orb = [(i, 0) for i in range(8)]
    z = np.linspace(-8, 8, 17) + 0.25j
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, n_blocks, w_t, z)
    ref = G.green(M, B, v_ref, E_ref, orb, n_blocks, w_t, z)
    assert dp == ref.plus.dim and dm == ref.minus.dim
    scale = np.max(np.abs(ref.G))
    assert np.max(np.abs(Gg - ref.G)) < 1e-7 * scale, np.max(np.abs(Gg - ref.G)) / scale


def test_exhausted_krylov_and_sum_rule():
    # small full sector: enough blocks to exhaust the Krylov space; compare
    # with the dense Lehmann sum, and z G(z) -> identity (anticommutator)
    n, U = 6, 4.0
    lat = L.ring(n)
    w = C.Workload("ring6", lat, U, 3, 3, 0, 0.4, mu=U / 2)
    Bf = fock.sector(6, 3, 3)
    ctx = device_ctx(w, basis=Bf)
    r, psi = gpu_ground(ctx, len(Bf))
    M = model(w)
    E_ref, v_ref, _ = LZ.dense_ground(H.build(M, Bf).dense())
    orb = [(i, 0) for i in range(n)]
    z = np.linspace(-6, 6, 25) + 0.1j
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, 80, 1.0, z)
    ex = G.green(M, Bf, v_ref, E_ref, orb, 0, 1.0, z, exact=True)
    assert np.max(np.abs(Gg - ex.G)) < 1e-8 * np.max(np.abs(ex.G))
    Gt, _, _ = ctx.mcd_band_lanczos_green(orb, 80, 1.0, np.array([1e7j]))
    assert np.max(np.abs(1e7j * Gt[0] - np.eye(n))) < 1e-6
    A = G.dos(Gg)
    assert np.max(np.abs(A - A[::-1])) < 1e-8 * np.max(A)    # particle-hole symmetry


@pytest.mark.parametrize("ground_dtype", [pkg.MCD_F64, pkg.MCD_F32])
def test_fp32_vectors_against_the_oracle(ground_dtype):
    # fp32 Krylov vectors (fp64 Gram-Schmidt and coefficients) against the
    # oracle's fp64 G from its own dense ground state; with the fp32 ground
    # state too (the whole fp32 form): E0 within 1e-6 and G within 1e-5 of
    # the largest |G| (measured 2e-7 and 4e-7: fp32 rounding of the Krylov
    # vectors, u = 6e-8, grown by the recursion)
    w = ring8_half_filled()
    ctx = device_ctx(w)
    B = ctx.mcd_get_basis()
    r, psi = gpu_ground(ctx, len(B), ground_dtype)
    M = model(w)
    E_ref, v_ref, _ = LZ.dense_ground(H.build(M, B).dense())
    assert abs(r["E0"] - E_ref) < (1e-6 if ground_dtype == pkg.MCD_F32 else 1e-11 * abs(E_ref))
    orb = [(i, 0) for i in range(8)]
    z = np.linspace(-8, 8, 17) + 0.25j
    G32, dp, dm = ctx.mcd_band_lanczos_green(orb, 20, 1.0, z, dtype=pkg.MCD_F32)
    ref = G.green(M, B, v_ref, E_ref, orb, 20, 1.0, z)
    assert dp == ref.plus.dim and dm == ref.minus.dim
    err = np.max(np.abs(G32 - ref.G)) / np.max(np.abs(ref.G))
    print(f"fp32 G vs oracle (ground state {'fp32' if ground_dtype else 'fp64'}): {err:.3e}, "
          f"|dE0| = {abs(r['E0'] - E_ref):.3e}")
    assert err < 1e-5


def tilted12_prefix_golden():
    import json
    import os
    return json.load(open(os.path.join(os.path.dirname(__file__), "golden", "green_tilted12_prefix.json")))


@pytest.mark.parametrize("dtype,tol", [(pkg.MCD_F64, 1e-10), (pkg.MCD_F32, 1e-5)])
def test_tilted12_prefix_150_blocks_matches_oracle(dtype, tol):
    # the 12-site Green-function workload (12 spin-up orbitals, 150 blocks,
    # w_t in the gap nearest above 0.999) on the nested 2e4-state prefix of its
    # Monte Carlo basis, against the oracle's G(i omega_n) at beta_M = 50,
    # n = 0..63 (stored by tests/golden/make_golden.py from the oracle's own
    # Lanczos ground state and block Krylov space, full reorthogonalisation)
    gold = tilted12_prefix_golden()
    w = C.tilted12_u8()
    w.mu = w.U / 2
    ctx = device_ctx(w, nf=gold["n_f"])
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    assert n == gold["n_basis"]
    r, _ = gpu_ground(ctx, n, dtype)
    assert abs(r["E0"] - gold["E0"]) < (1e-6 if dtype == pkg.MCD_F32 else 1e-10 * abs(gold["E0"]))
    wn = (2 * np.arange(gold["n_matsubara"]) + 1) * np.pi / gold["beta_M"]
    orb = [(i, 0) for i in range(12)]
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, gold["n_blocks"], gold["w_t"], 1j * wn, dtype=dtype)
    assert dp == gold["dim_plus"] and dm == gold["dim_minus"]
    ref = np.asarray(gold["G_diag_re"]) + 1j * np.asarray(gold["G_diag_im"])
    got = np.einsum("zaa->za", Gg)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    print(f"tilted12 prefix, {'fp32' if dtype else 'fp64'}: max |G - G_oracle| / max |G_oracle| = {err:.3e}, "
          f"|dE0| = {abs(r['E0'] - gold['E0']):.3e}")
    assert err < tol


def test_spin_down_orbitals_and_errors():
    w = ring8_half_filled()
    ctx = device_ctx(w, nf=600)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_band_lanczos_green([(0, 0)], 4, 1.0, [1j])
    assert e.value.status == -8                      # no ground state yet
    B = ctx.mcd_get_basis()
    r, psi = gpu_ground(ctx, len(B))
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_band_lanczos_green([(0, 0), (1, 1)], 4, 1.0, [1j])   # mixed spins
    assert e.value.status == -1
    with pytest.raises(pkg.MCDError):
        ctx.mcd_band_lanczos_green([(9, 0)], 4, 1.0, [1j])            # site out of range
    M = model(w)
    E_ref, v_ref, _ = LZ.dense_ground(H.build(M, B).dense())
    orb = [(1, 1), (4, 1)]
    z = np.array([0.3 + 0.2j, -1.0 + 0.5j])
    Gg, _, _ = ctx.mcd_band_lanczos_green(orb, 15, 1.0, z)
    ref = G.green(M, B, psi, r["E0"], orb, 15, 1.0, z)
    assert np.max(np.abs(Gg - ref.G)) < 1e-7 * np.max(np.abs(ref.G))


@pytest.mark.slow
def test_tilted12_full_size():
    # the 12-site configuration: 2^18-state MC basis, 12 spin-up orbitals,
    # w_t = 0.999, 150 band iterations in each excited space
    w = C.tilted12_u8()
    w.mu = w.U / 2
    ctx = device_ctx(w)
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    r, psi = gpu_ground(ctx, n)
    orb = [(i, 0) for i in range(12)]
    omega = np.linspace(-10, 10, 201)
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, 150, 0.999, omega + 0.05j)
    A = G.dos(Gg)
    assert np.all(A > -1e-9)
    Gt, _, _ = ctx.mcd_band_lanczos_green(orb, 150, 0.999, np.array([1e7j]))
    assert np.max(np.abs(1e7j * Gt[0] - np.eye(12))) < 1e-5
    assert dp > n // 10 and dm > n // 10
