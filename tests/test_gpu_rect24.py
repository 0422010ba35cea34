"""The 6x4 t-t' cluster (24 sites, 11 + 11 electrons: words above 32 bits,
4-byte record items and the n > 16 lookups) end to end on the device:

- the band-Lanczos Green function of its spin-up orbitals (48 start vectors:
  c^dag and c on every site) on a nested 5000-state prefix of its Monte Carlo
  basis against the oracle's block-Krylov G from the oracle's own ground
  state, fp64 and fp32 vectors (App. C; w_t inside a gap between weights);
- at the full 5e7-state basis, fp32 vectors with fp64 Gram-Schmidt: the
  excited-space sizes, the 1/z tail (anticommutator sum rule), the sign of
  Im G(i omega_n) and a non-negative spectral function;
- at the full basis, dE0/d(t, t', U) from the Hellmann-Feynman adjoint against
  fourth-order central finite differences of the device E0."""
import numpy as np
import pytest
import torch

import paper_2509_22975_gb300 as pkg
from paper_2509_22975_gb300 import autograd as AG
from oracle import green as G, hamiltonian as H, lanczos as LZ
from workloads import configs as C, lattice as L

from gpu_common import device_ctx, model

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()


def gap_w_t(psi, near):
    """w_t inside a gap between distinct weights of psi, at or above `near`."""
    p = np.sort((psi / np.linalg.norm(psi)) ** 2)[::-1]
    cum = np.cumsum(p)
    k0 = max(int(np.searchsorted(cum, near * cum[-1])), 1)
    k = next(k for k in range(k0, len(p) - 1) if p[k] > 1.001 * p[k + 1])
    return float((cum[k - 1] + 0.5 * p[k]) / cum[-1])


@pytest.mark.parametrize("dtype,tol", [(pkg.MCD_F64, 1e-9), (pkg.MCD_F32, 1e-5)])
def test_prefix_green_matches_oracle(dtype, tol):
    w = C.rect24_u8()
    ctx = device_ctx(w, nf=5000)
    B = ctx.mcd_get_basis()
    M = model(w)
    A = H.build(M, B).sparse()
    ref_gs = LZ.lanczos(lambda v: A @ v, len(B), max_iter=1500, tol=1e-13, seed=0, want_vector=True)
    psi = torch.empty(len(B), dtype=torch.float64 if dtype == pkg.MCD_F64 else torch.float32, device=DEV)
    r = ctx.mcd_lanczos_ground(1500, 1e-13 if dtype == pkg.MCD_F64 else 1e-7, 0, dtype, psi=psi,
                               allow_not_converged=True)
    assert abs(r["E0"] - ref_gs.E0) < (1e-10 * abs(ref_gs.E0) if dtype == pkg.MCD_F64 else 1e-6)
    w_t = gap_w_t(ref_gs.psi, 0.999)
    orb = [(i, 0) for i in range(24)]
    z = 1j * (2 * np.arange(16) + 1) * np.pi / 50.0
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, 12, w_t, z, dtype=dtype)
    ref = G.green(M, B, ref_gs.psi, ref_gs.E0, orb, 12, w_t, z)
    assert dp == ref.plus.dim and dm == ref.minus.dim
    err = np.max(np.abs(Gg - ref.G)) / np.max(np.abs(ref.G))
    print(f"6x4 prefix, {'fp32' if dtype else 'fp64'}: dims {dp} {dm}, max |G - G_oracle| / max |G| = {err:.3e}")
    assert err < tol


@pytest.mark.slow
def test_full_basis_green_sum_rules():
    w = C.rect24_u8()
    ctx = device_ctx(w)
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    assert n == 50_000_000
    r = ctx.mcd_lanczos_ground(600, 1e-7, 0, pkg.MCD_F32, allow_not_converged=True)
    assert r["residual"] < 1e-3 * abs(r["E0"])
    orb = [(i, 0) for i in range(24)]
    wn = (2 * np.arange(64) + 1) * np.pi / 50.0
    z = np.concatenate([1j * wn, np.linspace(-8, 8, 33) + 0.1j, [1e7j]])
    Gg, dp, dm = ctx.mcd_band_lanczos_green(orb, 20, 0.999, z, dtype=pkg.MCD_F32)
    print(f"6x4 full basis: |F+| = {dp}, |F-| = {dm}, E0 = {r['E0']:.10f}")
    assert dp > n // 100 and dm > n // 100
    assert np.max(np.abs(z[-1] * Gg[-1] - np.eye(24))) < 1e-4        # sum rule: z G(z) -> 1
    d = np.einsum("zaa->za", Gg[:64])
    assert np.all(d.imag < 0)                                          # Im G_mu mu(i w_n) < 0 for w_n > 0
    Gr = Gg[64:97]
    A = -np.imag(np.einsum("zaa->z", Gr)) / np.pi
    assert np.all(A > -1e-6 * np.max(A))                               # spectral function >= 0


@pytest.mark.slow
def test_full_basis_E0_adjoint_t_tprime_U():
    w = C.rect24_u8()
    ctx = device_ctx(w)

    def lattice_t(tv, tpv):
        return L.superlattice_cluster((6, 0), (0, 4), t=tv, tp=tpv).t

    t_nn = L.superlattice_cluster((6, 0), (0, 4), t=1.0, tp=0.0).t != 0
    t_nnn = L.superlattice_cluster((6, 0), (0, 4), t=0.0, tp=1.0).t != 0
    f64 = torch.float64
    T = torch.tensor(lattice_t(1.0, -0.3), requires_grad=True)
    eps = torch.zeros(24, dtype=f64, requires_grad=True)
    U = torch.tensor(8.0, dtype=f64, requires_grad=True)
    E = AG.ground_energy(ctx, T, eps, U, max_iter=1500, tol=1e-12)
    E.backward()
    g = T.grad.numpy()
    grads = {"t": -0.5 * np.sum(g[t_nn]), "tp": -0.5 * np.sum(g[t_nnn]), "U": U.grad.item()}

    def E0(tv, tpv, uv):
        return float(AG.ground_energy(ctx, torch.tensor(lattice_t(tv, tpv), dtype=f64), torch.zeros(24, dtype=f64),
                                      torch.tensor(uv, dtype=f64), max_iter=1500, tol=1e-12))

    h = 1e-3
    base = {"t": 1.0, "tp": -0.3, "U": 8.0}
    for k in ("t", "tp", "U"):
        def at(d):
            p = dict(base)
            p[k] += d
            return E0(p["t"], p["tp"], p["U"])
        fd = (at(-2 * h) - 8 * at(-h) + 8 * at(h) - at(2 * h)) / (12 * h)
        print(f"dE0/d{k}: adjoint {grads[k]:.10f}, finite differences {fd:.10f}")
        assert abs(fd - grads[k]) < 1e-6, (k, fd, grads[k])
