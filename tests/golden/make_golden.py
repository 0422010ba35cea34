"""Write the stored oracle values from the oracle alone.

Run from the repository root:
  python tests/golden/make_golden.py          -> tests/golden/oracle_values.json
  python tests/golden/make_golden.py green    -> tests/golden/green_tilted12_prefix.json
Every value comes from oracle/ (fp64) on inputs described by workloads/.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fock, green as G, hamiltonian as H, lanczos as LZ, sampler as S  # noqa: E402
from workloads import configs as C  # noqa: E402


def model(w):
    return H.Model(w.n_sites, w.lat.t, w.eps, w.U_sites)


def mc_basis(w, nf):
    return S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, nf, w.beta,
                          [w.seed_word()], seed=w.seed)


def ground(P, tol=1e-14):
    A = P.sparse()
    r = LZ.lanczos(lambda v: A @ v, P.n, max_iter=2000, tol=tol, want_vector=True)
    return r


def main():
    out = {"_generated_by": "python tests/golden/make_golden.py (oracle/ only, fp64)"}
    # 8-site ring, U = 4, 4 + 4 electrons
    w = C.ring8_u4()
    full = fock.sector(8, 4, 4)
    out["ring8_full_E0"] = LZ.dense_ground(H.build(model(w), full).dense())[0]
    B = mc_basis(w, w.n_f)
    P = H.build(model(w), B)
    out["ring8_mc_E0"] = LZ.dense_ground(P.dense())[0]
    out["ring8_mc_nnz"] = P.nnz_offdiag()
    # tilted 12-site cluster, U = 8, 6 + 6 electrons
    w = C.tilted12_u8()
    P = H.build(model(w), fock.sector(12, 6, 6))
    r = ground(P)
    out["tilted12_full_E0"] = r.E0
    out["tilted12_full_residual"] = r.residual
    B = mc_basis(w, w.n_f)
    P = H.build(model(w), B)
    r = ground(P)
    out["tilted12_mc_E0"] = r.E0
    out["tilted12_mc_residual"] = r.residual
    out["tilted12_mc_nnz"] = P.nnz_offdiag()
    # 4x4 t-t' cluster, 7 + 7 electrons, a 2^16-state MC basis
    w = C.square16_u8()
    B = mc_basis(w, 1 << 16)
    P = H.build(model(w), B)
    r = ground(P)
    out["square16_mc65536_E0"] = r.E0
    out["square16_mc65536_residual"] = r.residual
    out["square16_mc65536_nnz"] = P.nnz_offdiag()
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_values.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


def gap_w_t(psi, near):
    """A target weight inside a gap between distinct weights of psi, at or
    above `near`: the first k from the shortest prefix reaching `near` with
    p_k > 1.001 p_(k+1) (weights sorted descending), w_t halfway into p_k.  The
    kept set is then the same for any ground state that agrees with psi far
    below that gap (a device solve and the oracle's)."""
    p = np.sort((psi / np.linalg.norm(psi)) ** 2)[::-1]
    cum = np.cumsum(p)
    k0 = max(int(np.searchsorted(cum, near * cum[-1])), 1)
    k = next(k for k in range(k0, len(p) - 1) if p[k] > 1.001 * p[k + 1])
    return float((cum[k - 1] + 0.5 * p[k]) / cum[-1])


GREEN_NF = 20000
GREEN_BLOCKS = 150
GREEN_BETA_M = 50.0
GREEN_NZ = 64


def green_main():
    """The 12-site Green-function workload on a nested 2e4-state prefix of its
    Monte Carlo basis (mu = U/2, 12 spin-up orbitals, 150 blocks, w_t in the
    gap nearest above 0.999), G(i omega_n) at beta_M = 50, n = 0..63."""
    w = C.tilted12_u8()
    w.mu = w.U / 2
    B = mc_basis(w, GREEN_NF)
    M = model(w)
    P = H.build(M, B)
    r = ground(P)
    w_t = gap_w_t(r.psi, 0.999)
    orb = [(i, 0) for i in range(w.n_sites)]
    wn = (2 * np.arange(GREEN_NZ) + 1) * np.pi / GREEN_BETA_M
    g = G.green(M, B, r.psi, r.E0, orb, GREEN_BLOCKS, w_t, 1j * wn)
    d = np.einsum("zaa->za", g.G)
    out = {"_generated_by": "python tests/golden/make_golden.py green (oracle/ only, fp64)",
           "workload": "tilted12 U=8 mu=U/2 6+6, MC basis prefix", "n_f": GREEN_NF, "n_basis": int(len(B)),
           "E0": r.E0, "residual": r.residual, "w_t": w_t, "n_blocks": GREEN_BLOCKS,
           "beta_M": GREEN_BETA_M, "n_matsubara": GREEN_NZ,
           "dim_plus": int(g.plus.dim), "dim_minus": int(g.minus.dim),
           "krylov_plus": int(g.plus.krylov_dim), "krylov_minus": int(g.minus.krylov_dim),
           "kept": int(len(g.keep)),
           "G_diag_re": [[float(f"{v:.15g}") for v in row] for row in d.real],
           "G_diag_im": [[float(f"{v:.15g}") for v in row] for row in d.imag]}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "green_tilted12_prefix.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=0)
    print({k: v for k, v in out.items() if not k.startswith("G_")})


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "green":
        green_main()
    else:
        main()
