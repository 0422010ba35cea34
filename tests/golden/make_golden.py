"""Write tests/golden/oracle_values.json from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Every value comes from oracle/ (fp64) on inputs described by workloads/.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import fock, hamiltonian as H, lanczos as LZ, sampler as S  # noqa: E402
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


if __name__ == "__main__":
    main()
