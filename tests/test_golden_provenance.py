"""The stored expected values come from the oracle: the ring entries of
tests/golden/oracle_values.json are recomputed here, on the same inputs, with
the same oracle calls that tests/golden/make_golden.py makes (the larger
entries take minutes and are left to that script)."""
import json
import os

from oracle import fock, hamiltonian as H, lanczos as LZ, sampler as S
from workloads import configs as C

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_values.json")


def test_ring_entries_recomputed():
    g = json.load(open(GOLD))
    w = C.ring8_u4()
    M = H.Model(w.n_sites, w.lat.t, w.eps, w.U_sites)
    # energies to the last few bits (dense eigensolvers may round differently
    # on other BLAS builds); the count of nonzeros exactly
    assert abs(LZ.dense_ground(H.build(M, fock.sector(8, 4, 4)).dense())[0] - g["ring8_full_E0"]) <= 1e-12 * 8
    B = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, w.n_f, w.beta, [w.seed_word()], seed=w.seed)
    P = H.build(M, B)
    assert P.nnz_offdiag() == g["ring8_mc_nnz"]
    assert abs(LZ.dense_ground(P.dense())[0] - g["ring8_mc_E0"]) <= 1e-12 * 8
