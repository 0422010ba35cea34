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


def test_green_prefix_entries_recomputed():
    # tests/golden/green_tilted12_prefix.json: the same oracle calls as
    # `make_golden.py green` (about half a minute of CPU)
    import importlib.util

    import numpy as np
    spec = importlib.util.spec_from_file_location(
        "make_golden", os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    g = json.load(open(os.path.join(os.path.dirname(GOLD), "green_tilted12_prefix.json")))
    from oracle import green as G
    w = C.tilted12_u8()
    w.mu = w.U / 2
    B = mg.mc_basis(w, g["n_f"])
    M = mg.model(w)
    r = mg.ground(H.build(M, B))
    assert abs(r.E0 - g["E0"]) <= 1e-11 * abs(g["E0"])
    assert abs(mg.gap_w_t(r.psi, 0.999) - g["w_t"]) < 1e-12
    wn = (2 * np.arange(g["n_matsubara"]) + 1) * np.pi / g["beta_M"]
    res = G.green(M, B, r.psi, r.E0, [(i, 0) for i in range(12)], g["n_blocks"], g["w_t"], 1j * wn)
    assert (res.plus.dim, res.minus.dim, len(res.keep)) == (g["dim_plus"], g["dim_minus"], g["kept"])
    d = np.einsum("zaa->za", res.G)
    ref = np.asarray(g["G_diag_re"]) + 1j * np.asarray(g["G_diag_im"])
    assert np.max(np.abs(d - ref)) <= 1e-10 * np.max(np.abs(ref))
