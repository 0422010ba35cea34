"""Input recipes.  Lattice workloads: bond counts, fillings, and the
eigenvalues of each cluster's hopping matrix equal to the square-lattice
dispersion -2t (cos kx + cos ky) - 4t' cos kx cos ky at the cluster's momenta
(the ring: -2 cos k).  Batched impurity workload: every instance has the stated
structure and parameter ranges, is reproducible from its seed, and its seed
state is the smallest word among the states with up and down electrons on
complementary sites, which all share the diagonal energy sum(eps)."""
import itertools

import numpy as np

from oracle import fock
from workloads import impurity as IM


def test_instances_follow_the_recipe():
    for k in range(32):
        m = IM.impurity(k)
        n, c = IM.N_SITES, IM.N_CLUSTER
        assert m.t.shape == (n, n) and np.array_equal(m.t, m.t.T) and np.all(np.diag(m.t) == 0)
        cl = np.zeros((c, c))
        for i, j in IM.PLAQUETTE:
            cl[i, j] = cl[j, i] = -1.0
        assert np.array_equal(m.t[:c, :c], cl)                       # open 2x2 plaquette, t = 1
        assert np.all(m.t[c:, c:] == 0)                               # bath sites not coupled to each other
        assert np.all(m.t[:c, c:] != 0)                               # every bath site hybridised with every cluster site
        assert 2.0 <= m.U <= 8.0
        assert np.all(m.U_sites[:c] == m.U) and np.all(m.U_sites[c:] == 0)
        assert np.all(m.eps[:c] == -m.U / 2) and np.all(np.abs(m.eps[c:]) <= 2.0)
        assert 1000 <= m.n_f <= 100000 and abs(m.beta * m.U - 1.6) < 1e-12
        assert (m.n_up, m.n_dn) == (6, 6)
        again = IM.impurity(k)
        assert np.array_equal(again.t, m.t) and np.array_equal(again.eps, m.eps) and again.n_f == m.n_f
    assert len({IM.impurity(k).U for k in range(32)}) == 32        # instances differ


def test_seed_state_is_the_smallest_equal_energy_word():
    m = IM.impurity(5)
    n = m.n_sites
    full = (1 << n) - 1
    words = []
    for sites in itertools.combinations(range(n), m.n_up):
        up = sum(1 << i for i in sites)
        words.append((up << n) | (full ^ up))
    words = np.array(sorted(words), dtype=np.uint64)
    assert len(words) == 924
    d = fock.diagonal(words, n, m.eps, m.U_sites)
    assert np.allclose(d, m.eps.sum(), rtol=0, atol=1e-12)
    assert np.all(fock.double_occupancy(words, n) == 0)
    seed = np.uint64(m.seed_word())
    assert seed == words[0]
    up, dn = fock.split(np.array([seed]), n)
    assert fock.popcount(up)[0] == m.n_up and fock.popcount(dn)[0] == m.n_dn


def _bloch(lat, t, tp):
    """Single-particle energies of a periodic square-lattice cluster from the
    dispersion -2t (cos kx + cos ky) - 4t' cos kx cos ky over the cluster's
    momenta k (k . R1 and k . R2 multiples of 2 pi)."""
    M = np.array([lat.notes["R1"], lat.notes["R2"]], dtype=np.float64)
    n = lat.n_sites
    ks = {}
    for p in range(n):
        for q in range(n):
            k = 2 * np.pi * np.linalg.solve(M, [p, q])
            key = tuple(np.round(np.mod(k, 2 * np.pi), 9) % np.round(2 * np.pi, 9))
            ks.setdefault(key, k)
    assert len(ks) == n
    return np.sort([-2 * t * (np.cos(kx) + np.cos(ky)) - 4 * tp * np.cos(kx) * np.cos(ky)
                    for kx, ky in ks.values()])


def test_cluster_hoppings_match_the_dispersion():
    from workloads import configs as C
    expect = {"ring8": (8, 8), "tilted12": (12, 24), "square16": (16, 64), "rect24": (24, 96)}
    for name, make in C.WORKLOADS.items():
        w = make()
        n, bonds = expect[name]
        assert w.n_sites == n and np.count_nonzero(np.triu(w.lat.t, 1)) == bonds
        ev = np.linalg.eigvalsh(w.lat.t)
        if name == "ring8":
            ref = np.sort(-2 * np.cos(2 * np.pi * np.arange(8) / 8))
        else:
            ref = _bloch(w.lat, w.lat.notes["t"], w.lat.notes["tp"])
        assert np.allclose(ev, ref, atol=1e-12), name
    assert (C.square16_u8().n_up, C.rect24_u8().n_up, C.tilted12_u8().n_up, C.ring8_u4().n_up) == (7, 11, 6, 4)
