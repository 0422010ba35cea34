"""Input recipe of the batched impurity workload: every instance has the
stated structure and parameter ranges, is reproducible from its seed, and its
seed state is the smallest word among the states with up and down electrons
on complementary sites, which all share the diagonal energy sum(eps)."""
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
