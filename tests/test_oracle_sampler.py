"""Pins of the oracle's Monte Carlo sampler: the generator's published outputs,
the acceptance probability of the Boltzmann-factor Eq. measured empirically,
exhaustive coverage at beta = 0 against a brute-force graph search, and the
structural invariants of the step rule (sector, order, size, nesting)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import fock, sampler as S
from workloads import configs as C, lattice as L

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_splitmix64_published_outputs():
    g = json.load(open(os.path.join(GOLD, "splitmix64.json")))
    for s in g["streams"]:
        out = S.splitmix64_stream(s["seed"], len(s.get("outputs", s.get("outputs_hex", []))))
        if "outputs" in s:
            assert out == s["outputs"]
        else:
            assert [f"{x:016x}" for x in out] == s["outputs_hex"]
    # vectorised mix agrees with the scalar one
    zs = np.array([1, 2, 3, 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    assert [int(v) for v in S.mix64(zs)] == [S.mix64_int(int(z)) for z in zs]


def test_acceptance_probability_matches_boltzmann_factor():
    # Proposals of children with n_U = 0..3 at beta U = 1.6 are accepted at
    # rate exp(-1.6 n_U) (min with 1): check with many independent draws.
    n, U, beta = 8, 8.0, 0.2
    lat = L.ring(n)
    Uv = np.full(n, U)
    words = {}
    for w in fock.sector(n, 4, 4):
        k = int(fock.double_occupancy(np.array([w], dtype=np.uint64), n)[0])
        words.setdefault(k, w)
    parents = np.arange(1, 200001, dtype=np.uint64) * np.uint64(2654435761)
    for k, child in sorted(words.items()):
        if k > 3:
            continue
        p = S.acceptance(np.array([child], dtype=np.uint64), n, Uv, beta)[0]
        assert p == min(math.exp(-U * beta * k), 1.0)
        u = (S.draw(7, 3, parents, 5) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        rate = float(np.mean(u < p))
        sd = math.sqrt(max(p * (1 - p), 1e-12) / len(parents))
        assert abs(rate - p) < 5 * sd + 1e-12


def brute_component(n, t, n_up, n_dn, seed_word):
    """All sector states reachable from seed_word by hops (plain BFS on sets)."""
    seen = {seed_word}
    todo = [seed_word]
    while todo:
        w = todo.pop()
        for spin in (0, 1):
            for i in range(n):
                for j in range(n):
                    if i != j and t[i, j] != 0:
                        h = fock.hop_word(w, n, spin, i, j)
                        if h is not None and h[0] not in seen:
                            seen.add(h[0])
                            todo.append(h[0])
    return sorted(seen)


def test_beta_zero_covers_the_sector():
    w = C.ring8_u4()
    F = S.sample_basis(8, w.lat.t, w.U_sites, 4, 4, 4900, 0.0, [w.seed_word()], seed=1)
    assert np.array_equal(F, fock.sector(8, 4, 4))


def test_disconnected_lattice_stops_at_the_component():
    # two 3-site rings with no bond between them: the reachable set is a
    # proper subset of the sector; the sampler must stop there.
    t = np.zeros((6, 6))
    for a, b in [(0, 1), (1, 2), (2, 0), (3, 4), (4, 5), (5, 3)]:
        t[a, b] = t[b, a] = -1.0
    seed = (0b000011 << 6) | 0b011000
    comp = brute_component(6, t, 2, 2, seed)
    F = S.sample_basis(6, t, np.full(6, 4.0), 2, 2, 225, 0.0, [seed], seed=0)
    assert len(comp) < 225
    assert [int(x) for x in F] == comp


@pytest.mark.parametrize("name", ["ring8", "tilted12"])
def test_invariants_determinism_nesting(name):
    w = C.WORKLOADS[name]()
    nf = min(w.n_f, 3000)
    args = (w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn)
    F = S.sample_basis(*args, nf, w.beta, [w.seed_word()], seed=w.seed)
    assert len(F) == nf
    assert np.all(F[1:] > F[:-1])
    up, dn = fock.split(F, w.n_sites)
    assert np.all(fock.popcount(up) == w.n_up) and np.all(fock.popcount(dn) == w.n_dn)
    assert np.uint64(w.seed_word()) in F
    F2 = S.sample_basis(*args, nf, w.beta, [w.seed_word()], seed=w.seed)
    assert np.array_equal(F, F2)
    Fo = S.sample_basis(*args, nf, w.beta, [w.seed_word()], seed=w.seed + 1)
    assert not np.array_equal(F, Fo)
    small = S.sample_basis(*args, nf // 3, w.beta, [w.seed_word()], seed=w.seed)
    assert np.all(np.isin(small, F))


def test_low_double_occupancy_is_favoured():
    # With U beta = 1.6 the sampled basis is enriched in low n_U compared
    # with the sector (the paper's premise, Figs. 1-2).
    w = C.ring8_u4()
    F = S.sample_basis(8, w.lat.t, w.U_sites, 4, 4, 2000, w.beta, [w.seed_word()], seed=0)
    full = fock.sector(8, 4, 4)
    assert fock.double_occupancy(F, 8).mean() < fock.double_occupancy(full, 8).mean()
