"""Basis file (mcd_save_basis / mcd_load_basis) on host-only contexts: the
40-byte header and the words as documented, the hash equal to FNV-1a 64 (a
Python restatement pinned to the published test vectors), a round trip that
gives back the same words, and every rejected file with its status code:
missing, short, foreign magic, other version, other sector, size mismatch,
corrupted word, words out of order; no Hamiltonian or no basis."""
import struct

import numpy as np
import pytest

import paper_2509_22975_gb300 as pkg
from workloads import configs as C

HEADER = struct.Struct("<8sIIIIqQ")


def fnv1a64(data: bytes) -> int:
    h = 0xCBF29CE484222325
    for b in data:
        h = ((h ^ b) * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h


@pytest.fixture(scope="module", autouse=True)
def built():
    pkg.build()
    pkg.lib()


def host_ctx(w, n_up=None):
    ctx = pkg.Context(-1)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up if n_up is None else n_up, w.n_dn)
    return ctx


@pytest.fixture(scope="module")
def saved(tmp_path_factory):
    w = C.ring8_u4()
    ctx = host_ctx(w)
    ctx.mcd_build_basis(w.seed, 2000, w.beta, [w.seed_word()])
    B = ctx.mcd_get_basis()
    path = tmp_path_factory.mktemp("basis") / "ring8.mcdb"
    ctx.mcd_save_basis(path)
    return w, B, path, path.read_bytes()


def test_published_fnv1a64_vectors():
    assert fnv1a64(b"") == 0xCBF29CE484222325
    assert fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert fnv1a64(b"foobar") == 0x85944171F73967E8


def test_layout_and_hash(saved):
    w, B, _, raw = saved
    magic, version, ns, nu, nd, n, h = HEADER.unpack_from(raw)
    assert (magic, version, ns, nu, nd, n) == (b"MCDBASIS", 1, w.n_sites, w.n_up, w.n_dn, len(B))
    words = raw[HEADER.size:]
    assert len(words) == 8 * len(B)
    assert np.array_equal(np.frombuffer(words, dtype="<u8"), B)
    assert h == fnv1a64(words)


def test_round_trip(saved, tmp_path):
    w, B, path, _ = saved
    ctx = host_ctx(w)
    ctx.mcd_load_basis(path)
    assert np.array_equal(ctx.mcd_get_basis(), B)
    again = tmp_path / "again.mcdb"
    ctx.mcd_save_basis(again)
    assert again.read_bytes() == path.read_bytes()


def rejected(w, data, tmp_path, status, n_up=None):
    p = tmp_path / "bad.mcdb"
    p.write_bytes(data)
    ctx = host_ctx(w, n_up)
    keep = np.array([w.seed_word()], dtype=np.uint64)
    if n_up is None:
        ctx.mcd_set_basis(keep)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_load_basis(p)
    assert e.value.status == status
    if n_up is None:                      # rejected before the words: the old basis stays
        assert np.array_equal(ctx.mcd_get_basis(), keep)


def test_rejected_files(saved, tmp_path):
    w, B, _, raw = saved
    head, words = raw[:HEADER.size], raw[HEADER.size:]
    magic, version, ns, nu, nd, n, h = HEADER.unpack_from(raw)
    rejected(w, raw[:20], tmp_path, -1)                                            # short header
    rejected(w, HEADER.pack(b"NOTBASIS", version, ns, nu, nd, n, h) + words, tmp_path, -1)
    rejected(w, HEADER.pack(magic, 2, ns, nu, nd, n, h) + words, tmp_path, -1)   # version
    rejected(w, raw[:-8], tmp_path, -1)                                            # size
    rejected(w, HEADER.pack(magic, version, ns, nu, nd, n + 1, h) + words, tmp_path, -1)
    bad = bytearray(raw)
    bad[HEADER.size + 8 * 17 + 1] ^= 0x01                                           # one bit of word 17
    rejected(w, bytes(bad), tmp_path, -1)
    rejected(w, raw, tmp_path, -2, n_up=w.n_up - 1)                                 # other sector


def test_unsorted_words_with_a_valid_hash(saved, tmp_path):
    w, B, _, raw = saved
    magic, version, ns, nu, nd, n, _ = HEADER.unpack_from(raw)
    U = B.copy()
    U[[3, 4]] = U[[4, 3]]
    words = U.astype("<u8").tobytes()
    p = tmp_path / "unsorted.mcdb"
    p.write_bytes(HEADER.pack(magic, version, ns, nu, nd, n, fnv1a64(words)) + words)
    ctx = host_ctx(w)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_load_basis(p)
    assert e.value.status == -1


def test_state_and_path_errors(tmp_path):
    w = C.ring8_u4()
    bare = pkg.Context(-1)
    with pytest.raises(pkg.MCDError) as e:
        bare.mcd_load_basis(tmp_path / "x.mcdb")
    assert e.value.status == -8                       # no Hamiltonian
    ctx = host_ctx(w)
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_save_basis(tmp_path / "x.mcdb")
    assert e.value.status == -8                       # no basis
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_load_basis(tmp_path / "missing.mcdb")
    assert e.value.status == -1
    ctx.mcd_set_basis(np.array([w.seed_word()], dtype=np.uint64))
    with pytest.raises(pkg.MCDError) as e:
        ctx.mcd_save_basis(tmp_path / "no_such_dir" / "x.mcdb")
    assert e.value.status == -1
