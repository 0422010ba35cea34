"""The benchmark's candidate-hop count (bonds with exactly one endpoint
occupied, both spins) against the oracle's hop enumeration state by state, and
its full-sector mean against the closed form bonds * 2 k (n - k) / (n (n - 1))
per spin (k electrons of that spin on n sites); and the DRAM-traffic lookup,
which reports a captured figure only while the kernel sources hash to the
value recorded with it."""
import os
import sys

import numpy as np

from oracle import fock
from workloads import configs as C

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def closed_form(bonds, n, ks):
    return sum(bonds * 2 * k * (n - k) / (n * (n - 1)) for k in ks)


def test_full_sector_mean_is_the_closed_form():
    for w in (C.ring8_u4(), C.tilted12_u8()):
        n = w.n_sites
        B = fock.sector(n, w.n_up, w.n_dn)
        if len(B) > 20000:
            B = B[np.random.default_rng(0).choice(len(B), 20000, replace=False)]
            tol = 0.05 * closed_form(np.count_nonzero(np.triu(w.lat.t, 1)), n, (w.n_up, w.n_dn))
        else:
            tol = 1e-12
        mean, used = bench.candidate_hops_per_state(B, w.lat.t, n, sample=len(B))
        assert used == len(B)
        ref = closed_form(np.count_nonzero(np.triu(w.lat.t, 1)), n, (w.n_up, w.n_dn))
        assert abs(mean - ref) <= tol, (w.name, mean, ref)
    # the figures quoted for the ring and the 4x4: 9.14 and 67.2 per state
    assert abs(closed_form(8, 8, (4, 4)) - 64 / 7) < 1e-12
    assert abs(closed_form(64, 16, (7, 7)) - 67.2) < 1e-12


def test_counts_equal_allowed_directed_hops():
    w = C.ring8_u4()
    n = w.n_sites
    B = fock.sector(n, w.n_up, w.n_dn)[::37]
    hops = fock.directed_hops(w.lat.t)
    allowed = sum(1 for x in B for spin in (0, 1) for i, j, _ in hops if fock.hop_word(int(x), n, spin, i, j))
    mean, used = bench.candidate_hops_per_state(B, w.lat.t, n, sample=len(B))
    assert used == len(B) and abs(mean * len(B) - allowed) < 1e-9


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    import hashlib
    import json
    import shutil
    src = os.path.join(bench.ROOT, "paper_2509_22975_gb300", "csrc")
    dst = tmp_path / "paper_2509_22975_gb300" / "csrc"
    dst.mkdir(parents=True)
    h = hashlib.sha256()
    for f in ("hv_cache.cu", "hv_cache.cuh", "hv_common.cuh"):
        shutil.copy(os.path.join(src, f), dst / f)
        h.update((dst / f).read_bytes())
    (tmp_path / "profiles").mkdir()
    key = "hv_cached_pass_B_square16_fp32_L1"
    rec = {"read": 400, "write": 72, "bytes_per_launch": 472, "kernel_src_sha": h.hexdigest()[:16]}
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({key: rec}))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for(key) == 472
    assert bench.traffic_for("no_such_kernel") is None
    with open(dst / "hv_cache.cuh", "a") as f:       # any change to the kernel sources
        f.write("\n")
    assert bench.traffic_for(key) is None


def test_peak_from_the_measured_file_else_the_fallback(tmp_path, monkeypatch):
    import json
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    peak, src = bench.measured_peak()
    assert peak == bench.FALLBACK_HBM and src.startswith("fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6789.3, "bf16_tflops": 1941.7}))
    peak, src = bench.measured_peak()
    assert peak == 6789.3 and src.startswith("measured")
