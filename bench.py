#!/usr/bin/env python
"""Benchmark of the Monte Carlo diagonalization hot path on one GB300.

Workload (the 4x4 configuration the throughput metric is quoted on): 4x4
periodic square cluster, t = 1, t' = -0.3, U = 8, N_up = N_dn = 7, Monte Carlo
basis of 1e7 states (beta = 0.2, seed 0, AFM seed state).  One step = one pass
of the whole hot path over that basis: device index build from the
device-resident basis words, then 200 Lanczos steps (H~ v with fp32 vectors and
fp64 coefficients, fused Krylov update, fp64 tridiagonal eigensolves).

value   = H~ v connections processed per second (nnz_offdiag(H~) x 200 per
          step, all ranks) with the basis already in HBM;
e2e     = the same through the C ABI from host words: mcd_set_basis (copy in,
          index) + mcd_lanczos_ground + E0 back to the host, every step;
roofline: the H~ v pair of kernels (the cached-record kernels: the first
          H~ v of each step's basis enumerates and looks up every hop once and
          stores the found ones, the later ones stream them), algorithmic
          bytes N_f (8 + 2 L s) per application over their mean CUDA-event
          duration in the timed steps; the record bytes they also read are
          reported beside it.

--impl reference times the oracle (the CPU fp64 implementation that the tests
check the kernels against) on a bounded sample of the same workload.
Multi-GPU: the path is run as independent replicas, one per rank.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H·v Gconnections/s; Lanczos iters/s vs plain FP64 path at |ΔE0|<1e-6"
UNIT = "Gconnections/s"
L2_BYTES = 129 * 2 ** 20
FALLBACK_HBM = 6800.0


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def slowest_rank_ms(ms: float, dist, dev) -> float:
    """Step time of the slowest rank, received by every rank (one rank: ms).
    Each rank runs its own replica of the step, so the job ends with it."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step: float, ms: float) -> float:
    """Units of all ranks per second, in 1e9 (every rank processes
    units_per_step per step; ms = the slowest rank's step time)."""
    return world * units_per_step / (ms * 1e-3) / 1e9


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, copy test)"
    return FALLBACK_HBM, "fallback (recipe figure, no measured file)"


# ---- clocks ---------------------------------------------------------------------
CLOCK_Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, bus_id: str | None):
        self.bus = (bus_id or "").lower()
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        time.sleep(0.25)

    def stop(self) -> dict:
        time.sleep(0.25)
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(", ") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if self.bus:
            mine = [r for r in rows if len(r) > 1 and self.bus.endswith(r[1].lower()[-12:])]
            rows = mine or rows
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[2]))
                mx.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---- oracle (CPU) ----------------------------------------------------------------
def oracle_sample(n_states: int, lattice: str = "square16"):
    """Oracle-built MC basis of a benchmark lattice (bounded size) + model."""
    import numpy as np
    from oracle import hamiltonian as H, sampler as S
    from workloads import configs
    w = configs.square16_u8() if lattice == "square16" else configs.rect24_u8()
    B = S.sample_basis(w.n_sites, w.lat.t, w.U_sites, w.n_up, w.n_dn, n_states, w.beta,
                       [w.seed_word()], seed=w.seed)
    M = H.Model(w.n_sites, w.lat.t, w.eps, w.U_sites)
    x = np.random.default_rng(0).standard_normal(len(B))
    return B, M, x


def oracle_apply(B, M, x):
    """One oracle y = H~ x: enumerate every hop of every state with a sorted
    search over the basis (oracle.hamiltonian.build), then multiply."""
    from oracle import hamiltonian as H
    P = H.build(M, B)
    y = P.sparse() @ x
    return P.nnz_offdiag(), y


def _oracle_worker(args):
    """One host process: the oracle's H~x repeated for `seconds` (spawned)."""
    n_states, lattice, seconds = args
    B, M, x = oracle_sample(n_states, lattice)
    t0 = time.perf_counter()
    conns = 0
    while time.perf_counter() - t0 < seconds:
        nnz, _ = oracle_apply(B, M, x)
        conns += nnz
    return conns, time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(seconds: float = 10.0, n_states: int = 1 << 17) -> dict:
    """The oracle's H~x on the host cores: one thread on the 4x4 sample (the
    reported value), the same on every core at once (one process per core,
    each applying H~ to its own vector of the same basis: throughput), and
    one thread on a 6x4 sample."""
    B, M, x = oracle_sample(n_states)
    t0 = time.perf_counter()
    conns, reps = 0, 0
    while True:
        nnz, _ = oracle_apply(B, M, x)
        conns += nnz
        reps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    out = {"value": conns / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{reps} oracle H~x applications (hop enumeration + sorted search + fp64 multiply) on an "
                     f"oracle-sampled {len(B)}-state MC basis of the same 4x4 t-t' lattice (nnz {nnz}); "
                     f"{dt:.1f} s; numpy single-threaded; host has {os.cpu_count()} cores"}
    import multiprocessing as mp
    cores = host_cores()
    variants = {}
    try:
        with mp.get_context("spawn").Pool(cores) as pool:   # spawned: the parent has a CUDA context
            res = pool.map(_oracle_worker, [(n_states, "square16", seconds)] * cores)
        tot = sum(c for c, _ in res)
        wall = max(t for _, t in res)
        variants["all_cores"] = {"value": tot / wall / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{cores} processes at once, each repeating the oracle's H~x on the "
                                           f"same {len(B)}-state 4x4 basis with its own vector for "
                                           f"{seconds:.0f} s; total connections / slowest process time"}
    except Exception as e:   # noqa: BLE001 (a baseline only: report, do not fail the bench)
        variants["all_cores"] = {"error": repr(e)}
    c6, t6 = _oracle_worker((n_states, "rect24", seconds))
    B6, _, _ = oracle_sample(n_states, "rect24")
    variants["rect24_one_core"] = {"value": c6 / t6 / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                                   "sample": f"oracle H~x repeated for {t6:.1f} s on an oracle-sampled "
                                             f"{len(B6)}-state MC basis of the 6x4 t-t' lattice (11+11 electrons)"}
    out["variants"] = variants
    # the oracle's Lanczos (App. B, its matrix-free H~x each step) for 5
    # iterations on the 4x4 sample; the caller extrapolates per iteration to
    # the workload's nonzeros
    from oracle import lanczos as OL
    t0 = time.perf_counter()
    OL.lanczos(lambda v: oracle_apply(B, M, v)[1], len(B), max_iter=5, tol=0.0, seed=0)
    out["lanczos_sample"] = {"iterations": 5, "s_per_iter": (time.perf_counter() - t0) / 5, "nnz": nnz,
                             "n_states": len(B)}
    out["host_cpu"] = host_cpu_name()
    return out


def host_cpu_name() -> str:
    """The host CPU as /proc/cpuinfo names it (model name, or the Arm part
    number), with the machine type and core count."""
    import platform
    name = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and not name:
                    name = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return f"{platform.machine()} {name} x{os.cpu_count()}".strip()


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    B, M, x = oracle_sample(1 << 15)
    for _ in range(args.warmup):
        oracle_apply(B, M, x)
    t0 = time.perf_counter()
    conns = 0
    for _ in range(args.steps):
        nnz, _ = oracle_apply(B, M, x)
        conns += nnz
    dt = time.perf_counter() - t0
    value = conns / dt / 1e9
    sample = (f"each step: one oracle H~x on an oracle-sampled {len(B)}-state MC basis of the 4x4 t-t' lattice "
              f"(nnz {nnz}), fp64, numpy single-threaded")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: oracle Monte Carlo basis (no dataset)",
        "config": workload_config(args, reference=True),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def workload_config(args, reference=False):
    if getattr(args, "workload", "square16") == "rect24":
        return {"workload": f"rect6x4_tp-0.3_U8_Nup11_Ndn11_mcbasis{args.n_f:.0e}_lanczos{args.iters}_fp32",
                "lattice": "6x4 periodic square, R1=(6,0) R2=(0,4), t=1, t'=-0.3", "U": 8.0, "n_up": 11,
                "n_dn": 11, "n_f": args.n_f, "mc_beta": 0.2, "mc_seed": 0, "lanczos_steps": args.iters, "ncols": 1,
                "vectors": "fp32 (fp64 coefficients and reductions)",
                "parallelism": f"replicas x{args.gpus}" if not reference else "cpu"}
    label = ("square4x4_tp-0.3_U8_Nup7_Ndn7_mcbasis1e7_lanczos200_fp32" if (args.n_f, args.iters) == (10_000_000, 200)
             else f"square4x4_tp-0.3_U8_Nup7_Ndn7_mcbasis{args.n_f}_lanczos{args.iters}_fp32")
    return {"workload": label,
            "lattice": "4x4 periodic square, R1=(4,0) R2=(0,4), t=1, t'=-0.3", "U": 8.0, "n_up": 7, "n_dn": 7,
            "n_f": args.n_f, "mc_beta": 0.2, "mc_seed": 0, "lanczos_steps": args.iters, "ncols": 1,
            "vectors": "fp32 (fp64 coefficients and reductions)",
            "l2": "working set (3 fp32 vectors + index) > 129 MB L2 each H*v; no flush",
            "parallelism": f"replicas x{args.gpus}" if not reference else "cpu"}


def traffic_for(kernel_key: str):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel source changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    ent = d.get(kernel_key)
    if not ent:
        return None
    h = hashlib.sha256()
    for f in ("hv_cache.cu", "hv_cache.cuh", "hv_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2509_22975_gb300", "csrc", f), "rb").read())
    return ent["bytes_per_launch"] if ent.get("kernel_src_sha") == h.hexdigest()[:16] else None


def impurity_batch(pkg, dev, n_inst=256, steps=400, tol=1e-6):
    """256 impurity models (2x2 plaquette + 8 bath sites, Monte Carlo bases
    log-uniform in [1e3, 1e5] states): fp32 Lanczos of every instance to a
    relative residual of 1e-6 (the fp32 form's floor; at most 400 steps),
    batched (the default form: per-instance cached solves on a pool of
    streams; and the lockstep form: persistent launches, CUDA-graph replay)
    against the same contexts solved one after another; timed after one
    untimed run, contexts and bases built beforehand."""
    import numpy as np
    import torch
    from workloads import impurity as IM
    ms = IM.batch(n_inst)
    ctxs = []
    for m in ms:
        c = pkg.Context(dev.index or 0)
        c.mcd_set_hamiltonian(m.t, m.eps, m.U_sites, m.n_up, m.n_dn)
        c.mcd_build_basis(m.seed, m.n_f, m.beta, [m.seed_word()])
        ctxs.append(c)
    n_states = sum(c.mcd_basis_info(nnz=False)["n_states"] for c in ctxs)
    nnz_of = [c.mcd_basis_info()["nnz_offdiag"] for c in ctxs]
    run = dict(allow_not_converged=True)
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_LOCKSTEP)
    pkg.mcd_batch_lanczos_ground(ctxs, steps, tol, 0, pkg.MCD_F32, **run)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = pkg.mcd_batch_lanczos_ground(ctxs, steps, tol, 0, pkg.MCD_F32, **run)
    torch.cuda.synchronize()
    t_batch = time.perf_counter() - t0
    for c in ctxs[:4]:
        c.mcd_lanczos_ground(steps, tol, 0, pkg.MCD_F32, **run)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seq = [c.mcd_lanczos_ground(steps, tol, 0, pkg.MCD_F32, **run) for c in ctxs]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    E_seq = np.asarray([q["E0"] for q in seq])
    # the default form: every instance's own cached solve on the pool of streams
    ctxs[0].mcd_set_option(pkg.MCD_OPT_BATCH_MODE, pkg.BATCH_POOL)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rp = pkg.mcd_batch_lanczos_ground(ctxs, steps, tol, 0, pkg.MCD_F32, **run)
    torch.cuda.synchronize()
    t_pool = time.perf_counter() - t0
    pool_equal = bool(np.array_equal(rp["E0"], E_seq) and
                      np.array_equal(rp["iters"], np.asarray([q["iters"] for q in seq])))
    conns = int(sum(z * int(i) for z, i in zip(nnz_of, r["iters"])))
    out = {"workload": "impurity_batch256_plaquette4_bath8_mcbasis1e3to1e5_lanczos_tol1e-6_fp32",
           "n_inst": n_inst, "n_states": n_states, "nnz_offdiag": int(sum(nnz_of)),
           "batched_s": t_pool, "sequential_s": t_seq, "speedup": t_seq / t_pool,
           "batched_form": "default (MCD_OPT_BATCH_MODE 0): every instance's cached solve on a pool of 16 host "
                           "threads with their own streams; results equal to the sequential calls bit for bit",
           "stream_pool_equals_sequential": pool_equal,
           "lockstep_s": t_batch, "lockstep_speedup": t_seq / t_batch,
           "batched_Gconn_per_s": conns / t_pool / 1e9, "sequential_Gconn_per_s": conns / t_seq / 1e9,
           "lockstep_Gconn_per_s": conns / t_batch / 1e9,
           "max_dE0_lockstep_vs_sequential": float(np.max(np.abs(E_seq - r["E0"]))),
           "lanczos_steps": {"batched_min": int(np.min(r["iters"])), "batched_max": int(np.max(r["iters"])),
                             "batched_total": int(np.sum(r["iters"])),
                             "sequential_total": int(sum(q["iters"] for q in seq))},
           "tol": tol,
           "timing": "wall clock around each call with device synchronisation; includes host tridiagonal solves"}
    # Green function of the cluster's spin-up orbitals, G(i omega_n) on 64
    # Matsubara points at beta_M = 50, and its gradient (bath energies and
    # hybridisations included): the instances run concurrently on a pool of
    # streams, against the one-instance calls one after another
    orb = [(0, 0), (1, 0), (2, 0), (3, 0)]
    z = 1j * (2 * np.arange(64) + 1) * np.pi / 50.0
    blocks = 40
    pkg.mcd_batch_band_lanczos_green(ctxs[:8], orb, blocks, 1.0, z, dtype=pkg.MCD_F32)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Gb, dpb, dmb = pkg.mcd_batch_band_lanczos_green(ctxs, orb, blocks, 1.0, z, dtype=pkg.MCD_F32)
    torch.cuda.synchronize()
    t_bg = time.perf_counter() - t0
    t0 = time.perf_counter()
    Gs = [c.mcd_band_lanczos_green(orb, blocks, 1.0, z, dtype=pkg.MCD_F32)[0] for c in ctxs]
    torch.cuda.synchronize()
    t_sg = time.perf_counter() - t0
    n_grad = 32
    rng = np.random.default_rng(0)
    gG = rng.normal(size=(n_grad, len(z), 4, 4)) + 1j * rng.normal(size=(n_grad, len(z), 4, 4))
    t0 = time.perf_counter()
    gb = pkg.mcd_batch_green_gradient(ctxs[:n_grad], orb, blocks, 1.0, z, gG, allow_not_converged=True)
    t_bgr = time.perf_counter() - t0
    t0 = time.perf_counter()
    gs_ = [c.mcd_green_gradient(orb, blocks, 1.0, z, gG[i], allow_not_converged=True)
           for i, c in enumerate(ctxs[:n_grad])]
    t_sgr = time.perf_counter() - t0
    out["green"] = {"orbitals": "cluster sites 0..3, spin up", "matsubara": "64 points, beta_M 50",
                    "band_blocks": blocks, "w_t": 1.0, "vectors": "fp32 (fp64 ground state from the fp32 solve)",
                    "excited_states_total": int(np.sum(dpb) + np.sum(dmb)),
                    "batched_s": t_bg, "sequential_s": t_sg, "speedup": t_sg / t_bg,
                    "bit_equal_to_single_calls": bool(all(np.array_equal(Gb[i], Gs[i]) for i in range(len(ctxs))))}
    out["green_gradient"] = {"instances": n_grad, "batched_s": t_bgr, "sequential_s": t_sgr,
                             "speedup": t_sgr / t_bgr,
                             "bit_equal_to_single_calls": bool(all(np.array_equal(gb[1][i], gs_[i][1])
                                                                   for i in range(n_grad)))}
    for c in ctxs:
        c.close()
    return out


def candidate_hops_per_state(words, lat_t, n_sites, sample=100_000, seed=0):
    """Mean number of candidate hops per state (bonds, both spins, with exactly
    one endpoint occupied: the enumeration before the lookup discards targets
    outside the basis), on a random sample of the basis words."""
    import numpy as np
    rng = np.random.default_rng(seed)
    w = words[rng.choice(len(words), min(sample, len(words)), replace=False)].astype(np.uint64)
    iu = np.argwhere(np.triu(lat_t, 1) != 0)
    masks = np.array([(1 << int(i)) | (1 << int(j)) for i, j in iu], dtype=np.uint64)
    half = np.uint64((1 << n_sites) - 1)
    total = 0
    for spin in (w >> np.uint64(n_sites), w & half):
        for m in masks:
            x = spin & m
            total += int(np.count_nonzero((x != 0) & (x != m)))
    return total / len(w), len(w)


def cache_build_ms(pkg, ctx, n, dev):
    """Time of the first H~v of a basis (record build + one application)
    minus that of the next one (CUDA events, one column fp32)."""
    import torch
    x = torch.randn(n, dtype=torch.float32, device=dev)
    y = torch.empty_like(x)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 0)
    torch.cuda.synchronize()
    ev[0].record()
    ctx.mcd_apply(x, y)
    ev[1].record()
    ctx.mcd_apply(x, y)
    ev[2].record()
    torch.cuda.synchronize()
    ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 1)
    return ev[0].elapsed_time(ev[1]) - ev[1].elapsed_time(ev[2])


def median_apply_ms(ctx, x, y, reps=20):
    """Median of reps back-to-back applications, each bracketed by its own
    CUDA event pair on the launching stream (after 3 untimed ones)."""
    import torch
    for _ in range(3):
        ctx.mcd_apply(x, y)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record()
    for i in range(reps):
        ctx.mcd_apply(x, y)
        ev[i + 1].record()
    torch.cuda.synchronize()
    return statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(reps))


def rect24_hv(pkg, configs, dev, peak, cols=(1, 24, 48)):
    """H~V on the 6x4 t-t' cluster (24 sites, 11 + 11 electrons, Monte Carlo
    basis of 5e7 states), fp32, each width timed alone with CUDA events after
    warm-up; X and Y are far larger than L2.  The first H~v builds the
    connection records (timed separately: build_ms)."""
    import torch
    w = configs.rect24_u8()
    ctx = pkg.Context(dev.index or 0)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    t0 = time.perf_counter()
    ctx.mcd_build_basis(w.seed, w.n_f, w.beta, [w.seed_word()])
    t_sample = time.perf_counter() - t0
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    build_ms = cache_build_ms(pkg, ctx, n, dev)
    info = ctx.mcd_basis_info()
    nnz = info["nnz_offdiag"]
    res = {"workload": "rect6x4_tp-0.3_U8_Nup11_Ndn11_mcbasis5e7", "n_states": n, "nnz_offdiag": nnz,
           "n_up_blocks": info["n_up_blocks"], "sampler_s": t_sample, "hv_cache": ctx.mcd_hv_cache_info(),
           "cache_build_ms": build_ms}
    ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 0)   # back-to-back launches; waits checked below
    for L_ in cols:
        x = torch.randn(n, L_, dtype=torch.float32, device=dev)
        y = torch.empty_like(x)
        t_ms = median_apply_ms(ctx, x, y)
        bytes_ = n * (8 + 2 * L_ * 4)
        res[f"L{L_}"] = {"ms": t_ms, "Gconn_per_s": nnz * L_ / (t_ms * 1e-3) / 1e9,
                         "algorithmic_GBps": bytes_ / (t_ms * 1e-3) / 1e9,
                         "frac_of_peak": bytes_ / (t_ms * 1e-3) / 1e9 / peak}
        del x, y
    res["wait_errors"] = ctx.mcd_hv_cache_info()["wait_errors"]
    del ctx
    torch.cuda.empty_cache()
    return res


def band_green(pkg, configs, dev, peak, name, n_f, n_blocks, w_t=0.999, f32=True, mu_half=True, n_mats=64,
               beta_m=50.0):
    """Band-Lanczos Green function end to end (App. C): Monte Carlo basis,
    Lanczos ground state, target-weight truncation, excited spaces F~+- of the
    spin-up orbitals of every site, the start blocks and n_blocks band steps in
    each space, G(i omega_n) on n_mats Matsubara points at beta_M.  Wall time of
    the Green-function call, and the H~V share from per-kernel CUDA events."""
    import numpy as np
    import torch
    w = getattr(configs, name)()
    if mu_half:
        w.mu = w.U / 2
    ctx = pkg.Context(dev.index or 0)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    ctx.mcd_build_basis(w.seed, n_f, w.beta, [w.seed_word()])
    n = ctx.mcd_basis_info(nnz=False)["n_states"]
    dt = pkg.MCD_F32 if f32 else pkg.MCD_F64
    psi = torch.empty(n, dtype=torch.float32 if f32 else torch.float64, device=dev)   # the kept ground state
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = ctx.mcd_lanczos_ground(800, 1e-7 if f32 else 1e-12, 0, dt, psi=psi, allow_not_converged=True)
    torch.cuda.synchronize()
    t_gs = time.perf_counter() - t0
    del psi
    orb = [(i, 0) for i in range(w.n_sites)]
    z = 1j * (2 * np.arange(n_mats) + 1) * np.pi / beta_m
    ctx.mcd_set_option(pkg.MCD_OPT_KERNEL_TIMING, 1)
    ctx.mcd_kernel_times(reset=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    G, dp, dm = ctx.mcd_band_lanczos_green(orb, n_blocks, w_t, z, dtype=dt)
    torch.cuda.synchronize()
    t_g = time.perf_counter() - t0
    kms, kcnt = ctx.mcd_kernel_times(reset=True)
    ctx.mcd_set_option(pkg.MCD_OPT_KERNEL_TIMING, 0)
    s = 4 if f32 else 8
    L_ = len(orb)
    hv_ms = kms[0] + kms[1]
    hv_bytes = n_blocks * (dp + dm) * (8 + 2 * L_ * s)   # every block taken as L columns wide
    tail = float(np.max(np.abs(z[-1] * G[-1] - np.eye(L_))))
    out = {"workload": f"{name} mu={'U/2' if mu_half else 0} MC basis {n} states, {L_} spin-up orbitals x 2 "
                       f"(c^dag, c), {n_blocks} band blocks per space, w_t {w_t}, G(i w_n) n<{n_mats} "
                       f"beta_M {beta_m}",
           "dtype": "f32 vectors, f64 Gram-Schmidt" if f32 else "f64", "n_states": n, "E0": r["E0"],
           "lanczos_iters": r["iters"], "ground_state_s": t_gs, "dim_plus": dp, "dim_minus": dm,
           "green_s": t_g, "blocks_per_s": 2 * n_blocks / t_g,
           "hv_ms": hv_ms, "hv_launches": int(kcnt[0] + kcnt[1]), "hv_share": hv_ms * 1e-3 / t_g,
           "hv_algorithmic_GBps": hv_bytes / (hv_ms * 1e-3) / 1e9 if hv_ms > 0 else None,
           "hv_frac_of_peak": hv_bytes / (hv_ms * 1e-3) / 1e9 / peak if hv_ms > 0 else None,
           "max_abs_zG_minus_1_at_largest_w_n": tail}
    ctx.close()
    torch.cuda.empty_cache()
    return out


def green_precision(pkg, configs, dev):
    """The 12-site Green-function workload on the 2e4-state prefix of its
    basis in fp32 and fp64 against stored oracle values (G(i omega_n) diagonal
    and E0, written by tests/golden/make_golden.py from the oracle)."""
    import numpy as np
    gold = json.load(open(os.path.join(ROOT, "tests", "golden", "green_tilted12_prefix.json")))
    w = configs.tilted12_u8()
    w.mu = w.U / 2
    ref = np.asarray(gold["G_diag_re"]) + 1j * np.asarray(gold["G_diag_im"])
    z = 1j * (2 * np.arange(gold["n_matsubara"]) + 1) * np.pi / gold["beta_M"]
    orb = [(i, 0) for i in range(12)]
    out = {"workload": f"tilted12 U=8 mu=U/2, MC basis prefix of {gold['n_f']} states, {gold['n_blocks']} blocks, "
                       f"w_t {gold['w_t']:.6f}, G(i w_n) n<{gold['n_matsubara']} beta_M {gold['beta_M']}"}
    for key, dt in (("f32", pkg.MCD_F32), ("f64", pkg.MCD_F64)):
        ctx = pkg.Context(dev.index or 0)
        ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
        ctx.mcd_build_basis(w.seed, gold["n_f"], w.beta, [w.seed_word()])
        import torch
        psi = torch.empty(gold["n_f"], dtype=torch.float32 if dt == pkg.MCD_F32 else torch.float64, device=dev)
        r = ctx.mcd_lanczos_ground(800, 1e-7 if dt == pkg.MCD_F32 else 1e-13, 0, dt, psi=psi,
                                   allow_not_converged=True)
        G, dp, dm = ctx.mcd_band_lanczos_green(orb, gold["n_blocks"], gold["w_t"], z, dtype=dt)
        d = np.einsum("zaa->za", G)
        out[key] = {"dE0_vs_oracle": abs(r["E0"] - gold["E0"]),
                    "max_rel_dG_vs_oracle": float(np.max(np.abs(d - ref)) / np.max(np.abs(ref))),
                    "dims_match": (dp, dm) == (gold["dim_plus"], gold["dim_minus"])}
        ctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="mcd", choices=["mcd", "reference"])
    ap.add_argument("--iters", type=int, default=200)
    ap.add_argument("--n-f", dest="n_f", type=int, default=10_000_000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--hv-cols", type=int, nargs="*", default=[1, 8, 24])
    ap.add_argument("--no-batch", action="store_true", help="skip the 256-impurity batch measurement")
    ap.add_argument("--no-hv-cache", action="store_true",
                    help="matrix-free H*v kernels (no connection records) on the 4x4 workload")
    ap.add_argument("--no-rect24", action="store_true",
                    help="skip the 6x4 t-t' (24-site, 5e7-state) H*V measurements")
    ap.add_argument("--no-green", action="store_true", help="skip the band-Lanczos Green-function measurements")
    ap.add_argument("--workload", default="square16", choices=["square16", "rect24"],
                    help="lattice of the Lanczos steps (rect24: the 6x4 cluster, for profiling its kernels)")
    ap.add_argument("--green-c5-blocks", type=int, default=40,
                    help="band blocks per excited space of the 6x4 Green function")
    ap.add_argument("--band-only", type=int, default=0, metavar="N_F",
                    help="profiling: only the 6x4 band-Lanczos Green function on an N_F-state basis "
                         "(--green-c5-blocks blocks); prints its record, not the benchmark line")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.band_only:
        import torch
        import paper_2509_22975_gb300 as pkg
        from workloads import configs
        pkg.build()
        dev = torch.device("cuda", 0)
        peak, _ = measured_peak()
        print(json.dumps({"band_green_rect24": band_green(pkg, configs, dev, peak, "rect24_u8", args.band_only,
                                                          args.green_c5_blocks, mu_half=False)}))
        return

    import numpy as np
    import torch
    import paper_2509_22975_gb300 as pkg
    from workloads import configs

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    w = configs.square16_u8() if args.workload == "square16" else configs.rect24_u8()
    ctx = pkg.Context(local)
    ctx.mcd_set_hamiltonian(w.lat.t, w.eps, w.U, w.n_up, w.n_dn)
    if args.no_hv_cache:
        ctx.mcd_set_option(pkg.MCD_OPT_HV_CACHE, pkg.CACHE_OFF)
    t0 = time.perf_counter()
    ctx.mcd_build_basis(w.seed, args.n_f, w.beta, [w.seed_word()])
    t_sample = time.perf_counter() - t0
    words = ctx.mcd_get_basis()
    n = len(words)
    words_dev = torch.from_numpy(words.view(np.int64)).to(dev)
    info = ctx.mcd_basis_info()
    nnz = info["nnz_offdiag"]

    def step():
        ctx.mcd_set_basis_device(words_dev)
        return ctx.mcd_lanczos_ground(args.iters, 0.0, 0, pkg.MCD_F32)

    for _ in range(args.warmup):
        r32 = step()
    torch.cuda.synchronize()
    bus = None
    try:
        bus = torch.cuda.get_device_properties(local).pci_bus_id
    except Exception:
        pass
    clk = ClockSampler(bus)
    l0 = ctx.mcd_launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        r32 = step()
    e1.record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    launches = ctx.mcd_launch_count() - l0
    ms = e0.elapsed_time(e1) / args.steps
    # per-kernel split from separate steps with a CUDA event pair around
    # every H~v kernel (the timed steps above run without them)
    split_steps = 2
    ctx.mcd_set_option(pkg.MCD_OPT_KERNEL_TIMING, 1)
    ctx.mcd_kernel_times(reset=True)
    s0e, s1e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0e.record()
    for _ in range(split_steps):
        step()
    s1e.record()
    torch.cuda.synchronize()
    ms_instr = s0e.elapsed_time(s1e) / split_steps
    kms, kcnt = ctx.mcd_kernel_times(reset=True)
    ctx.mcd_set_option(pkg.MCD_OPT_KERNEL_TIMING, 0)
    ms = slowest_rank_ms(ms, dist, dev)
    conns_per_step = nnz * r32["iters"]
    value = whole_job_rate(world, conns_per_step, ms)

    # roofline of the H~v pair (pass B: dn-major up-hop kernel, pass A: up-major dn-hop + diagonal)
    tB = kms[0] / max(kcnt[0], 1)
    tA = kms[1] / max(kcnt[1], 1)
    tU = kms[2] / max(kcnt[2], 1)
    alg_bytes = n * (8 + 2 * 1 * 4)
    peak, peak_src = measured_peak()
    achieved = alg_bytes / ((tA + tB) * 1e-3) / 1e9
    tb, ta = (None, None) if args.no_hv_cache or args.workload != "square16" else (
        traffic_for("hv_cached_pass_B_square16_fp32_L1"), traffic_for("hv_cached_pass_A_square16_fp32_L1"))
    cinfo = ctx.mcd_hv_cache_info()
    rec_bytes = cinfo["bytes"]
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tb + ta) if (tb is not None and ta is not None) else None,
                "kernel": ("H~v pair (matrix-free hv_l1_kernel pass B + pass A), one application" if args.no_hv_cache else
                           "H~v pair (hv_stream_kernel pass B with its x permutation + pass A), records of the found "
                           "hops, one application"),
                "algorithmic_bytes": alg_bytes, "peak_source": peak_src,
                "record_bytes": rec_bytes,
                "achieved_incl_records": (alg_bytes + rec_bytes) / ((tA + tB) * 1e-3) / 1e9,
                "frac_incl_records": (alg_bytes + rec_bytes) / ((tA + tB) * 1e-3) / 1e9 / peak,
                "mean_ms": {"pass_B": tB, "pass_A": tA, "krylov_update": tU},
                "share_of_step": {"pass_B": kms[0] / split_steps / ms_instr,
                                  "pass_A": kms[1] / split_steps / ms_instr,
                                  "krylov_update": kms[2] / split_steps / ms_instr},
                "timing": f"kernel means from {split_steps} separate steps with per-kernel CUDA events "
                          f"({ms_instr:.2f} ms per step there); the headline steps run without them"}

    # end to end through the C ABI from host words (pinned host memory)
    words_host = torch.from_numpy(words.view(np.int64)).pin_memory()
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ctx.mcd_set_basis(words_host)
        re2e = ctx.mcd_lanczos_ground(args.iters, 0.0, 0, pkg.MCD_F32)
        _E0 = re2e["E0"]
    e2e_s = (time.perf_counter() - h0) / max(args.e2e_steps, 1)
    chunks = list(range(16, args.iters + 1, 16)) + ([args.iters] if args.iters % 16 else [])
    d2h = sum(8 * (2 * m + 1) for m in chunks) + 8 + 4 + 16   # a/b read-backs, E0, checks, block counts
    h2d = n * 8
    e2e = {"value": world * conns_per_step / e2e_s / 1e9 if args.e2e_steps else None, "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3,
           "path": "mcd_set_basis(pinned host words) + mcd_lanczos_ground + E0 to host",
           "note": "same path as the device-timed steps, plus the host words' copy and the E0 read-back"}

    # the record build alone: a fresh basis, first H~v minus the next one
    ctx.mcd_set_basis_device(words_dev)
    build_ms = None if args.no_hv_cache else cache_build_ms(pkg, ctx, n, dev)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic: Monte Carlo basis sampled by the library",
           "config": workload_config(args), "roofline": roofline, "e2e": e2e,
           "gpu_launches": launches, "clocks": clocks,
           "basis": {"n_states": n, "nnz_offdiag": nnz, "n_up_blocks": info["n_up_blocks"],
                     "n_dn_blocks": info["n_dn_blocks"], "sampler_s": t_sample},
           "hv_cache": dict(cinfo, build_ms=build_ms),
           "E0_fp32": r32["E0"], "lanczos_iters_per_s_fp32": r32["iters"] / (ms * 1e-3)}
    cand, cand_sample = candidate_hops_per_state(words, w.lat.t, w.n_sites)
    out["candidate_hops"] = {"per_state": cand, "sample_states": cand_sample,
                             "found_per_state": nnz / n,
                             "per_s": world * cand * n * r32["iters"] / (ms * 1e-3),
                             "note": "candidate hops (before the lookup) per second of the timed steps"}

    if args.hv_cols:
        # H~V with L columns (the band-Lanczos product), fp32, timed alone with
        # CUDA events; x, y of 1e7 x L fp32 are far larger than L2
        hv = {}
        ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 0)   # back-to-back launches; waits checked below
        for L_ in args.hv_cols:
            x = torch.randn(n, L_, dtype=torch.float32, device=dev)
            y = torch.empty_like(x)
            t_ms = median_apply_ms(ctx, x, y)
            bytes_ = n * (8 + 2 * L_ * 4)
            hv[f"L{L_}"] = {"ms": t_ms, "Gconn_per_s": nnz * L_ / (t_ms * 1e-3) / 1e9,
                            "algorithmic_GBps": bytes_ / (t_ms * 1e-3) / 1e9,
                            "frac_of_peak": bytes_ / (t_ms * 1e-3) / 1e9 / peak}
            del x, y
        hv["wait_errors"] = ctx.mcd_hv_cache_info()["wait_errors"]
        ctx.mcd_set_option(pkg.MCD_OPT_APPLY_SYNC, 1)
        out["hv_apply_fp32"] = hv

    if not args.no_rect24:
        out["hv_apply_rect24_fp32"] = rect24_hv(pkg, configs, dev, peak)
    if not args.no_green:
        out["green_precision_tilted12_prefix"] = green_precision(pkg, configs, dev)
        out["band_green_C2"] = band_green(pkg, configs, dev, peak, "tilted12_u8", 1 << 18, 150)
        out["band_green_C5"] = band_green(pkg, configs, dev, peak, "rect24_u8", 50_000_000, args.green_c5_blocks,
                                          mu_half=False)
    if not args.no_batch:
        out["impurity_batch"] = impurity_batch(pkg, dev)

    if not args.no_fp64:
        # fp64 form and the plain fp64 path (global binary search kernel), same 200 steps
        for algo, key in ((0, "fp64_blocked"), (1, "fp64_plain")):
            ctx.mcd_set_option(pkg.MCD_OPT_HV_ALGO, algo)
            torch.cuda.synchronize()
            a0 = time.perf_counter()
            r64 = ctx.mcd_lanczos_ground(args.iters, 0.0, 0, pkg.MCD_F64)
            torch.cuda.synchronize()
            dt = time.perf_counter() - a0
            out[f"lanczos_iters_per_s_{key}"] = r64["iters"] / dt
            out[f"E0_{key}"] = r64["E0"]
        ctx.mcd_set_option(pkg.MCD_OPT_HV_ALGO, 0)
        out["dE0_fp32_vs_plain_fp64"] = abs(out["E0_fp32"] - out["E0_fp64_plain"])
        out["dE0_fp32_vs_cached_fp64"] = abs(out["E0_fp32"] - out["E0_fp64_blocked"])
        # the precision comparison on the same cached kernels first, then against the plain path
        out["fp32_speedup_vs_cached_fp64"] = out["lanczos_iters_per_s_fp32"] / out["lanczos_iters_per_s_fp64_blocked"]
        out["fp32_speedup_vs_plain_fp64"] = out["lanczos_iters_per_s_fp32"] / out["lanczos_iters_per_s_fp64_plain"]

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline()
        ls = cb["lanczos_sample"]
        # one oracle Lanczos iteration on this workload, extrapolated by its nonzeros
        cb["lanczos_s_per_iter_extrapolated"] = ls["s_per_iter"] * nnz / ls["nnz"]
        cb["lanczos_iters_per_s_extrapolated"] = 1.0 / cb["lanczos_s_per_iter_extrapolated"]
        out["cpu_baseline"] = cb
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
