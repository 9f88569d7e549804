"""Benchmark of the two-scale domain-decomposition Eikonal solver on one GB300.

Workload (default): 2-D 4097^2 grid (h = 1/4096), slowness r = clip(1 + 0.3x +
0.4 F/max|F|, 0.2) with F a sum of 32 seeded Fourier modes, |k| in [64, 128]
(eps = 1/64); Gamma = the whole left edge x = 0, g = 0; 16 x 16 subdomains,
coarse ratio 16 (coarse grid 257^2); FP32 storage; weight theta = 0 (the
fastest weight measured on this workload: Step 4 then hands u^k to the causal
sweep); stop when the coarse update falls below 1e-6 or after 2*16 + 10 = 42
iterations.  --theta X runs another constant weight, --theta adaptive the
per-node weight of Sec. 4.2 (omega = (1, 1, 1), sigmoid damping gamma 0.75,
delta 0.01, x0 0.9, capped at 0.1, constant 0.1 where undefined).  The line
also carries the time to solution of the adaptive weight and of the constant
weights 0.05 and 0.2 under the same stop rule.

One step = one complete eik_dd_solve (set-up, Step 1, all parareal iterations)
on device-resident inputs.  value = local Godunov solves executed per second
(fine + coarse) in G updates/s; the line also carries the time to solution,
the fine-grid cell rate, the error against an FP64 full-grid reference and the
plain full-grid FSM solving the same grid.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 CPU oracle (the test suite's reference
implementation) on a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1805_04198_gb300 import inputs  # noqa: E402

METRIC = "time-to-solution & Gcell-updates/s vs plain GPU full-grid FSM at equal error"
N_SIDE = 4097
TILES = 16
COARSE = 16
THETA = 0.1          # fallback of the adaptive weight where its estimate is undefined
THETA_CAP = 0.1      # cap on the adaptive weight (cap 1 diverges on this workload)
THETA_SWEEP = ("adaptive", 0.05, 0.2)
MAX_ITER = 2 * TILES + 10
TOL = 1e-6
MAX_COARSE_SWEEPS = 8
BYTES_PER_UPDATE_F32 = 12  # one sweep pass streams u in, r in, u out per node update


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# DRAM traffic of the subdomain kernel comes from one ncu capture summarised in
# profiles/ (bytes read + written per fine update of the captured launch).  It
# is used only while the kernel sources still hash to the value recorded there.
TRAFFIC_SUMMARY = os.path.join(ROOT, "profiles", "dd_fine_subdomains_4097_ncu.md")
KERNEL_SOURCES = ["common.cuh", "engine.cuh", "dd_geom.cuh", "dd2_device.cuh", "eik_dd.cu"]


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1805_04198_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def fine_traffic_per_launch(fine_updates_per_launch):
    try:
        with open(TRAFFIC_SUMMARY) as f:
            kv = dict(ln.split(":", 1) for ln in f.read().splitlines() if ln.startswith(("source_hash:", "dram_bytes_per_fine_update:")))
        if kv.get("source_hash", "").strip() != kernel_source_hash():
            return None
        return float(kv["dram_bytes_per_fine_update"]) * fine_updates_per_launch
    except (OSError, KeyError, ValueError):
        return None


def make_workload(dtype=np.float32):
    w = inputs.workload_c1(n=N_SIDE, tiles=TILES, c=COARSE)
    return w["r"].astype(dtype), w["gamma"], w["g"].astype(dtype), w["h"]


def cpu_oracle_sample(r32, gamma, g, h, parallel=False):
    """Oracle (FP64) on a bounded sample of the workload: Step 1 and one fine
    pass over all 256 subdomains (max_iter = 0).  parallel=True runs the
    OpenMP build of the same source on every host core."""
    import oracle
    t0 = time.perf_counter()
    _, st, _ = oracle.dd(r32.astype(np.float64), gamma, g.astype(np.float64), h, (TILES, TILES), COARSE,
                         theta=THETA, max_iter=0, tol=TOL, max_coarse_sweeps=MAX_COARSE_SWEEPS, parallel=parallel)
    dt = time.perf_counter() - t0
    upd = st["fine_updates"] + st["coarse_updates"]
    return upd / dt / 1e9, dt, upd


def host_cpu():
    """Core count and CPU model of the host (lscpu, else /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() == "Model name":
                model = ln.split(":", 1)[1].strip()
                break
    except Exception:  # noqa: BLE001
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    threads = int(os.environ.get("OMP_NUM_THREADS", "0") or 0) or os.cpu_count()
    return {"nproc": os.cpu_count(), "threads": threads, "model": model}


def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r32, gamma, g, h = make_workload()
    host = host_cpu()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, upd = cpu_oracle_sample(r32, gamma, g, h, parallel=True)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    sample = ("4097^2 workload, Step 1 + one fine pass over all 256 subdomains (max_iter=0), "
              "FP64 oracle built with OpenMP over the subdomain and shifted-grid solves, %d threads on %s; "
              "value = local solves executed / wall time" % (host["threads"], host["model"]))
    line = {"metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "c1_2d_4097_leftedge_16x16_c16", "sample": "max_iter=0"},
            "cpu_baseline": {"value": value, "unit": "Gupdates/s", "cores": host["threads"], "kind": "oracle",
                             "sample": sample, "host": host},
            "e2e": {"value": value, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def max_over_ranks(x, dist, device):
    """The slowest rank's value (the job's time); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, total_ms):
    """Whole-job G units/s: every rank processed units_per_rank in total_ms
    (the max over ranks)."""
    return units_per_rank * world / (total_ms / 1e3) / 1e9


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--theta", default="0",
                    help="a constant weight (default 0) or 'adaptive' (the per-node weight of Sec. 4.2)")
    ap.add_argument("--workload", default="dd4097",
                    choices=["dd4097", "batch256", "dd3d257", "tomography1025", "obstacles", "dd1bump"],
                    help="dd4097 (default) is the benchmark line; the others measure the batched solve, the "
                         "3-D solve, the tomography gradient, the Sec. 4 obstacle fields and the 1-D method "
                         "with the same keys")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload != "dd4097":
        return run_extra(args)

    import torch
    from paper_1805_04198_gb300 import eik

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    eik.load()

    r32, gamma, g32, h = make_workload()
    R = torch.from_numpy(r32).to(dev)
    G = torch.from_numpy(gamma).to(dev)
    g = torch.from_numpy(g32).to(dev)
    tiles = (TILES, TILES)
    dd_kw = dict(theta=THETA, max_iter=MAX_ITER, tol=TOL, max_coarse_sweeps=MAX_COARSE_SWEEPS)
    if args.theta == "adaptive":
        dd_kw.update(theta_adaptive=True, theta_cap=THETA_CAP)
        theta_cfg = {"rule": "adaptive, Sec. 4.2", "omega": [1.0, 1.0, 1.0], "sig_gamma": 0.75,
                     "sig_delta": 0.01, "sig_x0": 0.9, "cap": THETA_CAP, "fallback": THETA}
    else:
        dd_kw["theta"] = float(args.theta)
        theta_cfg = dd_kw["theta"]

    # buffers allocated once, outside the timed region
    grid = eik.make_grid(R, h)
    params = eik.dd_params(tiles, COARSE, **dd_kw)
    ws = torch.empty(eik.eik_dd_workspace_size(grid, params) + 256, dtype=torch.uint8, device=dev)
    u = torch.empty_like(R)
    st_dev = torch.zeros(eik.ctypes.sizeof(eik.DDStats), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2
    stream = torch.cuda.current_stream()

    def solve():
        eik.eik_dd_solve(grid, R, G, g, params, u, ws, st_dev, stream)

    for _ in range(args.warmup):
        solve()
    torch.cuda.synchronize()
    stats0 = eik.parse_dd_stats(st_dev)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    upd_total = 0
    launches = 0
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    eik.eik_profile_enable(True)
    with ClockSampler(local_rank) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))  # evict L2 between timed steps (not timed)
            starts[i].record(stream)
            solve()
            stops[i].record(stream)
        torch.cuda.synchronize()
    eik.eik_profile_enable(False)
    prof = eik.eik_profile_collect()
    if dist is not None:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, stops)]
    total_ms = sum(step_ms)
    stats = eik.parse_dd_stats(st_dev)
    upd_step = stats["fine_updates"] + stats["coarse_updates"]
    upd_total = upd_step * args.steps
    launches = stats["launches"] * args.steps
    total_ms = max_over_ranks(total_ms, dist, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(upd_total, world, total_ms)
    cells = float(N_SIDE) * N_SIDE

    # roofline of the dominant kernel (event-timed inside the timed region)
    peak, peak_kind = load_peaks()
    fine = prof.get("dd_fine_subdomains", {"total_ms": float("nan"), "launches": 0})
    fine_upd = stats["fine_updates"] * args.steps
    achieved = fine_upd * BYTES_PER_UPDATE_F32 / (fine["total_ms"] / 1e3) / 1e9
    # per working launch: the launches after convergence return at once
    fine_upd_launch = stats["fine_updates"] / max(1, stats["iters"] + 1)
    traffic = fine_traffic_per_launch(fine_upd_launch)

    # accuracy against an FP64 full-grid reference, and the plain full-grid FSM
    # at equal error (not part of the timed DD steps)
    acc = {}
    fsm_line = None
    try:
        uf, fst = eik.fsm(R.double(), G, g.double(), h, max_sweeps=100000)
        umax = uf.abs().max().item()

        def rel_err(x):
            return (x.double() - uf).abs().max().item() / umax

        dd_err = rel_err(u)
        acc = {"rel_max_err_vs_fp64_fsm": dd_err, "fp64_fsm_sweeps": fst["sweeps"]}

        def fsm_timed(ms):
            reps = []
            for _ in range(3):
                flush.fill_(0.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                uu, ss = eik.fsm(R, G, g, h, max_sweeps=ms, sync=False)
                e1.record(stream)
                torch.cuda.synchronize()
                reps.append(e0.elapsed_time(e1))
            sweeps = eik.FsmStats.from_buffer_copy(bytes(ss.cpu().numpy())).sweeps
            return uu, min(reps), sweeps

        # smallest FP32 FSM sweep count whose error is at most the DD error; when
        # the DD is more accurate than the converged FP32 FSM, the FSM's own
        # converged error is the target (its time to convergence)
        uu_full, t_full, full_sweeps = fsm_timed(100000)
        fsm_floor = rel_err(uu_full)
        equal_cache = {}

        def fsm_at_equal_error(err):
            target = max(err, fsm_floor)
            if target not in equal_cache:
                lo, hi = 1, full_sweeps
                while lo < hi:
                    mid = (lo + hi) // 2
                    uu, _ = eik.fsm(R, G, g, h, max_sweeps=mid)
                    if rel_err(uu) <= target:
                        hi = mid
                    else:
                        lo = mid + 1
                uu_eq, t_eq, _ = fsm_timed(lo)
                equal_cache[target] = (target, lo, t_eq, rel_err(uu_eq))
            return equal_cache[target]

        target, lo, t_eq, err_eq = fsm_at_equal_error(dd_err)
        sweep_bytes = cells * BYTES_PER_UPDATE_F32
        fsm_line = {"target_err": target, "sweeps_to_equal_error": lo, "time_to_equal_error_ms": t_eq,
                    "rel_max_err_at_equal": err_eq, "converged_sweeps": full_sweeps,
                    "time_to_convergence_ms": t_full, "rel_max_err_converged": fsm_floor,
                    "dd_over_fsm_time_at_equal_error": ms_per_step / t_eq,
                    "fsm_over_dd_time_at_equal_error": t_eq / ms_per_step,
                    # the baseline's own sweep passes against HBM: 12 B per node per sweep
                    "roofline": {"bound": "hbm", "ms_per_sweep": t_eq / lo,
                                 "achieved": sweep_bytes * lo / (t_eq / 1e3) / 1e9, "peak": peak,
                                 "unit": "GB/s", "frac": sweep_bytes * lo / (t_eq / 1e3) / 1e9 / peak,
                                 "algorithmic_bytes": "12 B per node per sweep (u in, r in, u out)"}}
        # constant weights under the same stop rule (not part of the timed steps)
        sweep = []
        for th in THETA_SWEEP:
            if th == "adaptive":
                kw = dict(dd_kw, theta=THETA, theta_adaptive=True, theta_cap=THETA_CAP)
            else:
                kw = dict(dd_kw, theta=th, theta_adaptive=False)
            reps = []
            for rep in range(3):
                flush.fill_(0.0)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                uu, ss = eik.dd_solve(R, G, g, h, tiles, COARSE, sync=False, **kw)
                e1.record(stream)
                torch.cuda.synchronize()
                reps.append(e0.elapsed_time(e1))
            s2 = eik.parse_dd_stats(ss)
            err2 = rel_err(uu)
            _, lo2, t_eq2, _ = fsm_at_equal_error(err2)
            sweep.append({"theta": th, "iters": s2["iters"], "converged": s2["converged"], "ms": min(reps),
                          "rel_max_err_vs_fp64_fsm": err2, "fsm_sweeps_to_equal_error": lo2,
                          "fsm_time_to_equal_error_ms": t_eq2, "fsm_over_dd_time_at_equal_error": t_eq2 / min(reps)})
        fsm_line["dd_other_theta"] = sweep
    except Exception as e:  # noqa: BLE001
        acc = acc or {"rel_max_err_vs_fp64_fsm": None}
        fsm_line = {"unavailable": str(e)[:160]}

    # end to end through the public API with host buffers (pinned)
    e2e = None
    try:
        hr = torch.from_numpy(r32).pin_memory()
        hG = torch.from_numpy(gamma).pin_memory()
        hg = torch.from_numpy(g32).pin_memory()
        hu = torch.empty_like(hr).pin_memory()
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(args.steps):
            dr = hr.to(dev, non_blocking=True)
            dG = hG.to(dev, non_blocking=True)
            dg = hg.to(dev, non_blocking=True)
            du, _ = eik.dd_solve(dr, dG, dg, h, tiles, COARSE, sync=False, **dd_kw)
            hu.copy_(du, non_blocking=True)
        t1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = t0.elapsed_time(t1) / args.steps
        e2e = {"value": upd_step / (e2e_ms / 1e3) / 1e9, "unit": "Gupdates/s",
               "h2d_bytes_per_step": hr.numel() * 4 + hG.numel() + hg.numel() * 4,
               "d2h_bytes_per_step": hu.numel() * 4, "ms_per_step": e2e_ms}
    except Exception as e:  # noqa: BLE001
        e2e = {"value": None, "unit": "Gupdates/s", "note": str(e)[:160]}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        host = host_cpu()
        try:
            v, dt, upd = cpu_oracle_sample(r32, gamma, g32, h, parallel=True)
            v1, dt1, _ = cpu_oracle_sample(r32, gamma, g32, h, parallel=False)
            cpu = {"value": v, "unit": "Gupdates/s", "cores": host["threads"], "kind": "oracle",
                   "sample": "Step 1 + one fine pass over all 256 subdomains of the same 4097^2 workload "
                             "(max_iter=0), %d local solves: %.2f s with the OpenMP build on %d threads, "
                             "%.1f s serial" % (upd, dt, host["threads"], dt1),
                   "host": host, "serial_1core": {"value": v1, "seconds": dt1}}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": "Gupdates/s", "cores": host["threads"], "kind": "oracle",
                   "sample": str(e)[:160], "host": host}

    # time to solution at equal error for the benchmark's weight and for the
    # paper's per-node weight (Sec. 4.2), each against the plain FSM reaching
    # the same error
    equal = {}
    if fsm_line and "time_to_equal_error_ms" in fsm_line:
        equal["benchmark_weight"] = {
            "theta": theta_cfg, "dd_ms": ms_per_step, "rel_max_err": acc.get("rel_max_err_vs_fp64_fsm"),
            "fsm_ms": fsm_line["time_to_equal_error_ms"], "fsm_sweeps": fsm_line["sweeps_to_equal_error"],
            "fsm_over_dd": fsm_line["time_to_equal_error_ms"] / ms_per_step}
        for e in fsm_line.get("dd_other_theta", []):
            if e["theta"] == "adaptive":
                equal["adaptive_sec4_2"] = {
                    "theta": {"rule": "adaptive, Sec. 4.2", "cap": THETA_CAP, "fallback": THETA},
                    "dd_ms": e["ms"], "iters": e["iters"], "converged": e["converged"],
                    "rel_max_err": e["rel_max_err_vs_fp64_fsm"], "fsm_ms": e["fsm_time_to_equal_error_ms"],
                    "fsm_sweeps": e["fsm_sweeps_to_equal_error"], "fsm_over_dd": e["fsm_over_dd_time_at_equal_error"]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c1_2d_4097_leftedge_16x16_c16", "n": N_SIDE, "tiles": TILES,
                       "coarse_ratio": COARSE, "theta": theta_cfg, "max_iter": MAX_ITER, "tol": TOL,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"},
            "time_to_solution_ms": ms_per_step,
            "gcells_per_s": cells * world / (ms_per_step / 1e3) / 1e9,
            "dd_stats": {k: stats[k] for k in ("iters", "converged", "fsm_sweeps_max", "coarse_sweeps_max",
                                              "fine_updates", "coarse_updates", "last_delta",
                                              "fine_solves_skipped")},
            "accuracy": acc,
            "equal_error": equal,
            "fsm_baseline_f32": fsm_line,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "kernel": "dd_fine_subdomains",
                         "peak_source": peak_kind,
                         "algorithmic_bytes": "12 B per fine node update (u in, r in, u out) x fine updates"},
            "kernel_ms": {k: v["total_ms"] / args.steps for k, v in prof.items()},
            "gpu_launches": launches,
            "e2e": e2e,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


# --------------------------------------------------------------------------
# Further workloads (not the benchmark line): same keys, own metric.
# --------------------------------------------------------------------------
def _timed(torch, fn, steps, warmup, flush, stream):
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        stops[i].record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in zip(starts, stops)) / steps


def _profiled(torch, eik, fn):
    eik.eik_profile_enable(True)
    fn()
    torch.cuda.synchronize()
    eik.eik_profile_enable(False)
    return eik.eik_profile_collect()


def run_extra(args):
    import torch
    from paper_1805_04198_gb300 import eik
    import oracle
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    eik.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peak, peak_kind = load_peaks()
    cpu = None
    extra = {}
    t = lambda a, dt=None: torch.from_numpy(np.ascontiguousarray(a)).to(dev) if dt is None else \
        torch.from_numpy(np.ascontiguousarray(a)).to(dev, dt)

    if args.workload == "batch256":
        w = inputs.workload_c3()
        probs = [dict(r=t(q["r"].astype(np.float32)), gamma=t(q["gamma"]), g=t(q["g"].astype(np.float32)),
                      h=q["h"], tiles=q["tiles"], coarse_ratio=q["c"], theta=q["theta"], max_iter=q["max_iter"],
                      tol=q["tol"]) for q in w]
        B = eik.DDBatch(probs)
        best, tune_ms = B.autotune(tune_iters=2)
        prof = _profiled(torch, eik, B.run)
        B.capture()
        with ClockSampler(local_rank) as clk:
            ms = _timed(torch, B.replay, args.steps, args.warmup, flush, stream)
        st = B.stats()
        upd = sum(x["fine_updates"] + x["coarse_updates"] for x in st)
        fine_upd = sum(x["fine_updates"] for x in st)
        fine_ms = prof["dd_fine_subdomains"]["total_ms"]
        kern = ("dd_fine_subdomains", fine_upd * BYTES_PER_UPDATE_F32 / (fine_ms / 1e3) / 1e9)
        extra = {"autotuned": {"fine_queue": best.fine_queue, "coarse_queue": best.coarse_queue,
                               "ctas_per_sm": best.ctas_per_sm, "largest_first": best.largest_first,
                               "tune_ms": tune_ms},
                 "launches_per_solve": st[0]["launches"], "graph": True,
                 "iters": sorted(set(x["iters"] for x in st)),
                 "converged": sum(int(x["converged"]) for x in st)}
        # end to end: pinned host inputs in, every u out, each step
        hr = [torch.from_numpy(q["r"].astype(np.float32)).pin_memory() for q in w]
        hu = [torch.empty_like(x).pin_memory() for x in hr]
        def e2e_step():
            for p, x in zip(probs, hr):
                p["r"].copy_(x, non_blocking=True)
            B.replay()
            for y, u in zip(hu, B.u):
                y.copy_(u, non_blocking=True)
        e2e_ms = _timed(torch, e2e_step, max(1, args.steps // 2), 1, flush, stream)
        h2d = sum(x.numel() * 4 for x in hr)
        e2e = {"value": upd / (e2e_ms / 1e3) / 1e9, "unit": "Gupdates/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": h2d, "ms_per_step": e2e_ms,
               "note": "slowness of every problem in, every u out (sources stay resident)"}
        workload = {"workload": "batch_256_mixed_2d", "nprob": len(w), "sides": [257, 513, 1025, 2049],
                    "tiles": [8, 16, 32], "theta": w[0]["theta"], "tol": w[0]["tol"], "cap": "2T+10",
                    "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}
        unit, metric = "Gupdates/s", "batched DD: local solves per second over a 256-problem mixed batch"
        if rank == 0 and not args.no_cpu_baseline:
            small = [i for i, q in enumerate(w) if q["r"].shape[0] == 257][:2]
            t0 = time.perf_counter()
            cu = 0
            for i in small:
                q = w[i]
                _, so, _ = oracle.dd(q["r"].astype(np.float32).astype(np.float64), q["gamma"], q["g"], q["h"],
                                     q["tiles"], q["c"], theta=q["theta"], max_iter=q["max_iter"], tol=q["tol"],
                                     max_coarse_sweeps=8)
                cu += so["fine_updates"] + so["coarse_updates"]
            dt = time.perf_counter() - t0
            cpu = {"value": cu / dt / 1e9, "unit": unit, "cores": 1, "kind": "oracle",
                   "sample": "the first two 257^2 problems of the batch, full solves, %.1f s" % dt}
        value = upd * world / (ms / 1e3) / 1e9
    elif args.workload == "dd1bump":
        # the 1-D method (Sec. 3.1) on its example slowness (Gaussian bump at
        # x = 0.75, u(0) = u(1) = 0), 1024 subintervals of 1000 cells, FP64
        N, M = 1024, 1000
        n, h = N * M + 1, 1.0 / (N * M)
        x = np.arange(n) * h
        r64 = 1.0 + 10.0 * np.exp(-(x - 0.75) ** 2 / (2 * 0.01 ** 2))
        gam = np.zeros(n, np.uint8)
        gam[0] = gam[-1] = 1
        # theta = 1: the coarse grid (H = 1/1024) resolves the bump, and the
        # full parareal correction converges in 2 iterations; theta = 0.5
        # (119 iterations) is timed as an extra field
        kw = dict(theta=1.0, max_iter=400, tol=1e-12, max_coarse_sweeps=1000)
        R, G, g = t(r64), t(gam), t(np.zeros(n))
        grid = eik.make_grid(R, h)
        params = eik.dd_params((N,), M, **kw)
        ws = torch.empty(eik.eik_dd_workspace_size(grid, params) + 256, dtype=torch.uint8, device=dev)
        u = torch.empty_like(R)
        st_dev = torch.zeros(eik.ctypes.sizeof(eik.DDStats), dtype=torch.uint8, device=dev)
        solve = lambda: eik.eik_dd_solve(grid, R, G, g, params, u, ws, st_dev, stream)
        prof = _profiled(torch, eik, solve)
        with ClockSampler(local_rank) as clk:
            ms = _timed(torch, solve, args.steps, args.warmup, flush, stream)
        st = eik.parse_dd_stats(st_dev)
        upd = st["fine_updates"] + st["coarse_updates"]
        k_ms = prof["dd1_iteration"]["total_ms"]
        # FP64: u in, r in, u out per fine update
        kern = ("dd1_iteration", st["fine_updates"] * 24 / (k_ms / 1e3) / 1e9)
        p_half = eik.dd_params((N,), M, **dict(kw, theta=0.5))
        st_half = torch.zeros_like(st_dev)
        ms_half = _timed(torch, lambda: eik.eik_dd_solve(grid, R, G, g, p_half, u, ws, st_half, stream), 2, 1,
                         flush, stream)
        sh = eik.parse_dd_stats(st_half)
        extra = {"dd_stats": {k: st[k] for k in ("iters", "converged", "fsm_sweeps_max", "coarse_sweeps_max",
                                                 "causal_rounds_max", "fine_updates", "coarse_updates")},
                 "theta_0.5": {"ms": ms_half, "iters": sh["iters"], "converged": sh["converged"]},
                 "kernel_ms": {k: v["total_ms"] for k, v in prof.items()},
                 "note": "one cooperative launch: one thread per subinterval (a chain of dependent "
                         "updates), the serial coarse work on one thread of CTA 0, so the kernel is bound by "
                         "latency, not by HBM"}
        hr = torch.from_numpy(r64).pin_memory()
        hu = torch.empty_like(hr).pin_memory()
        def e2e_step():
            R.copy_(hr, non_blocking=True)
            solve()
            hu.copy_(u, non_blocking=True)
        e2e_ms = _timed(torch, e2e_step, max(1, args.steps // 2), 1, flush, stream)
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": hr.numel() * 8,
               "d2h_bytes_per_step": hu.numel() * 8, "ms_per_step": e2e_ms}
        workload = {"workload": "dd1_bump_1024001", "N": N, "M": M, "theta": 1.0, "tol": 1e-12,
                    "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}
        unit, metric = "ms", "1-D DD (Sec. 3.1) solve to tol 1e-12, milliseconds"
        if rank == 0 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            _, so, _ = oracle.dd1(r64, gam, 0.0, h, N, M, **kw)
            dt = time.perf_counter() - t0
            cpu = {"value": dt * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": "the whole solve, FP64, %d iterations" % so["iters"]}
        value = ms
    elif args.workload == "dd3d257":
        w = inputs.workload_c2()
        R, G, g = t(w["r"].astype(np.float32)), t(w["gamma"]), t(w["g"].astype(np.float32))
        kw = dict(theta=THETA, max_iter=w["max_iter"], tol=TOL, max_coarse_sweeps=8)
        if args.theta == "adaptive":
            raise SystemExit("the adaptive weight is not built for the 3-D solve")
        kw["theta"] = float(args.theta)
        grid = eik.make_grid(R, w["h"])
        params = eik.dd_params(w["tiles"], w["c"], **kw)
        ws = torch.empty(eik.eik_dd_workspace_size(grid, params) + 256, dtype=torch.uint8, device=dev)
        u = torch.empty_like(R)
        st_dev = torch.zeros(eik.ctypes.sizeof(eik.DDStats), dtype=torch.uint8, device=dev)
        solve = lambda: eik.eik_dd_solve(grid, R, G, g, params, u, ws, st_dev, stream)
        prof = _profiled(torch, eik, solve)
        with ClockSampler(local_rank) as clk:
            ms = _timed(torch, solve, args.steps, args.warmup, flush, stream)
        st = eik.parse_dd_stats(st_dev)
        upd = st["fine_updates"] + st["coarse_updates"]
        fine_ms = prof["dd3_fine_subdomains"]["total_ms"]
        kern = ("dd3_fine_subdomains", st["fine_updates"] * BYTES_PER_UPDATE_F32 / (fine_ms / 1e3) / 1e9)
        extra = {"dd_stats": {k: st[k] for k in ("iters", "fsm_sweeps_max", "fine_updates", "coarse_updates")},
                 "kernel_ms": {k: v["total_ms"] for k, v in prof.items()}}
        # accuracy against the FP64 full-grid FSM (the discrete solution) and the
        # plain FP32 full-grid FSM at equal error (not part of the timed steps)
        try:
            uf, fst = eik.fsm(R.double(), G, g.double(), w["h"])
            fin = torch.isfinite(uf)
            umax = uf[fin].abs().max().item()

            def rel_err(x):
                return (x.double() - uf)[fin].abs().max().item() / umax

            dd_err = rel_err(u)

            def fsm_timed(ms_):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                flush.fill_(0.0)
                e0.record(stream)
                uu, ss = eik.fsm(R, G, g, w["h"], max_sweeps=ms_, sync=False)
                e1.record(stream)
                torch.cuda.synchronize()
                return uu, e0.elapsed_time(e1), eik.FsmStats.from_buffer_copy(bytes(ss.cpu().numpy())).sweeps

            lo, hi = 1, fst["sweeps"]
            while lo < hi:
                mid = (lo + hi) // 2
                uu, _, _ = fsm_timed(mid)
                if rel_err(uu) <= dd_err:
                    hi = mid
                else:
                    lo = mid + 1
            uu_eq, t_eq, _ = fsm_timed(lo)
            uu_full, t_full, full_sweeps = fsm_timed(100000)
            extra["accuracy"] = {"rel_max_err_vs_fp64_fsm": dd_err, "fp64_fsm_sweeps": fst["sweeps"]}
            extra["fsm_baseline_f32"] = {"sweeps_to_equal_error": lo, "time_to_equal_error_ms": t_eq,
                                         "rel_max_err_at_equal": rel_err(uu_eq), "converged_sweeps": full_sweeps,
                                         "time_to_convergence_ms": t_full,
                                         "rel_max_err_converged": rel_err(uu_full),
                                         "dd_over_fsm_time_at_equal_error": ms / t_eq}
        except Exception as e:  # noqa: BLE001
            extra["fsm_baseline_f32"] = {"unavailable": str(e)[:160]}
        hr = torch.from_numpy(w["r"].astype(np.float32)).pin_memory()
        hu = torch.empty_like(hr).pin_memory()
        def e2e_step():
            R.copy_(hr, non_blocking=True)
            solve()
            hu.copy_(u, non_blocking=True)
        e2e_ms = _timed(torch, e2e_step, max(1, args.steps // 2), 1, flush, stream)
        e2e = {"value": upd / (e2e_ms / 1e3) / 1e9, "unit": "Gupdates/s", "h2d_bytes_per_step": hr.numel() * 4,
               "d2h_bytes_per_step": hu.numel() * 4, "ms_per_step": e2e_ms}
        workload = {"workload": "dd3d_257_pointsrc_8x8x8_c8", "n": 257, "tiles": 8, "coarse_ratio": 8, **kw,
                    "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}
        unit, metric = "Gupdates/s", "3-D DD: local solves per second, 257^3"
        if rank == 0 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            _, so, _ = oracle.dd(w["r"].astype(np.float32).astype(np.float64), w["gamma"], w["g"], w["h"],
                                 w["tiles"], w["c"], theta=0.2, max_iter=0, tol=0.0, max_coarse_sweeps=8)
            dt = time.perf_counter() - t0
            cu = so["fine_updates"] + so["coarse_updates"]
            cpu = {"value": cu / dt / 1e9, "unit": unit, "cores": 1, "kind": "oracle",
                   "sample": "Step 1 + one fine pass over all 512 subdomains (max_iter=0), %.1f s" % dt}
        value = upd * world / (ms / 1e3) / 1e9
    elif args.workload == "obstacles":
        # Sec. 4 mazes and obstacles / random checkerboard at the paper's sizes:
        # time to solution (stop at a coarse update below 1e-6, cap 60) of the
        # DD against the plain FP32 FSM at equal error, each workload solved once
        # per step
        ws_ = [inputs.workload_fast_strip(), inputs.workload_maze(), inputs.workload_checkerboard()]
        kw = dict(theta=THETA, max_iter=60, tol=1e-6, max_coarse_sweeps=8)
        if args.theta == "adaptive":
            kw.update(theta_adaptive=True, theta_cap=THETA_CAP)
        else:
            kw["theta"] = float(args.theta)
        cases = []
        for q in ws_:
            R, G, g = t(q["r"].astype(np.float32)), t(q["gamma"]), t(q["g"].astype(np.float32))
            cases.append((q, R, G, g))

        def solve_all():
            out = []
            for q, R, G, g in cases:
                out.append(eik.dd_solve(R, G, g, q["h"], q["tiles"], q["c"], sync=False, **kw))
            return out
        prof = _profiled(torch, eik, solve_all)
        with ClockSampler(local_rank) as clk:
            ms = _timed(torch, solve_all, args.steps, args.warmup, flush, stream)
        res = solve_all()
        torch.cuda.synchronize()
        per = []
        upd = 0
        fine_upd = 0
        for (q, R, G, g), (u, stt) in zip(cases, res):
            s2 = eik.parse_dd_stats(stt)
            upd += s2["fine_updates"] + s2["coarse_updates"]
            fine_upd += s2["fine_updates"]
            uf, _ = eik.fsm(R.double(), G, g.double(), q["h"])
            umax = uf.abs().max().item()
            err = lambda x: (x.double() - uf).abs().max().item() / umax
            dd_err = err(u)
            t_dd = _timed(torch, lambda: eik.dd_solve(R, G, g, q["h"], q["tiles"], q["c"], sync=False, **kw), 3, 1,
                          flush, stream)
            uu, fst = eik.fsm(R, G, g, q["h"])
            target = max(dd_err, err(uu))
            lo, hi = 1, fst["sweeps"]
            while lo < hi:
                mid = (lo + hi) // 2
                if err(eik.fsm(R, G, g, q["h"], max_sweeps=mid)[0]) <= target:
                    hi = mid
                else:
                    lo = mid + 1
            t_f = _timed(torch, lambda: eik.fsm(R, G, g, q["h"], max_sweeps=lo, sync=False), 3, 1, flush, stream)
            per.append({"workload": q["name"], "n": q["r"].shape[0], "tiles": q["tiles"][0], "coarse_ratio": q["c"],
                        "iters": s2["iters"], "converged": s2["converged"], "dd_ms": t_dd,
                        "rel_max_err_vs_fp64_fsm": dd_err, "fsm_f32_sweeps_to_equal_error": lo,
                        "fsm_f32_ms_to_equal_error": t_f, "dd_over_fsm": t_dd / t_f})
        fine_ms = prof["dd_fine_subdomains"]["total_ms"]
        kern = ("dd_fine_subdomains", fine_upd * BYTES_PER_UPDATE_F32 / (fine_ms / 1e3) / 1e9)
        extra = {"per_workload": per}
        hr = [torch.from_numpy(q["r"].astype(np.float32)).pin_memory() for q, *_ in cases]
        hu = [torch.empty_like(x).pin_memory() for x in hr]

        def e2e_step():
            for (q, R, G, g), x in zip(cases, hr):
                R.copy_(x, non_blocking=True)
            for (u, _), y in zip(solve_all(), hu):
                y.copy_(u, non_blocking=True)
        e2e_ms = _timed(torch, e2e_step, max(1, args.steps // 2), 1, flush, stream)
        e2e = {"value": e2e_ms, "unit": "ms", "h2d_bytes_per_step": sum(x.numel() * 4 for x in hr),
               "d2h_bytes_per_step": sum(x.numel() * 4 for x in hu), "ms_per_step": e2e_ms}
        workload = {"workload": "sec4_obstacles_fast_strip501_maze501_checkerboard1401", **kw,
                    "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}
        unit, metric = "ms", "Sec. 4 obstacle workloads: DD time to solution, the three solved in sequence"
        if rank == 0 and not args.no_cpu_baseline:
            q = ws_[0]
            t0 = time.perf_counter()
            _, so, _ = oracle.dd(q["r"].astype(np.float32).astype(np.float64), q["gamma"], q["g"], q["h"],
                                 q["tiles"], q["c"], **kw)
            dt = time.perf_counter() - t0
            cpu = {"value": dt * 1e3, "unit": "ms", "cores": 1, "kind": "oracle",
                   "sample": "the fast strip alone, full solve, FP64 (%d iterations)" % so["iters"]}
        value = ms
    else:
        w = inputs.workload_c4()
        n, h = w["n"], w["h"]
        R = t(w["r0"].astype(np.float32))
        g0 = torch.zeros_like(R)
        rec = torch.tensor([j * n + n - 1 for j in w["rec_rows"]], device=dev)
        S = len(w["src_rows"])
        gams = torch.zeros((S, n, n), dtype=torch.uint8, device=dev)
        for s_, srow in enumerate(w["src_rows"]):
            gams[s_, srow, 0] = 1
        gz = torch.zeros((S, n, n), dtype=torch.float32, device=dev)
        ut, _ = eik.fsm_many(t(w["r_true"].astype(np.float32)), gams, gz, h)
        data = ut.reshape(S, -1)[:, rec].clone()
        del ut

        # the forward of every source by the DD as configured (16 x 16
        # subdomains, coarse ratio 8, weight 0, stop at a coarse update below
        # 1e-6): one batched solve over the sources, built once for R
        many_dd = eik.ManyDD(R, gams, gz, h, (16, 16), 8, theta=0.0, max_iter=42, tol=TOL,
                             max_coarse_sweeps=MAX_COARSE_SWEEPS)

        def gradient(dd=many_dd):
            # all sources in one forward (the batched DD, or eik_fsm_many) and
            # one backward (eik_dd_adjoint_many, gradients summed in the library)
            rr = R.detach().requires_grad_(True)
            u = eik.EikonalSolveMany.apply(rr, gams, gz, h, dd)
            L = 0.5 * ((u.reshape(S, -1)[:, rec] - data) ** 2).sum()
            L.backward()
            return rr.grad
        prof = _profiled(torch, eik, gradient)
        with ClockSampler(local_rank) as clk:
            ms = _timed(torch, gradient, args.steps, args.warmup, flush, stream)
        fs = prof.get("dd_batch_fine_subdomains", prof.get("dd_fine_subdomains", {"total_ms": float("nan")}))
        fine_name = "dd_batch_fine_subdomains" if "dd_batch_fine_subdomains" in prof else "dd_fine_subdomains"
        ms_fsm_fwd = _timed(torch, lambda: gradient(None), args.steps, args.warmup, flush, stream)
        dst = many_dd.stats()
        extra = {"kernel_ms": {k: v["total_ms"] for k, v in prof.items()}, "sources": S,
                 "receivers": len(w["rec_rows"]),
                 "dd_forward": {"iters_max": max(x["iters"] for x in dst),
                                "converged": sum(x["converged"] for x in dst)},
                 "fsm_forward_ms_per_step": ms_fsm_fwd}
        # fine updates of every source for the algorithmic byte count of the subdomain kernel
        fwd_upd = sum(x["fine_updates"] for x in dst)
        kern = (fine_name, fwd_upd * BYTES_PER_UPDATE_F32 / (fs["total_ms"] / 1e3) / 1e9)
        hr = torch.from_numpy(w["r0"].astype(np.float32)).pin_memory()
        hg = torch.empty_like(hr).pin_memory()
        def e2e_step():
            R.copy_(hr, non_blocking=True)
            gr = gradient()
            hg.copy_(gr, non_blocking=True)
        e2e_ms = _timed(torch, e2e_step, max(1, args.steps // 2), 1, flush, stream)
        e2e = {"value": S / (e2e_ms / 1e3), "unit": "sources/s", "h2d_bytes_per_step": hr.numel() * 4,
               "d2h_bytes_per_step": hg.numel() * 4, "ms_per_step": e2e_ms}
        workload = {"workload": "tomography_1025_64src_256rec", "n": n, "sources": 64, "receivers": 256,
                    "forward": "DD (16 x 16 subdomains, coarse ratio 8, weight 0, stop at 1e-6), all sources in one "
                               "batched solve; the u of the converged solve is the only forward state kept",
                    "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"}
        unit, metric = "sources/s", "travel-time tomography: gradient dL/dr, sources (forward + adjoint) per second"
        if rank == 0 and not args.no_cpu_baseline:
            t0 = time.perf_counter()
            gam = np.zeros((n, n), np.uint8)
            gam[w["src_rows"][0], 0] = 1
            r64 = w["r0"].astype(np.float32).astype(np.float64)
            u0, so, _ = oracle.dd(r64, gam, np.zeros((n, n)), h, (16, 16), 8, theta=0.0, max_iter=42, tol=TOL,
                                  max_coarse_sweeps=MAX_COARSE_SWEEPS, parallel=True)
            dJ = np.zeros((n, n))
            dJ[w["rec_rows"], n - 1] = 1.0
            oracle.adjoint(r64, gam, u0, dJ, h)
            dt = time.perf_counter() - t0
            cpu = {"value": 1.0 / dt, "unit": unit, "cores": host_cpu()["threads"], "kind": "oracle",
                   "sample": "one source: forward DD (16 x 16, c = 8, %d iterations, OpenMP) + adjoint "
                             "(serial), FP64, %.1f s" % (so["iters"], dt)}
        value = S * world / (ms / 1e3)
    if rank == 0:
        line = {"metric": metric, "value": value, "unit": unit, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": unit != "ms", "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if args.workload == "dd1bump" else "f32", "data": "synthetic",
                "config": workload,
                "roofline": {"bound": "hbm", "achieved": kern[1], "peak": peak, "unit": "GB/s",
                             "frac": kern[1] / peak, "traffic": None, "kernel": kern[0], "peak_source": peak_kind,
                             "algorithmic_bytes": "%d B per node update (u in, r in, u out)" %
                                                  (24 if args.workload == "dd1bump" else 12)},
                "gpu_launches": sum(v["launches"] for v in prof.values()) * args.steps, "e2e": e2e,
                "clocks": clk.summary(), "cpu_baseline": cpu, **extra}
        print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
