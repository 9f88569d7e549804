"""Benchmark of the two-scale domain-decomposition Eikonal solver on one GB300.

Workload (default): 2-D 4097^2 grid (h = 1/4096), slowness r = clip(1 + 0.3x +
0.4 F/max|F|, 0.2) with F a sum of 32 seeded Fourier modes, |k| in [64, 128]
(eps = 1/64); Gamma = the whole left edge x = 0, g = 0; 16 x 16 subdomains,
coarse ratio 16 (coarse grid 257^2); FP32 storage; theta = 0.2; stop when the
coarse update falls below 1e-6 or after 2*16 + 10 = 42 iterations.

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
THETA = 0.2
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


def cpu_oracle_sample(r32, gamma, g, h):
    """Oracle (FP64, serial) on a bounded sample of the workload: Step 1 and
    one fine pass over all 256 subdomains (max_iter = 0)."""
    import oracle
    t0 = time.perf_counter()
    _, st, _ = oracle.dd(r32.astype(np.float64), gamma, g.astype(np.float64), h, (TILES, TILES), COARSE,
                         theta=THETA, max_iter=0, tol=TOL, max_coarse_sweeps=MAX_COARSE_SWEEPS)
    dt = time.perf_counter() - t0
    upd = st["fine_updates"] + st["coarse_updates"]
    return upd / dt / 1e9, dt, upd


def run_reference(args):
    """--impl reference: the oracle as it stands, on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    r32, gamma, g, h = make_workload()
    vals = []
    for i in range(args.warmup + args.steps):
        v, dt, upd = cpu_oracle_sample(r32, gamma, g, h)
        if i >= args.warmup:
            vals.append((v, dt))
    value = statistics.mean(v for v, _ in vals)
    ms = statistics.mean(dt for _, dt in vals) * 1e3
    sample = ("4097^2 workload, Step 1 + one fine pass over all 256 subdomains (max_iter=0), "
              "FP64 serial oracle; value = local solves executed / wall time")
    line = {"metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "c1_2d_4097_leftedge_16x16_c16", "sample": "max_iter=0"},
            "cpu_baseline": {"value": value, "unit": "Gupdates/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Gupdates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

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
    if dist is not None:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = upd_total * world / (total_ms / 1e3) / 1e9
    cells = float(N_SIDE) * N_SIDE

    # roofline of the dominant kernel (event-timed inside the timed region)
    peak, peak_kind = load_peaks()
    fine = prof.get("dd_fine_subdomains", {"total_ms": float("nan"), "launches": 0})
    fine_upd = stats["fine_updates"] * args.steps
    achieved = fine_upd * BYTES_PER_UPDATE_F32 / (fine["total_ms"] / 1e3) / 1e9
    fine_upd_launch = stats["fine_updates"] / max(1, fine["launches"] // args.steps)
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

        # smallest FP32 FSM sweep count whose error is at most the DD error
        lo, hi = 1, fst["sweeps"]
        while lo < hi:
            mid = (lo + hi) // 2
            uu, _ = eik.fsm(R, G, g, h, max_sweeps=mid)
            if rel_err(uu) <= dd_err:
                hi = mid
            else:
                lo = mid + 1
        uu_eq, t_eq, _ = fsm_timed(lo)
        uu_full, t_full, full_sweeps = fsm_timed(100000)
        fsm_line = {"sweeps_to_equal_error": lo, "time_to_equal_error_ms": t_eq,
                    "rel_max_err_at_equal": rel_err(uu_eq), "converged_sweeps": full_sweeps,
                    "time_to_convergence_ms": t_full, "rel_max_err_converged": rel_err(uu_full),
                    "dd_over_fsm_time_at_equal_error": ms_per_step / t_eq}
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
        try:
            v, dt, upd = cpu_oracle_sample(r32, gamma, g32, h)
            cpu = {"value": v, "unit": "Gupdates/s", "cores": 1, "kind": "oracle",
                   "sample": "Step 1 + one fine pass over all 256 subdomains of the same 4097^2 workload "
                             "(max_iter=0), %.1f s, %d local solves" % (dt, upd)}
        except Exception as e:  # noqa: BLE001
            cpu = {"value": None, "unit": "Gupdates/s", "cores": 1, "kind": "oracle", "sample": str(e)[:160]}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gupdates/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "c1_2d_4097_leftedge_16x16_c16", "n": N_SIDE, "tiles": TILES,
                       "coarse_ratio": COARSE, "theta": THETA, "max_iter": MAX_ITER, "tol": TOL,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": "replicas"},
            "time_to_solution_ms": ms_per_step,
            "gcells_per_s": cells * world / (ms_per_step / 1e3) / 1e9,
            "dd_stats": {k: stats[k] for k in ("iters", "converged", "fsm_sweeps_max", "coarse_sweeps_max",
                                              "fine_updates", "coarse_updates", "last_delta")},
            "accuracy": acc,
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


if __name__ == "__main__":
    sys.exit(main())
