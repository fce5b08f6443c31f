"""Benchmark: converged implicit time steps of the MLQD multigrid-in-frequency solver.

Workload (default): the fc_1024 slab -- 500 cells, double S32 (64 directions), 1024
log-spaced groups 1e-5..1e2 keV, grids {1024, 256, 64, 16, 1}, Fleck-Cummings opacity,
1 keV Planck inflow, cold start, dt = 1e-3 sh, eps = 1e-8, plain FP64.  Synthetic inputs
(the paper's only workload is this synthetic test problem).

A "step" is one converged time step of Algorithm 3 (sweeps + group LOQD on the grid
hierarchy + grey LOQD/MEB Newton).  value = sweep cell-angle-group updates per second of
wall time over the timed steps (all ranks); ms_per_step = mean time of a converged step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--precision fp64|mixed] [--cycle V|W]
Under torchrun each rank runs an independent replica of the slab (replicas only: the
solver's data path has no cross-GPU exchange on one slab).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2011_05427_gb300 import workloads as W  # noqa: E402

METRIC = "sweep cell·angle·group updates/s; ms per converged step vs plain FP64"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    def __init__(self, index=0):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.file.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.file.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def sweep_roofline(trt, s, cfg, reps=20):
    """Time the sweep kernels (K2 + its moment finalize) alone with CUDA events on the
    solver's stream, on the step's own sized inputs; algorithmic bytes per launch =
    updates x 4 intensity values + per (cell, group) sigma_t, e read and f written."""
    import torch
    r = W.rng(5)
    T = W.random_temperatures(r, cfg.n_cells, 1e-3, 1.0)
    sig, em, _ = s.k_opacity(T)
    rdt = torch.float32 if s.precision & trt.TRT_SWEEP_FP32 else torch.float64
    Iold = torch.rand((s.M, s.nx, 2, s.ldG), dtype=rdt, device=s.device)
    Inew = torch.empty_like(Iold)
    f = torch.empty((s.G, s.nx), dtype=torch.float64, device=s.device)
    b = [torch.empty(s.G, dtype=torch.float64, device=s.device) for _ in range(4)]
    L = trt.lib()
    args = (s.h, float(cfg.dt), sig.data_ptr(), em.data_ptr(), Iold.data_ptr(), Inew.data_ptr(),
            f.data_ptr(), *[x.data_ptr() for x in b])
    for _ in range(3):
        assert L.trt_k_sweep(*args) == 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(s.stream)
    for _ in range(reps):
        L.trt_k_sweep(*args)
    ev1.record(s.stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    esz = 4 if s.precision & trt.TRT_SWEEP_FP32 else 8
    upd = cfg.n_cells * cfg.M * cfg.G
    bytes_alg = upd * 4 * esz + cfg.n_cells * cfg.G * (2 * 8 + 8)
    hbm, src = peaks()
    ach = bytes_alg / (ms * 1e-3) / 1e9
    return dict(ms=ms, bytes=bytes_alg, achieved=ach, peak=hbm, src=src, updates=upd,
                upd_per_s=upd / (ms * 1e-3))


def run_ours(args):
    import torch
    from paper_2011_05427_gb300 import trt
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    cfg = W.fc_1024(args.cycle)
    upd_sweep = cfg.updates_per_sweep()
    s = trt.Solver.from_slab(cfg, precision=args.precision, device=f"cuda:{local}")
    for _ in range(args.warmup):
        s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps)
    clk = Clocks(local) if rank == 0 else None
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    stats = [s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps) for _ in range(args.steps)]
    ev1.record(s.stream)
    torch.cuda.synchronize()
    barrier(ws)
    wall = time.perf_counter() - t0
    clocks = clk.stop() if clk else None
    dev_s = ev0.elapsed_time(ev1) * 1e-3
    t_max = max_over_ranks(dev_s, ws)
    n_ti = sum(x["n_ti"] for x in stats)
    launches = sum(x.get("n_kernels", 0) for x in stats)
    total_upd = sum_over_ranks(n_ti * upd_sweep, ws)
    value = total_upd / t_max
    ms_step = t_max / args.steps * 1e3

    # e2e: the public API from host data -- create (uploads the host-built constants and
    # initial state), K steps each followed by a read of the step's result to pinned host
    # memory, destroy.
    res_bytes = 8 * (cfg.n_cells + cfg.G * cfg.n_cells + cfg.G * (cfg.n_cells + 1) +
                     2 * cfg.n_cells + 1)
    torch.cuda.synchronize()
    barrier(ws)
    te = time.perf_counter()
    s2 = trt.Solver.from_slab(cfg, precision=args.precision, device=f"cuda:{local}")
    e2e_ti = 0
    for _ in range(args.steps):
        st = s2.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps)
        e2e_ti += st["n_ti"]
        s2.moments()
    torch.cuda.synchronize()
    barrier(ws)
    te = max_over_ranks(time.perf_counter() - te, ws)
    h2d = 8 * (cfg.n_cells + 2 * (cfg.G + 1) + cfg.G * cfg.n_cells * 2 + cfg.G * (cfg.n_cells + 1)
               + 10 * cfg.G + 2 * cfg.M) + cfg.G * 8
    s2.close()
    e2e_val = sum_over_ranks(e2e_ti * upd_sweep, ws) / te

    roof = sweep_roofline(trt, s, cfg)
    if rank != 0:
        s.close()
        return
    out = {
        "metric": METRIC,
        "value": value,
        "unit": "updates/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64",
        "data": "synthetic (Fleck-Cummings slab, seeded, no dataset)",
        "config": {"workload": f"fc_1024: 500 cells, 64 directions (double S32), 1024 groups, "
                               f"grids 1024/256/64/16/1, {args.cycle}-cycle l_max {cfg.l_max}, "
                               f"dt 1e-3 sh, eps 1e-8, {args.precision}",
                   "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (intensity arrays 1 GB)",
                   "n_ti_per_step": n_ti / args.steps,
                   "n_c_per_step": sum(x["n_c"] for x in stats) / args.steps,
                   "n_lo_per_step": sum(x["n_lo"] for x in stats) / args.steps},
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": res_bytes,
                "note": "create + K steps + per-step moments read; state stays on device"},
        "gpu_launches": launches,
        "roofline": {"bound": "hbm", "achieved": roof["achieved"], "peak": roof["peak"],
                     "unit": "GB/s", "frac": roof["achieved"] / roof["peak"], "traffic": None,
                     "kernel": "k_sweep + k_sweep_finalize", "ms": roof["ms"],
                     "peak_source": roof["src"]},
        "clocks": clocks,
    }
    if args.cpu_baseline and ws == 1:
        out["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(out), flush=True)
    s.close()


def oracle_sample(orc, cfg):
    """Bounded oracle sample of the same workload: one fixed-iteration time step of
    fc_1024 (s = 0 low-order phase, one sweep, one more low-order phase; one cycle each)."""
    p = orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                    cfg.T_left, cfg.T_right)
    t = time.perf_counter()
    st, c = p.step(cfg.dt, cfg.cycle, 1, -1.0, max_outer=2)
    dt = time.perf_counter() - t
    return c["n_ti"] * cfg.updates_per_sweep(), dt


def cpu_baseline(args):
    from oracle import orc
    cfg = W.fc_1024(args.cycle)
    upd, dt = oracle_sample(orc, cfg)
    return {"value": upd / dt, "unit": "updates/s", "cores": 1, "kind": "oracle",
            "sample": "oracle (FP64 C, 1 thread): one fixed-iteration step of fc_1024 "
                      "(s=0 phase + 1 sweep + 1 phase, 1 cycle each), "
                      f"{dt:.1f} s; updates counted over the sweep"}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import orc
    cfg = W.fc_1024(args.cycle)
    for _ in range(args.warmup):
        oracle_sample(orc, cfg)
    tot_u = 0.0
    tot_t = 0.0
    for _ in range(args.steps):
        u, dt = oracle_sample(orc, cfg)
        tot_u += u
        tot_t += dt
    v = tot_u / tot_t
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "updates/s",
           "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_t / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (Fleck-Cummings slab, seeded, no dataset)",
           "config": {"workload": "fc_1024 (oracle sample: one fixed-iteration step, s=0 phase "
                                  "+ 1 sweep + 1 phase)", "parallelism": "1 host thread"},
           "cpu_baseline": {"kind": "oracle", "cores": 1, "value": v, "unit": "updates/s",
                            "sample": "each step: one fixed-iteration step of fc_1024"},
           "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed", "sweep32", "lo32"])
    ap.add_argument("--cycle", default="W", choices=["V", "W"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-step", action="store_true",
                    help="run the warm-up steps and one more step, print nothing (for ncu)")
    args = ap.parse_args()
    if args.profile_step:
        from paper_2011_05427_gb300 import trt
        cfg = W.fc_1024(args.cycle)
        s = trt.Solver.from_slab(cfg, precision=args.precision, device="cuda:0")
        for _ in range(args.warmup + 1):
            s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps)
        s.close()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
