"""Benchmark: converged implicit time steps of the MLQD multigrid-in-frequency solver.

Workload (default): the fc_1024 slab -- 500 cells, double S32 (64 directions), 1024
log-spaced groups 1e-5..1e2 keV, grids {1024, 256, 64, 16, 1}, Fleck-Cummings opacity,
1 keV Planck inflow, cold start, dt = 1e-3 sh, eps = 1e-8, plain FP64.  Synthetic inputs
(the paper's only workload is this synthetic test problem).

A "step" is one converged time step of Algorithm 3 (sweeps + group LOQD on the grid
hierarchy + grey LOQD/MEB Newton).  value = sweep cell-angle-group updates per second of
wall time over the timed steps (all ranks); ms_per_step = mean time of a converged step.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--precision fp64|mixed|sweep32|lo32|lopair|sweep32_lopair] [--cycle V|W] [--no-compare]
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
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=self.file, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def ready(self, limit_s=2.0):
        """Wait (at most limit_s) until the sampler has written its first sample, so that
        the samples that follow fall into the region timed next."""
        t0 = time.perf_counter()
        while self.p is not None and time.perf_counter() - t0 < limit_s:
            if self.p.poll() is not None or os.path.getsize(self.file.name) > 0:
                return
            time.sleep(0.01)

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


def dist_init(backend=None):
    """One process per GPU (torchrun's RANK / LOCAL_RANK / WORLD_SIZE).  The ranks are
    replicas: each steps its own slab; the only collectives are the timing barrier and the
    max / sum of scalars below (NCCL on GPUs, gloo for the host-side tests)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend or "nccl")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce(x, ws, op):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=getattr(dist.ReduceOp, op))
    return float(t.item())


def max_over_ranks(x, ws):
    return _reduce(x, ws, "MAX")


def sum_over_ranks(x, ws):
    return _reduce(x, ws, "SUM")


def job_throughput(units, seconds, ws):
    """Whole-job throughput of N replicas: the units all ranks processed over the slowest
    rank's time (weak scaling: each rank's work is fixed)."""
    return sum_over_ranks(units, ws) / max_over_ranks(seconds, ws)


# FP64 operations per sweep update (one cell, direction, group) of the simple corner
# balance solve and its moments, FMA = 2, the one division = 1: diagonal mu/2 +
# sigma_t h/2 (1), determinant (2), division (1), the two right-hand sides (4 + 2), the
# two corner values (4 + 4), their sum (1), the two angular moment accumulations (4) = 23.
FLOP_PER_UPDATE = 23
# FP64 peak of the part: 152 SMs x 2070 MHz x 2 FP64 FMA per clock per SM x 2 = 1.26e12,
# the nominal 1.25 TFLOP/s; the bench measures it in the run (trt_fp64_peak) and keeps the
# nominal figure only if the probe fails.
FP64_PEAK_TFLOPS = 1.25
_fp64_peak_cache = {}


def fp64_peak(trt, local=0):
    """(peak TFLOP/s, source): the FP64 FMA rate measured in this run, else the nominal."""
    if local not in _fp64_peak_cache:
        try:
            v = max(trt.fp64_peak(device=f"cuda:{local}") for _ in range(3))
            _fp64_peak_cache[local] = (v, "measured in this run: FP64 FMA chains on every SM "
                                          "(trt_fp64_peak), best of 3")
        except Exception as e:   # keep the bench line; say where the peak came from
            _fp64_peak_cache[local] = (FP64_PEAK_TFLOPS, f"nominal (probe failed: {e})")
    return _fp64_peak_cache[local]
# FP64 instruction issue of the part: one warp-wide FP64 instruction occupies a
# sub-partition's FP64 pipe for 64 cycles when one warp runs (measured), 76 when all four
# sub-partitions are busy, i.e. the FMA rate trt_fp64_peak measures (~1.056 TFLOP/s, 84%
# of the nominal 1.25); the instruction-rate fraction below divides by that measured rate.
# FP64 thread instructions per update (ncu, DFMA + DMUL + DADD over the updates of one
# fc_1024 launch): the strip sweep 17.6 (11.0 + 4.5 + 2.1), the paired sweep 13.5 (9.0 +
# 3.0 + 1.5: t and s formed once per pair of directions); the FLOP ceiling of a mix is
# 23 / (2 x instructions) of the FMA rate.
FP64_INST_PEAK = 152 * 4 * 2.07e9 / 64 * 32
FP64_INST_PER_UPDATE = {"strip": 17.6, "pair": 13.5}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of the
# sweep and its finalize on the fc_1024 workload), valid while the kernel sources hash to
# `sha` and the tuned tile (D, shape) is the captured one.
TRAFFIC = {
    # k_prescale64 + k_sweep_pair<4,2> + k_sweep_finalize<double>: the t, s scratch and the
    # 16 partial-moment tiles make it 1.70 x the algorithmic bytes (FP64-bound, not HBM)
    "sweep_fp64": {"files": ("sweep64.cu", "sweep.cu"), "sha": "f4740f50793cb9cb", "tile": (4, 4),
                   "bytes": 8202496 + 785604096 + 881712128 + 131672320 + 1171712},
    "sweep_fp32": {"files": ("sweepf.cu", "sweep.cu"), "sha": "1c55093d94e37681", "tile": (16, 0),
                   "bytes": 270072576 + 243014656 + 33098752 + 0},
}


def _src_sha(names):
    """SHA-256 of the sources' code: `//` comments and blank lines are left out, so that
    a comment edit does not void a measurement of unchanged kernels."""
    import hashlib
    import re
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2011_05427_gb300", "csrc", name)) as f:
            for line in f:
                code = re.sub(r"//.*", "", line).rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def _traffic(key, tile):
    t = TRAFFIC.get(key)
    if not t or t["bytes"] is None or tuple(tile) != t["tile"]:
        return None
    return t["bytes"] if _src_sha(t["files"]) == t["sha"] else None


def sweep_kernel(fp32, D, shape):
    """The kernels one sweep launches for tile (D, shape) (the library's shape table)."""
    if not fp32:
        if shape in (3, 4):   # paired sweep: its pre-scaled inputs, the sweep, the finalize
            S, NS = {3: (8, 2), 4: (4, 2)}[shape]
            return f"k_prescale64 + k_sweep_pair<{S},{NS}> + k_sweep_finalize<double>"
        S, NS = {0: (8, 2), 1: (16, 2), 2: (8, 3)}[shape]
        return f"k_sweep<double,double,{S},{NS}> + k_sweep_finalize<double>"
    if shape == 6 or D not in (4, 8, 16):   # the strip sweep (tile heights without a lean kernel)
        k = "k_sweep<float,float,16,2>"
    else:   # lean sweeps: groups per lane, strip, buffers, directions per CTA
        gpl, S, NS = {0: (1, 8, 4), 1: (1, 16, 2), 2: (1, 8, 3), 3: (1, 8, 2), 4: (2, 8, 2),
                      5: (2, 8, 4)}[shape]
        k = "k_sweepf<%d,%d,%d,%d>" % (gpl, S, NS, D)
    return k + " + k_sweep_finalize<float>"


def sweep_roofline(trt, s, cfg, fp32=False, local=0, reps=20):
    """Time the step's own sweep (K2 + its moment finalize; FP32 mode: the pre-scaled FP32
    inputs) with CUDA events on the solver's stream, `reps` launches after a warm-up, the
    intensity arrays (0.5 GB FP32 / 1 GB FP64 each) larger than L2.  FP64: bound by FP64
    issue; achieved = FLOP_PER_UPDATE x updates per launch / launch time.  FP32: bound by
    HBM; algorithmic bytes per launch = updates x 4 intensity values (2 corners read, 2
    written) + per (cell, group) sigma_t h/2 and h e/2 read and f written."""
    own = s is None
    tile = None
    if own:
        s = trt.Solver.from_slab(cfg, precision="sweep32" if fp32 else "fp64",
                                 device=f"cuda:{local}")
        tile = s.autotune(cfg.dt, reps=10)
    D, shape = s.sweep_tile()
    if D == 0:   # the library default: the largest power of two <= 8 dividing N
        D = max(d for d in (1, 2, 4, 8) if cfg.N % d == 0)
    ms = s.sweep_time(cfg.dt, reps=reps)
    if own:
        s.close()
    upd = cfg.n_cells * cfg.M * cfg.G
    if fp32:
        bytes_alg = upd * 4 * 4 + cfg.n_cells * cfg.G * (2 * 4 + 8)
        hbm, src = peaks()
        ach = bytes_alg / (ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
                "frac": ach / hbm, "traffic": _traffic("sweep_fp32", (D, shape)),
                "kernel": sweep_kernel(True, D, shape), "ms": ms,
                "algorithmic_bytes": bytes_alg,
                "peak_source": f"{src} (MEASURED_PEAKS hbm_gbs, copy)",
                "updates_per_s": upd / (ms * 1e-3)}
    else:
        kind64 = "pair" if shape in (3, 4) else "strip"
        flops = FLOP_PER_UPDATE * upd
        ach = flops / (ms * 1e-3) / 1e12
        pk, pk_src = fp64_peak(trt, local)
        roof = {"bound": "alu", "achieved": ach, "peak": pk, "unit": "TFLOP/s",
                "frac": ach / pk, "traffic": _traffic("sweep_fp64", (D, shape)),
                "kernel": sweep_kernel(False, D, shape), "ms": ms,
                "algorithmic_flops": flops,
                "peak_source": pk_src,
                "peak_nominal": FP64_PEAK_TFLOPS,
                "hbm_frac": upd * 32 / (ms * 1e-3) / 1e9 / peaks()[0],
                "fp64_inst_per_update": FP64_INST_PER_UPDATE[kind64],
                "fp64_inst_frac": FP64_INST_PER_UPDATE[kind64] * upd / (ms * 1e-3) /
                                  (pk * 1e12 / 2),
                "updates_per_s": upd / (ms * 1e-3)}
    if tile:
        roof["tile"] = {"D": tile[0], "S": tile[1], "NS": tile[2], "shape": shape}
    return {"roofline": roof, "ms": ms}


# Algorithm 3's l_max (cycles per low-order phase) for each form and cycle: the fastest of
# l_max = 1 .. 4 per converged fc_1024 step as measured by --lmax-sweep on a GB300.  FP64
# sweeps are dear, so the FP64 form spends more cycles per sweep (V: l_max 3); FP32 sweeps
# are cheap next to a cycle (V: l_max 2).  W and F take l_max 1: one such cycle already
# visits every grid.
def tuned_lmax(precision, cycle):
    if cycle != "V":
        return 1
    return 3 if precision in ("fp64", "lo32", "lopair") else 2


def timed_steps(trt, cfg, precision, cycle, steps, warmup, local, ws, clocks=False,
                l_max=None):
    """warmup + steps converged steps of one solver on the device; returns the device time
    of the timed steps (max over ranks), their stats, the clock record and the solver."""
    import torch
    s = trt.Solver.from_slab(cfg, precision=precision, device=f"cuda:{local}")
    s.tile = s.autotune(cfg.dt, reps=10)   # sweep tile for this problem (state unchanged)
    if l_max is None:
        l_max = tuned_lmax(precision, cycle)
    s.l_max = l_max
    for _ in range(warmup):
        s.step(cfg.dt, cycle, l_max, cfg.eps)
    clk = Clocks(local) if clocks else None
    if clk:
        clk.ready()
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(s.stream)
    stats = [s.step(cfg.dt, cycle, l_max, cfg.eps) for _ in range(steps)]
    ev1.record(s.stream)
    torch.cuda.synchronize()
    barrier(ws)
    rec = clk.stop() if clk else None
    t = max_over_ranks(ev0.elapsed_time(ev1) * 1e-3, ws)
    return t, stats, rec, s


def bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (MEASURED_PEAKS bf16_tflops, burst)"
    except Exception:
        return 1900.0, "fallback"


def mlp_bench(local, rows=512000, reps=10):
    """Closure network on the tensor cores: inference over fc_1024's 512,000 (cell, group)
    rows and one training step of 8192 rows, CUDA events on the network's stream."""
    import torch
    from paper_2011_05427_gb300 import closure, mlp
    dev = f"cuda:{local}"
    net = mlp.MLP(closure._init(7), device=dev)
    g = torch.Generator(device=dev)
    g.manual_seed(3)
    x = torch.rand((rows, 3), generator=g, device=dev) * 2 - 1
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(f):
        for _ in range(3):
            f(x)
        torch.cuda.synchronize()
        e0.record(net.stream)
        for _ in range(reps):
            f(x)
        e1.record(net.stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(net.forward_fused)
    ms3 = timed(net.forward)
    flops = 2.0 * rows * (3 * 256 + 2 * 256 * 256 + 256)
    peak, src = bf16_peak()
    ach = flops / (ms * 1e-3) / 1e12
    xb = torch.rand((8192, 3), generator=g, device=dev)
    yb = torch.rand(8192, generator=g, device=dev)
    for _ in range(3):
        net.train_step(xb, yb, lr=0.0)
    torch.cuda.synchronize()
    e0.record(net.stream)
    for _ in range(reps):
        net.train_step(xb, yb, lr=0.0)
    e1.record(net.stream)
    torch.cuda.synchronize()
    ms_train = e0.elapsed_time(e1) / reps
    return {"roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "traffic": None,
                         "kernel": "k_mlp_fused (persistent; both hidden layers on tcgen05 "
                                   "kind::f16, BF16 in, FP32 accumulate in TMEM; activations "
                                   "in shared memory)",
                         "ms": ms, "algorithmic_flops": flops, "peak_source": src},
            "rows": rows, "three_launch_ms": ms3, "train_step_ms_8192_rows": ms_train}


def batch_bench(local, steps=3, warmup=2):
    """batch_256: 256 independent slabs (cells 50-800, 16-64 directions per half range,
    64/256/1024 groups) stepped together, FP32 sweeps with pair low-order kernels, V-cycle
    at that form's l_max, converged steps."""
    import torch
    from paper_2011_05427_gb300 import trt
    slabs = W.batch_256()
    upd = [c.n_cells * 2 * c.N * c.G for c in slabs]
    cg = sum(c.n_cells * c.G for c in slabs)
    B = trt.Batch(slabs, precision="sweep32_lopair", device=f"cuda:{local}")
    best = B.autotune(1e-3, reps=4)
    ms = B.sweep_time(1e-3, reps=5)
    byt = sum(upd) * 16 + cg * 16
    lm = tuned_lmax("sweep32_lopair", "V")
    for _ in range(warmup):
        B.step(1e-3, "V", lm, 1e-8)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(B.stream)
    sts = [B.step(1e-3, "V", lm, 1e-8) for _ in range(steps)]
    e1.record(B.stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) * 1e-3
    tot = sum(x["n_ti"] * u for st in sts for x, u in zip(st, upd))
    hbm, src = peaks()
    out = {"workload": "batch_256 (seed 2011054270): 256 slabs, cells U{50..800}, N in "
                       f"{{16,32,64}}, G in {{64,256,1024}}, FP32 sweeps with pair low-order kernels, V-cycle l_max {lm}, "
                       "eps 1e-8",
           "value": tot / t, "unit": "updates/s", "ms_per_step": t / steps * 1e3,
           "updates_per_sweep": sum(upd), "workspace_gb": B.workspace_bytes / 1e9,
           "sweep_tile": {"D": best[1], "shape": best[2]},
           "n_ti_per_slab_step": float(np.mean([x["n_ti"] for st in sts for x in st])),
           "n_c_per_slab_step": float(np.mean([x["n_c"] for st in sts for x in st])),
           "roofline_batched_sweep": {"bound": "hbm", "ms": ms, "achieved": byt / (ms * 1e-3) / 1e9,
                                      "peak": hbm, "unit": "GB/s",
                                      "frac": byt / (ms * 1e-3) / 1e9 / hbm,
                                      "algorithmic_bytes": byt, "peak_source": src}}
    B.close()
    return out


def closure_bench(local, ms_fp64, steps=10, precision="sweep32_lopair"):
    """Learned warm start: trained on snapshots of 4 slabs x 10 steps of the method, then
    fc_1024 stepped in the fastest precision form (FP32 sweeps, pair low-order kernels, at
    its tuned l_max) with and without it."""
    import dataclasses
    from paper_2011_05427_gb300 import closure
    import torch
    t0 = time.perf_counter()
    X, Y = closure.collect(closure.training_slabs(4), 10, 16384, device=f"cuda:{local}")
    net, hist = closure.train(X, Y, iters=1000, batch=8192, lr=1e-3, device=f"cuda:{local}")
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    cfg = dataclasses.replace(W.fc_1024("V"), l_max=tuned_lmax(precision, "V"))
    r = closure.compare(cfg, net, steps, precision=precision, device=f"cuda:{local}")
    a, b = r["plain"], r["closure"]
    dT = float(np.max(np.abs(a["state"]["T"] - b["state"]["T"]) / a["state"]["T"]))
    return {"train_rows": int(len(X)), "train_loss_first_last": [hist[0][1], hist[-1][1]],
            "collect_and_train_s": t_train,
            "precision": precision,
            "plain": {k: a[k] for k in ("n_ti", "n_c", "ms_per_step")},
            "closure": {k: b[k] for k in ("n_ti", "n_c", "ms_per_step")},
            "speedup_closure_vs_plain_fp64": ms_fp64 / b["ms_per_step"],
            "max_rel_T_closure_vs_plain": dT, "steps": steps, "l_max": cfg.l_max}


def closure_config5_run(local=0, n_slabs=20, steps=100, eval_steps=200):
    """The learned closure at the stated size: snapshots of n_slabs x steps = 2000 converged
    steps of batch-family slabs (cells, angles, inflow temperature and opacity scale drawn
    as in batch_256; 1024 groups on the fc_1024 hierarchy; FP32 sweeps), 16384 random rows
    per step, the network trained by its tensor-core kernels (two passes over the rows),
    then fc_1024 stepped eval_steps times with FP32 sweeps at their tuned l_max with and
    without the warm start."""
    import dataclasses
    import torch
    from paper_2011_05427_gb300 import closure
    dev = f"cuda:{local}"
    t0 = time.perf_counter()
    X, Y = closure.collect(closure.training_slabs(n_slabs), steps, 16384, precision="sweep32",
                           device=dev)
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    iters = max(1000, 2 * len(X) // 8192)
    t0 = time.perf_counter()
    net, hist = closure.train(X, Y, iters=iters, batch=8192, lr=1e-3, device=dev)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    cfg = dataclasses.replace(W.fc_1024("V"), l_max=tuned_lmax("sweep32", "V"))
    r = closure.compare(cfg, net, eval_steps, precision="sweep32", device=dev)
    a, b = r["plain"], r["closure"]
    dT = float(np.max(np.abs(a["state"]["T"] - b["state"]["T"]) / a["state"]["T"]))
    return {"training": {"slab_steps": n_slabs * steps, "rows": int(len(X)), "iters": iters,
                         "loss_first_last": [hist[0][1], hist[-1][1]],
                         "collect_s": t_collect, "train_s": t_train},
            "eval_steps": eval_steps, "l_max": cfg.l_max,
            "plain": {k: a[k] for k in ("n_ti", "n_c", "n_lo", "ms_per_step")},
            "closure": {k: b[k] for k in ("n_ti", "n_c", "n_lo", "ms_per_step")},
            "max_rel_T_closure_vs_plain": dT}


def fc4096_bench(local, steps=10):
    """fc_4096 (1000 cells, double S64 = 128 directions, 4096 groups, 7 grids, W-cycle
    l_max 2): FP32 sweeps against the plain FP64 path, step by step from the same start;
    per-step error of the FP32-sweep state against the FP64 state, and the FP32 sweep's
    HBM roofline at this size."""
    import torch
    from paper_2011_05427_gb300 import trt
    cfg = W.fc_4096("W")
    dev = f"cuda:{local}"
    out = {"workload": "fc_4096: 1000 cells, 128 directions (double S64), 4096 groups, grids "
                       "4096/1024/256/64/16/4/1, W-cycle l_max 2, dt 1e-3 sh, eps 1e-8"}
    errs = []
    solvers = {}
    for prec in ("fp64", "sweep32"):
        s = trt.Solver.from_slab(cfg, precision=prec, device=dev)
        s.autotune(cfg.dt, reps=4)
        solvers[prec] = s
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tot = {"fp64": 0.0, "sweep32": 0.0}
    nti = {"fp64": 0, "sweep32": 0}
    for k in range(steps):
        for prec, s in solvers.items():
            torch.cuda.synchronize()
            ev[0].record(s.stream)
            st = s.step(cfg.dt, "W", 2, cfg.eps)
            ev[1].record(s.stream)
            torch.cuda.synchronize()
            tot[prec] += ev[0].elapsed_time(ev[1])
            nti[prec] += st["n_ti"]
        a, b = solvers["fp64"].moments(), solvers["sweep32"].moments()
        errs.append({"step": k + 1,
                     "max_rel_T": float(np.max(np.abs(b["T"] - a["T"]) / a["T"])),
                     "max_rel_Eg": float(np.max(np.abs(b["Eg"] - a["Eg"]) /
                                                a["Eg"].sum(0)[None, :]))})
    roof = sweep_roofline(trt, solvers["sweep32"], cfg, fp32=True, reps=10)["roofline"]
    for s in solvers.values():
        s.close()
    upd = cfg.updates_per_sweep()
    out.update({"ms_per_step_fp64": tot["fp64"] / steps,
                "ms_per_step_sweep32": tot["sweep32"] / steps,
                "n_ti_per_step_fp64": nti["fp64"] / steps,
                "n_ti_per_step_sweep32": nti["sweep32"] / steps,
                "value_sweep32": nti["sweep32"] * upd / (tot["sweep32"] * 1e-3),
                "error_sweep32_vs_fp64_per_step": errs,
                "max_rel_T_over_steps": max(e["max_rel_T"] for e in errs),
                "max_rel_Eg_over_steps": max(e["max_rel_Eg"] for e in errs),
                "roofline_sweep_fp32": roof})
    return out


def mixed_vs_oracle(local, precision):
    """One fixed-iteration fc_1024 step (s = 0 phase, one sweep, one more phase; one V cycle
    each) of the GPU path in `precision` against the FP64 oracle (on all host cores):
    T, the energy-weighted E_g, and the pure relative E_g on groups holding more than 1e-20
    of their cell's energy."""
    from oracle import orc
    from paper_2011_05427_gb300 import trt
    cfg = W.fc_1024("V")
    orc.set_threads(os.cpu_count() or 1)
    s = trt.Solver.from_slab(cfg, precision=precision, device=f"cuda:{local}")
    o = orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                    cfg.T_left, cfg.T_right)
    s.step(cfg.dt, "V", 1, -1.0, max_outer=2)
    o.step(cfg.dt, "V", 1, -1.0, max_outer=2)
    orc.set_threads(1)
    g, r = s.moments(), o.state()
    s.close()
    Ec = r["Eg"].sum(0)[None, :]
    sel = r["Eg"] > 1e-20 * Ec
    return {"max_rel_T_vs_oracle": float(np.max(np.abs(g["T"] - r["T"]) / r["T"])),
            "max_rel_Eg_vs_oracle": float(np.max(np.abs(g["Eg"] - r["Eg"]) / Ec)),
            "max_pure_rel_Eg_vs_oracle": float(np.max(np.abs(g["Eg"] - r["Eg"])[sel] /
                                                      r["Eg"][sel])),
            "sample": "one fixed-iteration fc_1024 step from the cold start (s=0 phase, one "
                      "sweep, one phase; one V cycle each), GPU against the FP64 oracle"}


PAPER_TABLES = os.path.join(ROOT, "tests", "golden", "paper_tables.txt")


def cycle_schedule(cycle, Gamma):
    """The coarse grids a cycle visits, in order (Sec. 4, Fig. 1): V the two-grid cycle
    (none), W S = w(2) with w(Gamma) = [] and w(g) = w(g + 1) + [g] + w(g + 1), F the
    grids Gamma - 1 down to 2."""
    if cycle == "V":
        return []
    if cycle == "F":
        return list(range(Gamma - 1, 1, -1))
    if cycle == "W":
        def w(g):
            return [] if g >= Gamma else w(g + 1) + [g] + w(g + 1)
        return w(2)
    raise ValueError(cycle)


def lo_solves_per_cycle(grids, cycle):
    """Group-wise low-order solves of one cycle: the fine grid's groups, each visited coarse
    grid's groups and one grey solve per visit (the tables' N_lo / N_c)."""
    S = cycle_schedule(cycle, len(grids))
    return grids[0] + sum(grids[g - 1] for g in S) + len(S) + 1


def paper_tables_run(local=0):
    """Sec. 6's Fleck-Cummings test (4 cm, 10 cells, 256 groups up to 1e7 keV, double S8,
    T0 = 1 eV, 1 keV inflow, eps = 1e-6, eps_inner = 1e-7) on every grid hierarchy of Tables
    1-2 (0.02 ns x 150 steps and 0.04 ns x 75 steps), plain FP64: the counters N_ti, N_c,
    N_lo summed over the run next to the tables' (the stored rows are the paper's, cited in
    the file), and whether the per-cycle count N_lo / N_c equals n^1 + sum_S n^gamma +
    (|S| + 1) of the cycle's schedule S, as in the tables.  Context: the counts depend on
    the readings of the paper's unspecified details."""
    import dataclasses
    import torch
    from paper_2011_05427_gb300 import trt
    out = []
    for line in open(PAPER_TABLES):
        if line.startswith("#") or not line.strip():
            continue
        t, dt_ns, steps, printed, Gam, grids, lmax, nti, nc, nlo, cyc = line.split()
        grids = [int(g) for g in grids.split(",")]
        def run(cycle):
            cfg = dataclasses.replace(W.fc_paper(float(dt_ns)), levels=grids, cycle=cycle,
                                      l_max=int(lmax))
            assert cfg.steps == int(steps)
            s = trt.Solver.from_slab(cfg, precision="fp64", device=f"cuda:{local}")
            tot = {"N_ti": 0, "N_c": 0, "N_lo": 0}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(cfg.steps):
                st = s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps)
                tot["N_ti"] += st["n_ti"]
                tot["N_c"] += st["n_c"]
                tot["N_lo"] += st["n_lo"]
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            s.close()
            return tot, sec
        tot, sec = run(cyc)
        per = lo_solves_per_cycle(grids, cyc)
        row = {"table": int(t), "dt_ns": float(dt_ns), "Gamma": int(Gam), "grids": grids,
               "cycle_printed": printed, "cycle": cyc, "l_max": int(lmax),
               "ours": tot, "paper": {"N_ti": int(nti), "N_c": int(nc), "N_lo": int(nlo)},
               "N_lo_per_cycle_is_schedule": tot["N_lo"] == per * tot["N_c"], "run_s": sec}
        if printed != cyc:   # the printed cycle too, where the counters decode to another
            row["ours_printed_cycle"] = run(printed)[0]
        out.append(row)
    return out


def adaptive_cycle_run(local=0):
    """Fixed V (l_max 3), W and F (l_max 1) cycles against the per-step controller
    (`cycles.CycleController`, candidates V/3, V/2, V/4, F/1, W/1) on Sec. 6's test with the
    7-grid hierarchy of Table 1 (150 steps of 0.02 ns, eps 1e-6) and on fc_1024 (20 steps of
    1e-3 sh, eps 1e-8), plain FP64: wall time of the whole run (host clock around the steps,
    synchronised), counters, and the controller's picks."""
    import dataclasses
    import torch
    from paper_2011_05427_gb300 import trt
    from paper_2011_05427_gb300.cycles import CycleController
    cases = [("fc_paper_gamma7", dataclasses.replace(W.fc_paper(0.02),
                                                     levels=[256, 128, 32, 16, 8, 4, 1]), 150),
             ("fc_1024", W.fc_1024("V"), 20)]
    cands = (("V", 3), ("V", 2), ("V", 4), ("F", 1), ("W", 1))
    fixed = {"V": 3, "W": 1, "F": 1}
    out = []
    for name, cfg, steps in cases:
        res = {"workload": name, "steps": steps}
        for mode in ("V", "W", "F", "adaptive"):
            s = trt.Solver.from_slab(cfg, precision="fp64", device=f"cuda:{local}")
            ctl = CycleController(cands) if mode == "adaptive" else None
            tot = {"N_ti": 0, "N_c": 0, "N_lo": 0}
            picks = {}
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(steps):
                if ctl:
                    st = ctl.step(s, cfg.dt, cfg.eps)
                    key = f"{st['cycle']}{st['l_max']}"
                    picks[key] = picks.get(key, 0) + 1
                else:
                    st = s.step(cfg.dt, mode, fixed[mode], cfg.eps)
                tot["N_ti"] += st["n_ti"]
                tot["N_c"] += st["n_c"]
                tot["N_lo"] += st["n_lo"]
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            s.close()
            res[mode] = dict(tot, s=sec, **({"picks": picks} if ctl else {}))
        out.append(res)
    return out


def lmax_sweep_run(local=0, steps=10, warmup=3):
    """ms per converged fc_1024 step, sweeps and cycles for each form (FP64, FP32 sweeps),
    cycle and l_max: the measurement behind tuned_lmax.  Each run's final state is compared
    with the FP64 V-cycle l_max 4 state after the same steps."""
    from paper_2011_05427_gb300 import trt
    cfg = W.fc_1024("V")
    cands = [("V", 1), ("V", 2), ("V", 3), ("V", 4), ("W", 1), ("W", 2), ("F", 1), ("F", 2)]
    out, states = [], []
    for prec in ("fp64", "sweep32"):
        for cyc, lm in cands:
            t, st, _, s = timed_steps(trt, cfg, prec, cyc, steps, warmup, local, 1, l_max=lm)
            states.append(s.moments()["T"])
            s.close()
            out.append({"precision": prec, "cycle": cyc, "l_max": lm,
                        "ms": t / steps * 1e3, **counters(st, steps)})
    ref = states[cands.index(("V", 4))]
    for r, T in zip(out, states):
        r["max_rel_T_vs_fp64_V4"] = float(np.max(np.abs(T - ref) / ref))
    return out


def counters(stats, steps):
    return {k: sum(x[k] for x in stats) / steps for k in ("n_ti", "n_c", "n_lo")}


def run_ours(args):
    import torch
    from paper_2011_05427_gb300 import trt
    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    cfg = W.fc_1024(args.cycle)
    upd_sweep = cfg.updates_per_sweep()

    lm = tuned_lmax(args.precision, args.cycle)
    t_max, stats, clocks, s = timed_steps(trt, cfg, args.precision, args.cycle, args.steps,
                                          args.warmup, local, ws, clocks=(rank == 0), l_max=lm)
    n_ti = sum(x["n_ti"] for x in stats)
    launches = sum(x.get("n_kernels", 0) for x in stats)
    value = sum_over_ranks(n_ti * upd_sweep, ws) / t_max
    ms_step = t_max / args.steps * 1e3

    # e2e: the public API from host data -- create (uploads the host-built constants and
    # initial state), K steps each followed by a read of the step's result to host memory:
    # the temperature and the grey energy and flux (the group fields stay on the device)
    res_bytes = 8 * (cfg.n_cells + cfg.n_cells + cfg.n_cells + 1)
    torch.cuda.synchronize()
    barrier(ws)
    te = time.perf_counter()
    s2 = trt.Solver.from_slab(cfg, precision=args.precision, device=f"cuda:{local}")
    e2e_ti = 0
    for _ in range(args.steps):
        st = s2.step(cfg.dt, args.cycle, lm, cfg.eps)
        e2e_ti += st["n_ti"]
        s2.moments(groups=False)
    torch.cuda.synchronize()
    barrier(ws)
    te = max_over_ranks(time.perf_counter() - te, ws)
    h2d = 8 * (cfg.n_cells + 2 * (cfg.G + 1) + cfg.G * cfg.n_cells * 2 + cfg.G * (cfg.n_cells + 1)
               + 10 * cfg.G + 2 * cfg.M) + cfg.G * 8
    s2.close()
    e2e_val = sum_over_ranks(e2e_ti * upd_sweep, ws) / te

    # the other cycle and the mixed-precision form on the same workload, same step count
    extra = {}
    if args.compare:
        for other in [c for c in ("V", "W", "F") if c != args.cycle]:
            lo = tuned_lmax(args.precision, other)
            t_o, st_o, _, s_o = timed_steps(trt, cfg, args.precision, other, args.steps, 1,
                                            local, ws, l_max=lo)
            s_o.close()
            extra[f"cycle_{other}"] = {"ms_per_step": t_o / args.steps * 1e3, "l_max": lo,
                                       "value": sum(x["n_ti"] for x in st_o) * upd_sweep / t_o,
                                       **counters(st_o, args.steps)}
        if args.precision == "fp64":
            lm32 = tuned_lmax("sweep32", args.cycle)
            t_m, st_m, _, s_m = timed_steps(trt, cfg, "sweep32", args.cycle, args.steps,
                                            args.warmup, local, ws, l_max=lm32)
            a, b = s.moments(), s_m.moments()
            s_m.close()
            # the same form at the FP64 form's l_max: the speed-up at equal iteration settings
            t_e, st_e, _, s_e = timed_steps(trt, cfg, "sweep32", args.cycle, args.steps,
                                            args.warmup, local, ws, l_max=lm)
            s_e.close()
            extra["mixed_sweep32"] = {
                "ms_per_step": t_m / args.steps * 1e3,
                "l_max": lm32,
                "value": sum(x["n_ti"] for x in st_m) * upd_sweep / t_m,
                "speedup_vs_fp64": ms_step / (t_m / args.steps * 1e3),
                "max_rel_T_vs_fp64": float(np.max(np.abs(b["T"] - a["T"]) / a["T"])),
                "max_rel_Eg_vs_fp64": float(np.max(np.abs(b["Eg"] - a["Eg"]) /
                                                   a["Eg"].sum(0)[None, :])),
                "at_fp64_l_max": {"l_max": lm, "ms_per_step": t_e / args.steps * 1e3,
                                  "speedup_vs_fp64": ms_step / (t_e / args.steps * 1e3),
                                  **counters(st_e, args.steps)},
                "note": "FP32 sweeps, FP64 group/grey LOQD + MEB; each form at its own tuned "
                        "l_max, both converged to eps; compared after the same warm-up + "
                        "timed steps",
                **counters(st_m, args.steps)}
            if ws == 1 and args.cpu_baseline:
                extra["mixed_sweep32"]["vs_oracle"] = mixed_vs_oracle(local, "sweep32")
            t_x, st_x, _, s_x = timed_steps(trt, cfg, "mixed", args.cycle, args.steps,
                                            args.warmup, local, ws, l_max=lm32)
            c = s_x.moments()
            s_x.close()
            extra["mixed"] = {
                "ms_per_step": t_x / args.steps * 1e3,
                "value": sum(x["n_ti"] for x in st_x) * upd_sweep / t_x,
                "speedup_vs_fp64": ms_step / (t_x / args.steps * 1e3),
                "max_rel_T_vs_fp64": float(np.max(np.abs(c["T"] - a["T"]) / a["T"])),
                "max_rel_Eg_vs_fp64": float(np.max(np.abs(c["Eg"] - a["Eg"]) /
                                                   a["Eg"].sum(0)[None, :])),
                "l_max": lm32,
                "note": "FP32 sweeps and FP32 group LOQD eliminations refined by two "
                        "FP64-residual steps, FP64 grey LOQD + MEB",
                **counters(st_x, args.steps)}
            # FP32 sweeps with the group LOQD solves and opacities in FP32-pair arithmetic
            t_p, st_p, _, s_p = timed_steps(trt, cfg, "sweep32_lopair", args.cycle, args.steps,
                                            args.warmup, local, ws, l_max=lm32)
            d = s_p.moments()
            s_p.close()
            extra["mixed_sweep32_lopair"] = {
                "ms_per_step": t_p / args.steps * 1e3,
                "value": sum(x["n_ti"] for x in st_p) * upd_sweep / t_p,
                "speedup_vs_fp64": ms_step / (t_p / args.steps * 1e3),
                "max_rel_T_vs_fp64": float(np.max(np.abs(d["T"] - a["T"]) / a["T"])),
                "max_rel_Eg_vs_fp64": float(np.max(np.abs(d["Eg"] - a["Eg"]) /
                                                   a["Eg"].sum(0)[None, :])),
                "l_max": lm32,
                "note": "FP32 sweeps; group LOQD solves and opacities in FP32-pair arithmetic "
                        "(FP64 in and out); restriction, grey LOQD + MEB in FP64",
                **counters(st_p, args.steps)}
            if ws == 1 and args.cpu_baseline:
                extra["mixed_sweep32_lopair"]["vs_oracle"] = mixed_vs_oracle(local,
                                                                             "sweep32_lopair")

        if args.mlp:
            extra["mlp"] = mlp_bench(local)
        if args.closure and args.precision == "fp64":
            extra["closure"] = closure_bench(local, ms_step)
        if args.batch and ws == 1:
            extra["batch_256"] = batch_bench(local)
        if args.large and ws == 1:
            extra["fc_4096"] = fc4096_bench(local)

    tile = s.tile
    if args.precision in ("fp64", "lo32"):
        roof = sweep_roofline(trt, s, cfg, fp32=False)
        roof["roofline"]["tile"] = {"D": tile[0], "S": tile[1], "NS": tile[2]}
        roof32 = sweep_roofline(trt, None, cfg, fp32=True, local=local)
    else:
        roof32 = sweep_roofline(trt, s, cfg, fp32=True)
        roof32["roofline"]["tile"] = {"D": tile[0], "S": tile[1], "NS": tile[2]}
        roof = sweep_roofline(trt, None, cfg, fp32=False, local=local)
    if rank != 0:
        s.close()
        return
    main_roof = roof32 if args.precision != "fp64" and args.precision != "lo32" else roof
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
        "dtype": "f64" if args.precision in ("fp64", "lo32") else "f32+f64",
        "data": "synthetic (Fleck-Cummings slab, seeded, no dataset)",
        "config": {"workload": f"fc_1024: 500 cells, 64 directions (double S32), 1024 groups, "
                               f"grids 1024/256/64/16/1, {args.cycle}-cycle "
                               f"l_max {lm}, dt 1e-3 sh, eps 1e-8, {args.precision}",
                   "l_max": lm,
                   "parallelism": f"replicas x{ws}",
                   "sweep_tile": {"D": tile[0], "S": tile[1], "NS": tile[2],
                                  "picked_by": "trt_autotune"},
                   "l2": "inputs larger than L2 (intensity arrays 1 GB each in FP64)",
                   **{k + "_per_step": v for k, v in counters(stats, args.steps).items()}},
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": h2d / args.steps,
                "d2h_bytes_per_step": res_bytes,
                "note": "create + K steps from the initial state, each followed by a read of "
                        "T and the grey E, F; the state stays on the device"},
        "gpu_launches": launches,
        "roofline": main_roof["roofline"],
        "roofline_sweep_fp32": roof32["roofline"],
        "roofline_sweep_fp64": roof["roofline"],
        "clocks": clocks,
        **extra,
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


def cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo), or None."""
    import subprocess
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def oracle_config1_ms(orc, steps=10):
    """ms per converged step of the oracle on the 60-cell, 17-group Fleck-Cummings slab
    (two-grid cycles, eps 1e-8), over `steps` steps from the cold start."""
    cfg = W.fc_small()
    p = orc.Problem(cfg.h(), cfg.N, cfg.edges(), cfg.levels, cfg.opac_scale, cfg.cv, cfg.T0,
                    cfg.T_left, cfg.T_right)
    t = time.perf_counter()
    for _ in range(steps):
        p.step(cfg.dt, "V", cfg.l_max, cfg.eps)
    return (time.perf_counter() - t) / steps * 1e3


def cpu_baseline(args):
    """The oracle on the host cores: fc_1024 fixed-iteration samples (updates/s) on one
    thread and on all cores (its group-parallel loops under OpenMP), and ms per converged
    step of the 60-cell slab on both."""
    from oracle import orc
    cfg = W.fc_1024(args.cycle)
    nproc = os.cpu_count() or 1
    res = {}
    for threads in (1, nproc):
        orc.set_threads(threads)
        upd = dt = 0.0
        for _ in range(3 if threads == 1 else 6):
            u, t = oracle_sample(orc, cfg)
            upd += u
            dt += t
        res[threads] = (upd / dt, dt, oracle_config1_ms(orc))
    orc.set_threads(1)
    v1, t1, c1 = res[1]
    vn, tn, cn = res[nproc]
    return {"value": vn, "unit": "updates/s", "cores": nproc, "kind": "oracle",
            "sample": f"oracle (FP64 C, OpenMP over groups, {nproc} threads): six fixed-"
                      "iteration steps of fc_1024 from the cold start (each: s=0 phase + 1 "
                      f"sweep + 1 phase, 1 cycle each), {tn:.1f} s; updates counted over the "
                      "sweeps",
            "cpu_model": cpu_model(), "nproc": nproc,
            "single_thread": {"value": v1, "unit": "updates/s", "cores": 1,
                              "sample": f"three of the same steps, {t1:.1f} s"},
            "ms_per_step_config1": {"1_thread": c1, f"{nproc}_threads": cn,
                                    "workload": "fc_small: 60 cells, double S8, 17 groups, "
                                                "two-grid, eps 1e-8, 10 converged steps"}}


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import orc
    cfg = W.fc_1024(args.cycle)
    nproc = os.cpu_count() or 1
    orc.set_threads(nproc)
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
                                  "+ 1 sweep + 1 phase)",
                      "parallelism": f"{nproc} host threads (OpenMP over groups)"},
           "cpu_baseline": {"kind": "oracle", "cores": nproc, "value": v, "unit": "updates/s",
                            "cpu_model": cpu_model(),
                            "sample": "each step: one fixed-iteration step of fc_1024"},
           "e2e": {"value": v, "unit": "updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def launch_table(path):
    """Per-kernel summary of an ncu launch list (`--metrics gpu__time_duration.sum --csv`):
    launches, total device time, share and mean per launch, as a markdown table."""
    import collections
    import csv
    scale = {"ns": 1e-3, "nsecond": 1e-3, "us": 1.0, "usecond": 1.0, "ms": 1e3, "msecond": 1e3}
    with open(path) as fh:
        rows = list(csv.reader(fh))
    hi = next(i for i, r in enumerate(rows) if r and r[0] == "ID")
    hdr, data = rows[hi], rows[hi + 1:]
    ki, mi = hdr.index("Kernel Name"), hdr.index("Metric Name")
    vi, ui = hdr.index("Metric Value"), hdr.index("Metric Unit")
    tot, cnt = collections.defaultdict(float), collections.Counter()
    for r in data:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        us = float(r[vi].replace(",", "")) * scale[r[ui]]
        name = r[ki].split("(")[0].replace("void ", "")
        tot[name] += us
        cnt[name] += 1
    T = sum(tot.values())
    out = ["| kernel | launches | total ms | share | mean us |", "|---|---|---|---|---|"]
    for k, v in sorted(tot.items(), key=lambda x: -x[1]):
        out.append(f"| `{k}` | {cnt[k]} | {v / 1e3:.2f} | {100 * v / T:.1f}% | {v / cnt[k]:.1f} |")
    out.append(f"| total | {sum(cnt.values())} | {T / 1e3:.2f} | 100% | |")
    return "\n".join(out)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64",
                    choices=["fp64", "mixed", "sweep32", "lo32", "lopair", "sweep32_lopair"])
    ap.add_argument("--cycle", default="V", choices=["V", "W", "F"])
    ap.add_argument("--no-compare", dest="compare", action="store_false",
                    help="skip the comparison runs (other cycle, FP32 sweeps, MLP, closure, "
                         "batch)")
    ap.add_argument("--no-mlp", dest="mlp", action="store_false")
    ap.add_argument("--no-closure", dest="closure", action="store_false")
    ap.add_argument("--no-batch", dest="batch", action="store_false")
    ap.add_argument("--no-large", dest="large", action="store_false",
                    help="skip the 4096-group comparison (fc_4096)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--profile-step", action="store_true",
                    help="run the warm-up steps and one more step, print nothing (for ncu)")
    ap.add_argument("--profile-mlp", action="store_true",
                    help="run the fused MLP inference over 512,000 rows 3 times (for ncu)")
    ap.add_argument("--profile-sweep", default="", metavar="NX,N,G,D,SHAPE",
                    help="one FP32-sweep step of a Fleck-Cummings slab of NX cells, 2N "
                         "directions, G groups with sweep tile (D, SHAPE) (for ncu)")
    ap.add_argument("--profile-batch", type=int, default=0, metavar="N",
                    help="step the first N slabs of batch_256 (FP32 sweeps, V-cycle): tile "
                         "(8, 4), one warm-up step and one step (for ncu launch lists)")
    ap.add_argument("--paper-tables", action="store_true",
                    help="run Sec. 6's test on the 12 grid hierarchies of Tables 1-2 and print "
                         "the counters next to the paper's (one JSON line)")
    ap.add_argument("--adaptive-cycle", action="store_true",
                    help="fixed V/W/F cycles against the per-step cycle controller (one JSON "
                         "line)")
    ap.add_argument("--closure-config5", action="store_true",
                    help="the learned closure trained on 2000 batch-family steps and evaluated "
                         "over 200 fc_1024 steps (one JSON line)")
    ap.add_argument("--lmax-sweep", action="store_true",
                    help="ms per converged fc_1024 step for each form, cycle and l_max (one "
                         "JSON line)")
    ap.add_argument("--tile", default=None,
                    help="D,shape: sweep tile for --profile-step (default: the library's)")
    ap.add_argument("--launch-table", default="", metavar="CSV",
                    help="print the per-kernel table of an ncu launch list and exit")
    args = ap.parse_args()
    if args.launch_table:
        print(launch_table(args.launch_table))
        return
    if args.adaptive_cycle:
        print(json.dumps({"adaptive_cycle": adaptive_cycle_run()}))
        return
    if args.paper_tables:
        print(json.dumps({"paper_tables": paper_tables_run()}))
        return
    if args.lmax_sweep:
        print(json.dumps({"lmax_sweep": lmax_sweep_run()}))
        return
    if args.closure_config5:
        print(json.dumps({"closure_config5": closure_config5_run()}))
        return
    if args.profile_sweep:
        from paper_2011_05427_gb300 import trt
        nx, n, g, d, sh = (int(v) for v in args.profile_sweep.split(","))
        cfg = W.scaled(W.fc_4096(), nx, n, g, levels=[g, 1])
        s = trt.Solver.from_slab(cfg, precision="sweep32", device="cuda:0")
        s.set_sweep_tile(d, sh)
        s.step(cfg.dt, "V", 1, -1.0, max_outer=2)
        s.close()
        return
    if args.profile_batch:
        from paper_2011_05427_gb300 import trt
        B = trt.Batch(W.batch_256(args.profile_batch), precision="sweep32", device="cuda:0")
        B.set_tile(8, 4)
        for _ in range(2):
            B.step(1e-3, "V", 4, 1e-8)
        B.close()
        return
    if args.profile_mlp:
        import torch
        from paper_2011_05427_gb300 import closure, mlp
        net = mlp.MLP(closure._init(7), device="cuda:0")
        g = torch.Generator(device="cuda:0")
        g.manual_seed(3)
        x = torch.rand((512000, 3), generator=g, device="cuda:0") * 2 - 1
        for _ in range(3):
            net.forward_fused(x)
        torch.cuda.synchronize()
        return
    if args.profile_step:
        from paper_2011_05427_gb300 import trt
        cfg = W.fc_1024(args.cycle)
        s = trt.Solver.from_slab(cfg, precision=args.precision, device="cuda:0")
        if args.tile:
            s.set_sweep_tile(*[int(x) for x in args.tile.split(",")])
        for _ in range(args.warmup + 1):
            s.step(cfg.dt, cfg.cycle, tuned_lmax(args.precision, args.cycle), cfg.eps)
        s.close()
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
