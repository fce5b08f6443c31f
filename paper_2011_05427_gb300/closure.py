"""Learned closure: snapshots the method itself generates, training of the MLP on them, and
the A/B comparison of warm-started steps against the plain method.

A snapshot row is one (group g, cell i) of a time step j: the features of the step's
initial state (T_i^{j-1}, sigma_E,g(T_i^{j-1}), E_g,i^{j-1} / E_i^{j-1}) and the target
f_g,i^j, the QD factor of the step's last sweep.  Features are computed by the library's
kernel (trt_mlp_features), the network is trained by its tensor-core kernels
(trt_mlp_grad, trt_mlp_adam); this module only schedules the calls and moves buffers."""
import ctypes

import numpy as np

from . import mlp as _mlp
from . import trt
from . import workloads as W


def _features(s, T_dev):
    """Features of solver s's current state, rows g-major [G*nx][3] (device FP32)."""
    t = s.torch
    sig, _, _ = s.k_opacity(T_dev)
    m = s.moments()
    Eg = t.as_tensor(m["Eg"], dtype=t.float64, device=s.device).contiguous()
    E = t.as_tensor(m["Eg"].sum(0), dtype=t.float64, device=s.device).contiguous()
    x = t.empty((s.G * s.nx, 3), dtype=t.float32, device=s.device)
    rc = trt.lib().trt_mlp_features(s.nx, s.G, T_dev.data_ptr(), sig.data_ptr(), Eg.data_ptr(),
                                    E.data_ptr(), x.data_ptr(),
                                    ctypes.c_void_p(s.stream.cuda_stream))
    if rc != 0:
        raise trt.TRTError(rc, "trt_mlp_features")
    return x


def collect(slabs, steps, rows_per_step, seed=0, precision="fp64", device="cuda:0"):
    """Run each slab for `steps` converged steps; keep `rows_per_step` random rows of every
    step.  Returns (X [n][3], Y [n]) as numpy float32."""
    import torch
    r = np.random.default_rng(seed)
    xs, ys = [], []
    for cfg in slabs:
        s = trt.Solver.from_slab(cfg, precision=precision, device=device)
        for _ in range(steps):
            T = torch.as_tensor(s.moments()["T"], dtype=torch.float64, device=s.device)
            x = _features(s, T).cpu().numpy()
            s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps)
            f = s.qd_factors().reshape(-1)
            idx = r.choice(f.size, min(rows_per_step, f.size), replace=False)
            xs.append(x[idx])
            ys.append(f[idx].astype(np.float32))
        s.close()
    return np.concatenate(xs), np.concatenate(ys)


def _init(seed):
    """He-uniform weights, zero biases, small output layer (same recipe as the oracle's
    init, written here so that the product path does not import the oracle)."""
    r = np.random.default_rng(seed)
    p = np.zeros(_mlp.NPARAM, np.float32)
    p[0:768] = r.uniform(-1, 1, 768) * np.sqrt(6.0 / 3)
    p[1024:1024 + 65536] = r.uniform(-1, 1, 65536) * np.sqrt(6.0 / 256)
    p[66816:66816 + 65536] = r.uniform(-1, 1, 65536) * np.sqrt(6.0 / 256)
    p[132608:132608 + 256] = r.uniform(-1, 1, 256) * np.sqrt(1.0 / 256)
    return p


def train(X, Y, iters=2000, batch=8192, lr=1e-3, seed=1, device="cuda:0", net=None):
    """Adam on shuffled contiguous minibatches (batch a multiple of 128).  Returns the
    network and the loss history (read back every 100 steps)."""
    import torch
    assert batch % 128 == 0
    r = np.random.default_rng(seed)
    n = (len(X) // batch) * batch
    perm = r.permutation(len(X))[:n]
    Xd = torch.as_tensor(X[perm], dtype=torch.float32, device=device)
    Yd = torch.as_tensor(Y[perm], dtype=torch.float32, device=device)
    net = net or _mlp.MLP(_init(seed), device=device)
    hist = []
    nb = n // batch
    for it in range(iters):
        b = it % nb
        loss = net.train_step(Xd[b * batch:(b + 1) * batch], Yd[b * batch:(b + 1) * batch], lr=lr)
        if it % 100 == 0 or it == iters - 1:
            hist.append((it, float(loss.item())))
    return net, hist


def compare(cfg, net, steps, precision="fp64", device="cuda:0"):
    """The same slab stepped with and without the learned warm start.  Returns per-variant
    counters, device time per step and the final states."""
    import torch
    out = {}
    for name, use in (("plain", False), ("closure", True)):
        s = trt.Solver.from_slab(cfg, precision=precision, device=device)
        if use:
            s.set_closure(net)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(s.stream)
        st = [s.step(cfg.dt, cfg.cycle, cfg.l_max, cfg.eps) for _ in range(steps)]
        ev1.record(s.stream)
        torch.cuda.synchronize()
        out[name] = dict(n_ti=sum(x["n_ti"] for x in st), n_c=sum(x["n_c"] for x in st),
                         n_lo=sum(x["n_lo"] for x in st),
                         ms_per_step=ev0.elapsed_time(ev1) / steps, state=s.moments())
        s.close()
    return out


def training_slabs(n, seed=W.BATCH_SEED + 1, G=1024):
    """Slabs of the batched family (cells, angles, inflow temperature, opacity scale drawn
    as in batch_256) with G groups on the fc_1024 hierarchy."""
    out = []
    for k, cfg in enumerate(W.batch_256(n, seed)):
        levels = [1024, 256, 64, 16, 1] if G == 1024 else W.uniform_levels(G, 4)
        c = W.scaled(cfg, cfg.n_cells, cfg.N, G, levels=levels, name=f"train{k}")
        c.cycle, c.l_max = "V", 4
        out.append(c)
    return out
