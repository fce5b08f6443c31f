"""The allocation-free sweep (trt_sweep_noalloc) against the workspace-backed sweep
(trt_k_sweep), both called through the C ABI.

trt_sweep_noalloc serves callers that cannot allocate device memory (a plug-in whose host
application owns all device allocations, or a running time loop that must not call
cudaMalloc); its scratch is a static device array shared by every call.  This file is
named to be collected last so that a run that stops at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

from paper_2011_05427_gb300 import workloads as W

C = 299.792458

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_05427_gb300 import build, trt
    build.build()
    return torch, trt


def pair_err(a, b):
    scale = np.maximum(np.abs(b[:, :, 0:1, :]), np.abs(b[:, :, 1:2, :]))
    return np.max(np.abs(a - b) / scale)


@pytest.mark.parametrize("precision", ["fp64", "sweep32"])
def test_noalloc_sweep_matches_workspace_sweep(env, orc, precision):
    """Two calls in a row through the shared static scratch give the workspace sweep's
    results (same kernels and default tile: FP64 to round-off; FP32 sweeps on the same
    pre-scaled FP32 inputs, bit for bit) and the oracle's sweep to the kernel tolerance."""
    torch, trt = env
    cfg = W.fc_small()
    nx, N, G = cfg.n_cells, cfg.N, cfg.G
    M, ldG = 2 * N, (G + 31) // 32 * 32
    dev = torch.device("cuda", 0)
    s = trt.Solver.from_slab(cfg, precision=precision, device=dev)
    fp32 = precision == "sweep32"
    code = trt.TRT_SWEEP_FP32 if fp32 else trt.TRT_FP64
    L = trt.lib()
    assert L.trt_sweep_noalloc_scratch_bytes(nx, N, G) <= 8 << 20

    mu, w = orc.double_gl(N)
    Iin0 = orc.group_physics(cfg.edges(), cfg.T_left)[0]
    IinX = np.zeros(G)
    d = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
    h_d, mu_d, w_d, i0_d, iX_d = d(cfg.h()), d(mu), d(w), d(Iin0), d(IinX)
    rdt = torch.float32 if fp32 else torch.float64
    tol_ref, tol_orc = (0.0, 2e-5) if fp32 else (1e-12, 1e-11)

    r = W.rng(606)
    for call in range(2):   # two calls in a row through the shared static scratch
        T = W.random_temperatures(r, nx, 1e-3, 1.2)
        sig, em, _ = s.k_opacity(T)
        I_old = W.random_intensity(r, M, nx, G)
        if fp32:   # the FP32 intensities both paths read
            I_old = I_old.astype(np.float32).astype(np.float64)
        ref = [t.cpu().numpy() for t in s.k_sweep(cfg.dt, sig, em, I_old)]
        oI, of, ofb0, ofbX, oC0, oCX = orc.sweep(cfg.h(), mu, w, sig.cpu().numpy(),
                                                 em.cpu().numpy(), 1.0 / (C * cfg.dt), I_old,
                                                 Iin0, IinX)

        Ip = torch.zeros((M, nx, 2, ldG), dtype=rdt, device=dev)
        Ip[..., :G] = torch.as_tensor(I_old, dtype=rdt, device=dev)
        In = torch.empty_like(Ip)
        f = torch.empty((G, nx), dtype=torch.float64, device=dev)
        b = [torch.empty(G, dtype=torch.float64, device=dev) for _ in range(4)]
        stream = torch.cuda.current_stream(dev)
        rc = L.trt_sweep_noalloc(nx, N, G, code, float(cfg.dt), h_d.data_ptr(),
                                 mu_d.data_ptr(), w_d.data_ptr(), i0_d.data_ptr(),
                                 iX_d.data_ptr(), sig.data_ptr(), em.data_ptr(), Ip.data_ptr(),
                                 In.data_ptr(), f.data_ptr(), *[t.data_ptr() for t in b],
                                 ctypes.c_void_p(stream.cuda_stream))
        assert rc == trt.TRT_OK, L.trt_sweep_noalloc_error()
        torch.cuda.synchronize(dev)
        got = [In[..., :G].double().cpu().numpy(), f.cpu().numpy()] + [t.cpu().numpy() for t in b]
        assert pair_err(got[0], ref[0]) <= tol_ref, call
        for a_, b_ in zip(got[1:], ref[1:]):
            assert np.max(np.abs(a_ - b_) / np.abs(b_)) <= max(tol_ref, 1e-12), call
        assert pair_err(got[0], oI) < tol_orc, call
        for a_, b_ in zip(got[1:], (of, ofb0, ofbX, oC0, oCX)):
            assert np.max(np.abs(a_ - b_) / np.abs(b_)) < tol_orc, call
    s.close()


def test_noalloc_rejects_oversize(env):
    torch, trt = env
    L = trt.lib()
    cfg = W.fc_1024()
    need = L.trt_sweep_noalloc_scratch_bytes(cfg.n_cells, cfg.N, cfg.G)
    assert need > 8 << 20
    buf = torch.zeros(1, dtype=torch.float64, device="cuda:0")   # the size check comes first
    p = ctypes.c_void_p(buf.data_ptr())
    rc = L.trt_sweep_noalloc(cfg.n_cells, cfg.N, cfg.G, trt.TRT_FP64, 1e-3, *([p] * 14), None)
    assert rc == trt.TRT_ENOSPACE
    assert b"static array" in L.trt_sweep_noalloc_error()
