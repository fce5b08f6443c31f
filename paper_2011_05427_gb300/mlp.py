"""Thin binding of the learned closure (include/trt_mlp.h): device buffers for the MLP's
parameters, their BF16 copies and the Adam moments, and calls into libtrt.so.  Every
arithmetic step runs in the library's kernels; this module only allocates torch tensors
and passes pointers."""
import ctypes

import numpy as np

from . import trt

NPARAM = 132868
W16_ELEMS = 6 * 65536


class MLP:
    def __init__(self, params=None, device="cuda:0", stream=None):
        import torch
        self.torch = torch
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.params = torch.zeros(NPARAM, dtype=torch.float32, device=self.device)
        if params is not None:
            self.params.copy_(torch.as_tensor(np.asarray(params, np.float32)))
        self.w16 = torch.zeros(W16_ELEMS, dtype=torch.bfloat16, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.grad_buf = torch.zeros_like(self.params)
        self.loss_buf = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.t = 0
        self._scratch = None
        self.refresh()

    @property
    def _s(self):
        return ctypes.c_void_p(self.stream.cuda_stream)

    def _check(self, rc):
        if rc != 0:
            raise trt.TRTError(rc, "MLP call failed")

    def scratch(self, rows, training):
        n = trt.lib().trt_mlp_scratch_bytes(int(rows), int(training))
        if self._scratch is None or self._scratch.numel() < n:
            self._scratch = self.torch.empty(n, dtype=self.torch.uint8, device=self.device)
        return self._scratch

    def refresh(self):
        self._check(trt.lib().trt_mlp_refresh(self.params.data_ptr(), self.w16.data_ptr(), self._s))

    def forward(self, x):
        """x [rows][3] (FP32 device tensor or array) -> y [rows] FP32 device tensor."""
        t = self.torch
        x = t.as_tensor(x, dtype=t.float32, device=self.device).contiguous()
        rows = x.shape[0]
        y = t.empty(rows, dtype=t.float32, device=self.device)
        sc = self.scratch(rows, 0)
        self._check(trt.lib().trt_mlp_forward(rows, x.data_ptr(), self.params.data_ptr(),
                                              self.w16.data_ptr(), sc.data_ptr(), sc.numel(),
                                              y.data_ptr(), self._s))
        return y

    def forward_fused(self, x):
        """The same network in one persistent tensor-core kernel (no scratch)."""
        t = self.torch
        x = t.as_tensor(x, dtype=t.float32, device=self.device).contiguous()
        rows = x.shape[0]
        y = t.empty(rows, dtype=t.float32, device=self.device)
        self._check(trt.lib().trt_mlp_forward_fused(rows, x.data_ptr(), self.params.data_ptr(),
                                                    self.w16.data_ptr(), y.data_ptr(), self._s))
        return y

    def grad(self, x, target):
        """(grad [NPARAM] FP32 device tensor, loss device tensor [1]); rows % 128 == 0."""
        t = self.torch
        x = t.as_tensor(x, dtype=t.float32, device=self.device).contiguous()
        target = t.as_tensor(target, dtype=t.float32, device=self.device).contiguous()
        rows = x.shape[0]
        sc = self.scratch(rows, 1)
        self._check(trt.lib().trt_mlp_grad(rows, x.data_ptr(), target.data_ptr(),
                                           self.params.data_ptr(), self.w16.data_ptr(),
                                           sc.data_ptr(), sc.numel(), self.grad_buf.data_ptr(),
                                           self.loss_buf.data_ptr(), self._s))
        return self.grad_buf, self.loss_buf

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        self._check(trt.lib().trt_mlp_adam(self.params.data_ptr(), self.grad_buf.data_ptr(),
                                           self.m.data_ptr(), self.v.data_ptr(), self.t,
                                           float(lr), float(beta1), float(beta2), float(eps),
                                           self.w16.data_ptr(), self._s))

    def train_step(self, x, target, lr=1e-3):
        _, loss = self.grad(x, target)
        self.adam_step(lr)
        return loss

    @staticmethod
    def status():
        return trt.lib().trt_mlp_status()


def gemm_bf16(A, B, bias=None, relu=False, mask=None, out32=True, out16=False, out16T=False,
              stream=None):
    """C = A B^T through trt_gemm_bf16 (A [M][K], B [N][K] BF16 device tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    dev = A.device
    o32 = torch.empty((M, N), dtype=torch.float32, device=dev) if out32 else None
    o16 = torch.empty((M, N), dtype=torch.bfloat16, device=dev) if out16 else None
    o16T = torch.empty((N, M), dtype=torch.bfloat16, device=dev) if out16T else None
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    p = lambda t: t.data_ptr() if t is not None else None
    rc = trt.lib().trt_gemm_bf16(M, N, K, A.data_ptr(), B.data_ptr(), p(bias), int(relu),
                                 p(mask), p(o32), p(o16), p(o16T), M,
                                 ctypes.c_void_p(st.cuda_stream))
    if rc != 0:
        raise trt.TRTError(rc, "trt_gemm_bf16")
    return o32, o16, o16T
