"""Python binding of the C ABI in include/trt.h (argument marshalling only).

Every step of the method runs in the CUDA library libtrt.so; this module allocates the
device workspace with torch, passes raw pointers and the current torch stream, and
converts results to numpy / torch.  If the library is missing it raises -- there is no
CPU fallback.
"""
import ctypes
import math
import os
from typing import Dict, Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtrt.so")

TRT_OK, TRT_EINVAL, TRT_ENOTCONVERGED, TRT_ENUMERIC, TRT_ETIMEOUT, TRT_ECUDA, TRT_ENOSPACE = \
    0, -1, -2, -3, -4, -5, -6
TRT_FP64, TRT_SWEEP_FP32, TRT_LO_FP32, TRT_MIXED, TRT_LO_PAIR = 0, 1, 2, 3, 4
CYCLES = {"V": 0, "W": 1, "F": 2}
PRECISIONS = {"fp64": TRT_FP64, "mixed": TRT_MIXED, "sweep32": TRT_SWEEP_FP32,
              "lo32": TRT_LO_FP32, "lopair": TRT_LO_PAIR,
              "sweep32_lopair": TRT_SWEEP_FP32 | TRT_LO_PAIR}

_dp = ctypes.POINTER(ctypes.c_double)
_vp = ctypes.c_void_p


class trt_grid(ctypes.Structure):
    _fields_ = [("n_cells", ctypes.c_int), ("x_edges", _dp), ("length_cm", ctypes.c_double),
                ("T_left_keV", ctypes.c_double), ("T_right_keV", ctypes.c_double)]


class trt_angles(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int)]


class trt_groups(ctypes.Structure):
    _fields_ = [("n_groups", ctypes.c_int), ("edges_keV", _dp), ("nu_a", ctypes.c_double),
                ("nu_b", ctypes.c_double), ("n_levels", ctypes.c_int),
                ("level_groups", ctypes.POINTER(ctypes.c_int))]


class trt_opacity(ctypes.Structure):
    _fields_ = [("scale", ctypes.c_double), ("tr_mode", ctypes.c_int)]


class trt_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("T0_keV", ctypes.c_double), ("stream", _vp),
                ("workspace", _vp), ("workspace_bytes", ctypes.c_size_t)]


class trt_cycle(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("l_max", ctypes.c_int), ("eps", ctypes.c_double),
                ("eps_inner", ctypes.c_double), ("max_outer", ctypes.c_int)]


class trt_stats(ctypes.Structure):
    _fields_ = [("n_ti", ctypes.c_int), ("n_c", ctypes.c_int), ("n_lo", ctypes.c_int),
                ("n_outer", ctypes.c_int), ("ms", ctypes.c_double), ("status", ctypes.c_int),
                ("n_kernels", ctypes.c_int)]


LEVEL_FIELDS = ("phi", "sig", "emis", "Eold", "Esum", "sigR", "etaR", "etaL", "Fold",
                "phib0", "phibX", "C0", "CX", "Ein0", "Fin0", "EinX", "FinX",
                "E", "F", "Eb0", "EbX")
CELL_FIELDS = ("phi", "sig", "emis", "Eold", "Esum", "E")
FACE_FIELDS = ("sigR", "etaR", "etaL", "Fold", "F")


class trt_level(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("fine", ctypes.c_int)] + [(k, _dp) for k in LEVEL_FIELDS]


_lib = None
_rt = None


def _cudart():
    """The CUDA runtime library libtrt.so links against (for test-aid copies)."""
    global _rt
    if _rt is None:
        _rt = ctypes.CDLL(os.path.join("/usr/local/cuda/lib64", "libcudart.so"))
        _rt.cudaMemcpy.restype = ctypes.c_int
        _rt.cudaMemcpy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int]
    return _rt


def lib():
    """Load libtrt.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(the solver has no CPU fallback)")
    L = ctypes.CDLL(LIB_PATH)
    L.trt_workspace_bytes.restype = ctypes.c_size_t
    L.trt_workspace_bytes.argtypes = [ctypes.POINTER(trt_grid), ctypes.POINTER(trt_angles),
                                      ctypes.POINTER(trt_groups), ctypes.POINTER(trt_options)]
    L.trt_create.restype = ctypes.c_int
    L.trt_create.argtypes = [ctypes.POINTER(trt_grid), ctypes.POINTER(trt_angles),
                             ctypes.POINTER(trt_groups), ctypes.POINTER(trt_opacity),
                             ctypes.c_double, ctypes.POINTER(trt_options),
                             ctypes.POINTER(_vp)]
    L.trt_step.restype = ctypes.c_int
    L.trt_step.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(trt_cycle),
                           ctypes.POINTER(trt_stats)]
    L.trt_moments.restype = ctypes.c_int
    L.trt_moments.argtypes = [_vp, _dp, _dp, _dp, _dp, _dp]
    L.trt_intensity.restype = ctypes.c_int
    L.trt_intensity.argtypes = [_vp, _dp, _dp]
    L.trt_set_state.restype = ctypes.c_int
    L.trt_set_state.argtypes = [_vp] + [_dp] * 9
    L.trt_dims.restype = ctypes.c_int
    L.trt_dims.argtypes = [_vp] + [ctypes.POINTER(ctypes.c_int)] * 7
    L.trt_destroy.restype = ctypes.c_int
    L.trt_destroy.argtypes = [_vp]
    L.trt_last_error.restype = ctypes.c_char_p
    L.trt_last_error.argtypes = [_vp]
    L.trt_k_opacity.restype = ctypes.c_int
    L.trt_k_opacity.argtypes = [_vp, _vp, _vp, _vp, _vp]
    L.trt_k_opacity_tr.restype = ctypes.c_int
    L.trt_k_opacity_tr.argtypes = [_vp] * 6
    L.trt_k_sweep.restype = ctypes.c_int
    L.trt_k_sweep.argtypes = [_vp, ctypes.c_double] + [_vp] * 9
    L.trt_k_lo_solve.restype = ctypes.c_int
    L.trt_k_lo_solve.argtypes = [_vp, ctypes.c_double, ctypes.POINTER(trt_level)]
    L.trt_level_view.restype = ctypes.c_int
    L.trt_level_view.argtypes = [_vp, ctypes.c_int, ctypes.POINTER(trt_level)]
    L.trt_k_restrict.restype = ctypes.c_int
    L.trt_k_restrict.argtypes = [_vp, ctypes.POINTER(trt_level), ctypes.POINTER(trt_level)]
    L.trt_k_grey_newton.restype = ctypes.c_int
    L.trt_k_grey_newton.argtypes = [_vp, ctypes.c_double, _vp, _vp, _vp, _vp, ctypes.c_int,
                                    ctypes.c_double, ctypes.POINTER(trt_level), _vp]
    _ip = ctypes.POINTER(ctypes.c_int)
    L.trt_sweep_time.restype = ctypes.c_int
    L.trt_sweep_time.argtypes = [_vp, ctypes.c_double, ctypes.c_int,
                                 ctypes.POINTER(ctypes.c_float)]
    L.trt_autotune.restype = ctypes.c_int
    L.trt_autotune.argtypes = [_vp, ctypes.c_double, ctypes.c_int, _ip, _ip, _ip]
    L.trt_sweep_shapes.restype = ctypes.c_int
    L.trt_sweep_shapes.argtypes = [_vp]
    L.trt_set_sweep_tile.restype = ctypes.c_int
    L.trt_set_sweep_tile.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.trt_get_sweep_tile.restype = ctypes.c_int
    L.trt_get_sweep_tile.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.trt_set_closure.restype = ctypes.c_int
    L.trt_set_closure.argtypes = [_vp] * 4 + [ctypes.c_size_t] + [_vp] * 2
    # learned closure (include/trt_mlp.h)
    L.trt_gemm_bf16.restype = ctypes.c_int
    L.trt_gemm_bf16.argtypes = [ctypes.c_int] * 3 + [_vp] * 3 + [ctypes.c_int] + [_vp] * 4 + \
        [ctypes.c_int, _vp]
    L.trt_mlp_scratch_bytes.restype = ctypes.c_size_t
    L.trt_mlp_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    L.trt_mlp_refresh.restype = ctypes.c_int
    L.trt_mlp_refresh.argtypes = [_vp] * 3
    L.trt_mlp_forward.restype = ctypes.c_int
    L.trt_mlp_forward.argtypes = [ctypes.c_int] + [_vp] * 4 + [ctypes.c_size_t] + [_vp] * 2
    L.trt_mlp_forward_fused.restype = ctypes.c_int
    L.trt_mlp_forward_fused.argtypes = [ctypes.c_int] + [_vp] * 5
    L.trt_mlp_grad.restype = ctypes.c_int
    L.trt_mlp_grad.argtypes = [ctypes.c_int] + [_vp] * 5 + [ctypes.c_size_t] + [_vp] * 3
    L.trt_mlp_adam.restype = ctypes.c_int
    L.trt_mlp_adam.argtypes = [_vp] * 4 + [ctypes.c_int] + [ctypes.c_float] * 4 + [_vp] * 2
    L.trt_mlp_features.restype = ctypes.c_int
    L.trt_mlp_features.argtypes = [ctypes.c_int] * 2 + [_vp] * 6
    L.trt_mlp_status.restype = ctypes.c_int
    L.trt_mlp_status.argtypes = []
    L.trt_fp64_peak.restype = ctypes.c_int
    L.trt_fp64_peak.argtypes = [ctypes.c_int, _vp, ctypes.POINTER(ctypes.c_double)]
    L.trt_k_fastmath.restype = ctypes.c_int
    L.trt_k_fastmath.argtypes = [ctypes.c_int] + [_vp] * 4
    # batched slabs
    L.trt_batch_workspace_bytes.restype = ctypes.c_size_t
    L.trt_batch_workspace_bytes.argtypes = [ctypes.c_int] + [_vp] * 4
    L.trt_create_batch.restype = ctypes.c_int
    L.trt_create_batch.argtypes = [ctypes.c_int] + [_vp] * 7
    L.trt_step_batch.restype = ctypes.c_int
    L.trt_step_batch.argtypes = [_vp, ctypes.c_double, _vp, _vp]
    L.trt_batch_slab.restype = ctypes.c_void_p
    L.trt_batch_slab.argtypes = [_vp, ctypes.c_int]
    L.trt_batch_set_tile.restype = ctypes.c_int
    L.trt_batch_set_tile.argtypes = [_vp, ctypes.c_int, ctypes.c_int]
    L.trt_batch_sweep_time.restype = ctypes.c_int
    L.trt_batch_sweep_time.argtypes = [_vp, ctypes.c_double, ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_float)]
    L.trt_destroy_batch.restype = ctypes.c_int
    L.trt_destroy_batch.argtypes = [_vp]
    L.trt_batch_last_error.restype = ctypes.c_char_p
    L.trt_batch_last_error.argtypes = [_vp]
    L.trt_sweep_noalloc_scratch_bytes.restype = ctypes.c_size_t
    L.trt_sweep_noalloc_scratch_bytes.argtypes = [ctypes.c_int] * 3
    L.trt_sweep_noalloc.restype = ctypes.c_int
    L.trt_sweep_noalloc.argtypes = [ctypes.c_int] * 4 + [ctypes.c_double] + [_vp] * 15
    L.trt_sweep_noalloc_error.restype = ctypes.c_char_p
    L.trt_sweep_noalloc_error.argtypes = []
    _lib = L
    return L


EXPORTED = ("trt_workspace_bytes", "trt_create", "trt_step", "trt_moments", "trt_intensity",
            "trt_set_state", "trt_dims", "trt_destroy", "trt_last_error", "trt_k_opacity",
            "trt_k_opacity_tr", "trt_fp64_peak", "trt_k_sweep", "trt_k_lo_solve", "trt_k_restrict",
            "trt_k_grey_newton",
            "trt_sweep_time", "trt_autotune", "trt_sweep_shapes", "trt_get_sweep_tile",
            "trt_set_sweep_tile",
            "trt_sweep_noalloc_scratch_bytes", "trt_sweep_noalloc", "trt_sweep_noalloc_error",
            "trt_set_closure", "trt_gemm_bf16", "trt_mlp_scratch_bytes", "trt_mlp_refresh", "trt_mlp_forward", "trt_mlp_forward_fused", "trt_level_view",
            "trt_mlp_grad", "trt_mlp_adam", "trt_mlp_features", "trt_mlp_status",
            "trt_batch_workspace_bytes", "trt_create_batch", "trt_step_batch",
            "trt_batch_slab", "trt_batch_set_tile", "trt_batch_sweep_time",
            "trt_destroy_batch", "trt_batch_last_error", "trt_k_fastmath")


def fp64_peak(reps=4000, device=None):
    """The device's FP64 FMA rate in TFLOP/s, measured by trt_fp64_peak on the current
    torch stream of `device`."""
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda")
    st = torch.cuda.current_stream(dev)
    out = ctypes.c_double()
    with torch.cuda.device(dev):
        rc = lib().trt_fp64_peak(int(reps), ctypes.c_void_p(st.cuda_stream), ctypes.byref(out))
    if rc != TRT_OK:
        raise TRTError(rc, "trt_fp64_peak failed")
    return out.value


class TRTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"trt error {code}: {msg}")
        self.code = code


def _ptr(a):
    return ctypes.cast(ctypes.c_void_p(a.data_ptr()), _dp) if a is not None else None


def _np_dp(a):
    return a.ctypes.data_as(_dp) if a is not None else None


class Solver:
    """One slab on one GPU: trt_create / trt_step / trt_moments / trt_destroy."""

    def __init__(self, n_cells, length_cm, N, edges, level_groups, opac_scale=1.0,
                 cv=0.5917 * 0.01372, T0=1e-3, T_left=1.0, T_right=0.0, precision="fp64",
                 device=None, stream=None, x_edges=None, tr_mode=False):
        import torch
        self.torch = torch
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.index is None:   # always pass an explicit index to the CUDA runtime
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        L = lib()
        self._edges = np.ascontiguousarray(edges, np.float64)
        self._levels = np.ascontiguousarray(level_groups, np.int32)
        self._xe = None if x_edges is None else np.ascontiguousarray(x_edges, np.float64)
        self.grid = trt_grid(int(n_cells), _np_dp(self._xe), float(length_cm), float(T_left),
                             float(T_right))
        self.angles = trt_angles(int(N))
        self.groups = trt_groups(self._edges.size - 1, _np_dp(self._edges), 0.0, 0.0,
                                 self._levels.size,
                                 self._levels.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        self.opacity = trt_opacity(float(opac_scale), int(bool(tr_mode)))
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        torch.cuda.synchronize(self.device)   # initialise torch's context on the device
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        opt = trt_options(self.precision, float(T0), ctypes.c_void_p(self.stream.cuda_stream),
                          None, 0)
        nbytes = L.trt_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.angles),
                                       ctypes.byref(self.groups), ctypes.byref(opt))
        if nbytes == 0:
            raise TRTError(TRT_EINVAL, "invalid problem (trt_workspace_bytes returned 0)")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.workspace.data_ptr()
        aligned = (base + 255) // 256 * 256
        opt.workspace = ctypes.c_void_p(aligned)
        opt.workspace_bytes = nbytes
        h = ctypes.c_void_p()
        rc = L.trt_create(ctypes.byref(self.grid), ctypes.byref(self.angles),
                          ctypes.byref(self.groups), ctypes.byref(self.opacity), float(cv),
                          ctypes.byref(opt), ctypes.byref(h))
        if rc != TRT_OK:
            raise TRTError(rc, L.trt_last_error(None).decode())
        self.h = h
        self.workspace_bytes = nbytes
        dims = [ctypes.c_int() for _ in range(7)]
        L.trt_dims(self.h, *[ctypes.byref(d) for d in dims])
        self.nx, self.N, self.M, self.G, self.ldG, self.n_levels, _ = [d.value for d in dims]

    @classmethod
    def from_slab(cls, slab, precision="fp64", **kw):
        return cls(slab.n_cells, slab.length_cm, slab.N, slab.edges(), slab.levels,
                   slab.opac_scale, slab.cv, slab.T0, slab.T_left, slab.T_right,
                   precision=precision, **kw)

    def _check(self, rc, allow=()):
        if rc != TRT_OK and rc not in allow:
            raise TRTError(rc, lib().trt_last_error(self.h).decode())
        return rc

    def step(self, dt, cycle="V", l_max=4, eps=1e-8, eps_inner=None, max_outer=100):
        if eps_inner is None:
            eps_inner = eps / 10.0 if eps > 0 else -1.0
        c = trt_cycle(CYCLES[cycle] if isinstance(cycle, str) else int(cycle), int(l_max),
                      float(eps), float(eps_inner), int(max_outer))
        st = trt_stats()
        rc = lib().trt_step(self.h, float(dt), ctypes.byref(c), ctypes.byref(st))
        self._check(rc, allow=(TRT_ENOTCONVERGED,))
        return dict(n_ti=st.n_ti, n_c=st.n_c, n_lo=st.n_lo, n_outer=st.n_outer, ms=st.ms,
                    status=rc, n_kernels=st.n_kernels)

    def moments(self, groups=True) -> Dict[str, np.ndarray]:
        """T, the grey E and F and, with groups, the group E_g and F_g of the current state
        (trt_moments; groups=False reads only the cell and face fields of the grey level)."""
        T = np.zeros(self.nx)
        Eg = np.zeros((self.G, self.nx)) if groups else None
        Fg = np.zeros((self.G, self.nx + 1)) if groups else None
        E = np.zeros(self.nx)
        F = np.zeros(self.nx + 1)
        self._check(lib().trt_moments(self.h, _np_dp(T), _np_dp(Eg), _np_dp(Fg), _np_dp(E),
                                      _np_dp(F)))
        out = dict(T=T, E=E, F=F)
        if groups:
            out.update(Eg=Eg, Fg=Fg)
        return out

    def qd_factors(self):
        """The cell QD factors f [G][nx] of the last sweep (FP64 numpy array)."""
        f = np.zeros((self.G, self.nx))
        self._check(lib().trt_intensity(self.h, None, _np_dp(f)))
        return f

    def intensity(self):
        """(I [M][nx][2][G], f [G][nx]) as FP64 numpy arrays (group padding dropped)."""
        I = np.zeros((self.M, self.nx, 2, self.ldG))
        f = np.zeros((self.G, self.nx))
        self._check(lib().trt_intensity(self.h, _np_dp(I), _np_dp(f)))
        return I[..., :self.G].copy(), f

    def set_state(self, T=None, Eg=None, Fg=None, I=None, f=None, fb0=None, fbX=None, C0=None,
                  CX=None):
        def c(a):
            return None if a is None else np.ascontiguousarray(a, np.float64)
        if I is not None:
            Ip = np.zeros((self.M, self.nx, 2, self.ldG))
            Ip[..., :self.G] = I
            I = Ip
        arrs = [c(a) for a in (T, Eg, Fg, I, f, fb0, fbX, C0, CX)]
        self._check(lib().trt_set_state(self.h, *[_np_dp(a) for a in arrs]))

    # ---- kernel-level entry points (torch CUDA tensors in, torch tensors out) ----
    def _t(self, a, dtype=None):
        t = self.torch
        dtype = dtype or t.float64
        if isinstance(a, np.ndarray):
            a = t.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=dtype).contiguous()

    def k_opacity(self, T):
        t = self.torch
        T = self._t(T)
        out = [t.empty((self.G, self.nx), dtype=t.float64, device=self.device) for _ in range(3)]
        self._check(lib().trt_k_opacity(self.h, T.data_ptr(), *[o.data_ptr() for o in out]))
        return tuple(out)

    def k_opacity_tr(self, T, Erad):
        """sigma_E, e_g, sigma_R at (T, T_r = (Erad/a_R)^{1/4}) (a T_r handle only)."""
        t = self.torch
        T, Erad = self._t(T), self._t(Erad)
        out = [t.empty((self.G, self.nx), dtype=t.float64, device=self.device) for _ in range(3)]
        self._check(lib().trt_k_opacity_tr(self.h, T.data_ptr(), Erad.data_ptr(),
                                           *[o.data_ptr() for o in out]))
        return tuple(out)

    def k_sweep(self, dt, sigE, emis, I_old):
        """I_old: [M][nx][2][G] (padded to ldG here); returns I_new [M][nx][2][G], f, fb0,
        fbX, C0, CX as torch tensors."""
        t = self.torch
        rdt = t.float32 if self.precision & TRT_SWEEP_FP32 else t.float64
        Ip = t.zeros((self.M, self.nx, 2, self.ldG), dtype=rdt, device=self.device)
        Ip[..., :self.G] = self._t(I_old, rdt)
        In = t.zeros_like(Ip)
        f = t.empty((self.G, self.nx), dtype=t.float64, device=self.device)
        b = [t.empty(self.G, dtype=t.float64, device=self.device) for _ in range(4)]
        sigE, emis = self._t(sigE), self._t(emis)
        self._check(lib().trt_k_sweep(self.h, float(dt), sigE.data_ptr(), emis.data_ptr(),
                                      Ip.data_ptr(), In.data_ptr(), f.data_ptr(),
                                      *[x.data_ptr() for x in b]))
        return (In[..., :self.G], f, *b)

    def _level(self, d, n, fine=False):
        t = self.torch
        keep = {}
        for k in LEVEL_FIELDS:
            shape = (n, self.nx) if k in CELL_FIELDS else (n, self.nx + 1) if k in FACE_FIELDS else (n,)
            if fine and k == "sigR":
                shape = (n, self.nx)
            v = d.get(k)
            v = t.zeros(shape, dtype=t.float64, device=self.device) if v is None else self._t(v)
            assert tuple(v.shape) == shape, (k, v.shape, shape)
            keep[k] = v
        lv = trt_level(n, int(fine), *[_ptr(keep[k]) for k in LEVEL_FIELDS])
        return lv, keep

    def k_lo_solve(self, dt, level, fine=False):
        n = int(self._t(level["phi"]).shape[0])
        lv, keep = self._level(level, n, fine)
        self._check(lib().trt_k_lo_solve(self.h, float(dt), ctypes.byref(lv)))
        return {k: keep[k] for k in ("E", "F", "Eb0", "EbX")}

    def k_restrict(self, src, n_to, fine=False):
        n = int(self._t(src["phi"]).shape[0])
        ls, ks = self._level(src, n, fine)
        ld, kd = self._level({}, n_to)
        self._check(lib().trt_k_restrict(self.h, ctypes.byref(ls), ctypes.byref(ld)))
        return kd

    def k_grey_newton(self, dt, Tstar, Told, grey, sig_prev=None, T_prev=None, secant_cut=1e-7):
        t = self.torch
        lv, keep = self._level(grey, 1)
        Ts, To = self._t(Tstar), self._t(Told)
        have = sig_prev is not None
        sp = self._t(sig_prev) if have else None
        tp = self._t(T_prev) if have else None
        T = t.empty(self.nx, dtype=t.float64, device=self.device)
        rc = lib().trt_k_grey_newton(self.h, float(dt), Ts.data_ptr(), To.data_ptr(),
                                     sp.data_ptr() if have else None,
                                     tp.data_ptr() if have else None, int(have),
                                     float(secant_cut), ctypes.byref(lv), T.data_ptr())
        self._check(rc, allow=(TRT_ENUMERIC,))
        return rc, T, {k: keep[k] for k in ("E", "F", "Eb0", "EbX")}

    def set_closure(self, net):
        """Warm-start every step's s = 0 phase from the MLP `net` (paper_2011_05427_gb300.mlp.MLP);
        None removes it."""
        t = self.torch
        if net is None:
            self._check(lib().trt_set_closure(self.h, None, None, None, 0, None, None))
            self._closure = None
            return
        rows = self.G * self.nx
        x = t.empty((rows, 3), dtype=t.float32, device=self.device)
        y = t.empty(rows, dtype=t.float32, device=self.device)
        sc = t.empty(lib().trt_mlp_scratch_bytes(rows, 0), dtype=t.uint8, device=self.device)
        self._check(lib().trt_set_closure(self.h, net.params.data_ptr(), net.w16.data_ptr(),
                                          sc.data_ptr(), sc.numel(), x.data_ptr(), y.data_ptr()))
        self._closure = (net, x, y, sc)   # keep the buffers alive

    def level_view(self, which):
        """Host copies of the handle's fine (0), coarse (1) or grey (2) level arrays."""
        lv = trt_level()
        self._check(lib().trt_level_view(self.h, int(which), ctypes.byref(lv)))
        n, nx = lv.n, self.nx
        shapes = dict(phi=(n, nx), sig=(n, nx), emis=(n, nx), Eold=(n, nx), Esum=(n, nx),
                      sigR=(n, nx) if lv.fine else (n, nx + 1), etaR=(n, nx + 1),
                      etaL=(n, nx + 1), Fold=(n, nx + 1), phib0=(n,), phibX=(n,), C0=(n,),
                      CX=(n,), Ein0=(n,), Fin0=(n,), EinX=(n,), FinX=(n,), E=(n, nx),
                      F=(n, nx + 1), Eb0=(n,), EbX=(n,))
        out = {"n": n, "fine": lv.fine}
        self.torch.cuda.synchronize(self.device)
        rt = _cudart()
        for k, shp in shapes.items():
            ptr = ctypes.cast(getattr(lv, k), ctypes.c_void_p).value
            if not ptr:
                continue
            a = np.empty(shp, np.float64)
            if rt.cudaMemcpy(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(ptr),
                             ctypes.c_size_t(a.nbytes), 2) != 0:   # device to host
                raise TRTError(TRT_ECUDA, "cudaMemcpy of a level array failed")
            out[k] = a
        return out

    def sweep_time(self, dt, reps=10) -> float:
        """ms per sweep of the step's own sweep configuration (state unchanged)."""
        ms = ctypes.c_float()
        self._check(lib().trt_sweep_time(self.h, float(dt), int(reps), ctypes.byref(ms)))
        return ms.value

    def autotune(self, dt, reps=5):
        """Time every candidate sweep tile and keep the fastest; returns (D, S, NS)."""
        D, S, NS = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(lib().trt_autotune(self.h, float(dt), int(reps), ctypes.byref(D),
                                       ctypes.byref(S), ctypes.byref(NS)))
        return D.value, S.value, NS.value

    def set_sweep_tile(self, D, shape):
        self._check(lib().trt_set_sweep_tile(self.h, int(D), int(shape)))

    def sweep_shapes(self) -> int:
        return lib().trt_sweep_shapes(self.h)

    def sweep_tile(self):
        """The sweep tile the next step uses: (D, shape); D = 0 is the library default."""
        D, sh = ctypes.c_int(), ctypes.c_int()
        self._check(lib().trt_get_sweep_tile(self.h, ctypes.byref(D), ctypes.byref(sh)))
        return D.value, sh.value

    def close(self):
        if getattr(self, "h", None) and getattr(self, "_owned", True):
            lib().trt_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many slabs stepped together (trt_create_batch / trt_step_batch).  Every slab's
    results are read through `slab(s)`, a Solver view of the batch's handle for slab s."""

    def __init__(self, slabs, precision="fp64", device=None, T0=None, tr_mode=False):
        import torch
        self.torch = torch
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.n = n = len(slabs)
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        L = lib()
        self._keep = []
        grids = (trt_grid * n)()
        angles = (trt_angles * n)()
        groups = (trt_groups * n)()
        opac = (trt_opacity * n)()
        cv = (ctypes.c_double * n)()
        for k, sl in enumerate(slabs):
            e = np.ascontiguousarray(sl.edges(), np.float64)
            lv = np.ascontiguousarray(sl.levels, np.int32)
            self._keep += [e, lv]
            grids[k] = trt_grid(int(sl.n_cells), None, float(sl.length_cm), float(sl.T_left),
                                float(sl.T_right))
            angles[k] = trt_angles(int(sl.N))
            groups[k] = trt_groups(e.size - 1, _np_dp(e), 0.0, 0.0, lv.size,
                                   lv.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
            opac[k] = trt_opacity(float(sl.opac_scale), int(bool(tr_mode)))
            cv[k] = float(sl.cv)
        torch.cuda.synchronize(dev)
        # a stream of its own: the batch captures its stages as CUDA graphs
        self.stream = torch.cuda.Stream(dev)
        t0 = float(T0 if T0 is not None else slabs[0].T0)
        opt = trt_options(self.precision, t0, ctypes.c_void_p(self.stream.cuda_stream), None, 0)
        nbytes = L.trt_batch_workspace_bytes(n, grids, angles, groups, ctypes.byref(opt))
        if nbytes == 0:
            raise TRTError(TRT_EINVAL, "invalid batch (trt_batch_workspace_bytes returned 0)")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=dev)
        opt.workspace = ctypes.c_void_p((self.workspace.data_ptr() + 255) // 256 * 256)
        opt.workspace_bytes = nbytes
        self.workspace_bytes = nbytes
        b = ctypes.c_void_p()
        rc = L.trt_create_batch(n, grids, angles, groups, opac, cv, ctypes.byref(opt),
                                ctypes.byref(b))
        if rc != TRT_OK:
            raise TRTError(rc, L.trt_last_error(None).decode())
        self.b = b
        self._views = [None] * n

    def _check(self, rc, allow=()):
        if rc != TRT_OK and rc not in allow:
            raise TRTError(rc, lib().trt_batch_last_error(self.b).decode())
        return rc

    def step(self, dt, cycle="V", l_max=4, eps=1e-8, eps_inner=None, max_outer=100):
        if eps_inner is None:
            eps_inner = eps / 10.0 if eps > 0 else -1.0
        c = trt_cycle(CYCLES[cycle] if isinstance(cycle, str) else int(cycle), int(l_max),
                      float(eps), float(eps_inner), int(max_outer))
        st = (trt_stats * self.n)()
        rc = lib().trt_step_batch(self.b, float(dt), ctypes.byref(c), st)
        self._check(rc, allow=(TRT_ENOTCONVERGED,))
        return [dict(n_ti=x.n_ti, n_c=x.n_c, n_lo=x.n_lo, n_outer=x.n_outer, status=x.status,
                     n_kernels=x.n_kernels) for x in st]

    def slab(self, s) -> "Solver":
        if self._views[s] is None:
            v = Solver.__new__(Solver)
            v.torch = self.torch
            v.device = self.device
            v.stream = self.stream
            v.precision = self.precision
            v.h = ctypes.c_void_p(lib().trt_batch_slab(self.b, int(s)))
            dims = [ctypes.c_int() for _ in range(7)]
            lib().trt_dims(v.h, *[ctypes.byref(d) for d in dims])
            v.nx, v.N, v.M, v.G, v.ldG, v.n_levels, _ = [d.value for d in dims]
            v._owned = False
            self._views[s] = v
        return self._views[s]

    def set_tile(self, D, shape):
        self._check(lib().trt_batch_set_tile(self.b, int(D), int(shape)))

    def sweep_time(self, dt, reps=5) -> float:
        ms = ctypes.c_float()
        self._check(lib().trt_batch_sweep_time(self.b, float(dt), int(reps), ctypes.byref(ms)))
        return ms.value

    def autotune(self, dt, reps=3):
        """Time the batched sweep for every (D, shape) every slab admits; keep the fastest."""
        best = None
        Ds = [D for D in (16, 8, 4, 2) if all(self.slab(s).N % D == 0 for s in range(self.n))
              and all(D >= min(4, self.slab(s).N & -self.slab(s).N) for s in range(self.n))]
        nshape = lib().trt_sweep_shapes(self.slab(0).h)
        for D in Ds:
            for sh in range(nshape):
                try:
                    self.set_tile(D, sh)
                    t = self.sweep_time(dt, reps)
                except TRTError:
                    continue
                if best is None or t < best[0]:
                    best = (t, D, sh)
        self.set_tile(best[1], best[2])
        return best

    def close(self):
        if getattr(self, "b", None):
            self.torch.cuda.synchronize(self.device)
            lib().trt_destroy_batch(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
