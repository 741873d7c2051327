"""Thin Python binding of libslingbag (the sm_103a SlingBAG Pro hot path).

Argument marshalling only: every step runs in the CUDA library through its
C ABI (include/slingbag.h). PyTorch supplies device memory and the current
stream. There is no CPU fallback: if the library is missing or no GPU is
present, the calls raise.

Point clouds are (5, n_cap) float32 CUDA tensors with rows x, y, z, R, p0;
gradients and optimizer moments use the same layout. The live ball count can
be a Python int or a one-element int32 CUDA tensor (kept on the device so
that growth needs no host round trip).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libslingbag.so")

SBP_OK = 0
# status codes of include/slingbag.h
SBP_ERR_ARG, SBP_ERR_CUDA, SBP_ERR_CAPACITY = -1, -2, -3
SBP_ERR_LEVEL, SBP_ERR_TIMEOUT, SBP_ERR_NUMERIC = -4, -5, -6
W_MODES = {"clamp": 0, "none": 1, "cos": 2}
MASK_P0, MASK_R, MASK_XYZ, MASK_ALL = 1, 2, 4, 7
SOFTPLUS_R = 8  # optimise R through R = softplus(a) (positivity-constrained refinement)
KEEP_NEG, KEEP_NONPOS, DROP_ZERO, GROW = 0, 1, 2, 3
# or'ed into a forward tile (set_tiles): 832 trace cells per sensor in shared
# memory and 32 warps per CTA instead of 416 and 16
TILE_WIDE = 0x10000

_P = ctypes.c_void_p


class SlingbagError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


class _Balls(ctypes.Structure):
    _fields_ = [("x", _P), ("y", _P), ("z", _P), ("R", _P), ("p0", _P)]


class _Params(ctypes.Structure):
    _fields_ = [("weight_mode", ctypes.c_int), ("reserved", ctypes.c_int * 7)]


class _GrowParams(ctypes.Structure):
    _fields_ = [("p_min", ctypes.c_float), ("R_min", ctypes.c_float), ("R_max", ctypes.c_float),
                ("g_dup", ctypes.c_float), ("seed", ctypes.c_uint64), ("grad_mask", ctypes.c_int),
                ("prune_zero", ctypes.c_int), ("destroy", ctypes.c_int), ("split", ctypes.c_int),
                ("duplicate", ctypes.c_int)]


class _AdamParams(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float * 5), ("beta1", ctypes.c_float), ("beta2", ctypes.c_float),
                ("eps", ctypes.c_float)]


class _Stage(ctypes.Structure):
    _fields_ = [("level", ctypes.c_int), ("iterations", ctypes.c_int),
                ("grad_mask", ctypes.c_uint), ("grow", ctypes.c_int),
                ("duplicate", ctypes.c_int)]


MAX_STAGES = 32


class _ReconParams(ctypes.Structure):
    _fields_ = [("zero_grad_mode", ctypes.c_int), ("zero_grad_level", ctypes.c_int),
                ("n_stages", ctypes.c_int), ("stages", _Stage * MAX_STAGES),
                ("adam", _AdamParams), ("grow", _GrowParams), ("loss_log_dev", _P),
                ("n_log_dev", _P), ("log_capacity", ctypes.c_int),
                ("spatial_sort", ctypes.c_int)]


_lib = None

# name -> (restype, argtypes); the C ABI of include/slingbag.h
_SIGS = {
    "sbp_version": (ctypes.c_char_p, []),
    "sbp_last_error": (ctypes.c_char_p, []),
    "sbp_create_array": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, _P, ctypes.c_int, ctypes.c_int,
                                        ctypes.POINTER(_Params), ctypes.POINTER(_P)]),
    "sbp_destroy_array": (ctypes.c_int, [_P]),
    "sbp_level_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_double)]),
    "sbp_set_sampling_level": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "sbp_forward": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, ctypes.c_uint, _P]),
    "sbp_forward_static": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, ctypes.c_int, _Balls, _P, ctypes.c_int,
                                          _P, _P]),
    "sbp_residual": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "sbp_adjoint": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _Balls, ctypes.c_uint, _P]),
    "sbp_store_windows": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _P]),
    "sbp_adjoint_stored": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _P, _Balls,
                                          ctypes.c_uint, _P]),
    "sbp_filter_grow": (ctypes.c_int, [_P, _Balls, _Balls, ctypes.POINTER(_P), ctypes.c_int, _P,
                                       ctypes.c_int, ctypes.POINTER(_GrowParams), ctypes.c_int,
                                       _P]),
    "sbp_adam_step": (ctypes.c_int, [_P, _Balls, _Balls, _Balls, _Balls, _P, ctypes.c_int,
                                     ctypes.c_int, ctypes.POINTER(_AdamParams), ctypes.c_uint,
                                     _P]),
    "sbp_sort_cloud": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, ctypes.c_int, _P]),
    "sbp_reconstruct": (ctypes.c_int, [_P, _P, _Balls, _P, ctypes.c_int,
                                       ctypes.POINTER(_ReconParams), _P]),
    "sbp_launch_count": (ctypes.c_longlong, []),
    "sbp_set_frames": (ctypes.c_int, [_P, _P, ctypes.c_int, _P]),
    "sbp_set_sampling_level_frames": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P]),
    "sbp_forward_frames": (ctypes.c_int, [_P, _Balls, _P, _P, _P]),
    "sbp_residual_frames": (ctypes.c_int, [_P, _P, _P, _P, _P, _P]),
    "sbp_adjoint_frames": (ctypes.c_int, [_P, _Balls, _P, _P, _Balls, ctypes.c_uint, _P]),
    "sbp_filter_grow_frames": (ctypes.c_int, [_P, _Balls, _Balls, ctypes.POINTER(_P),
                                              ctypes.c_int, _P, ctypes.POINTER(_GrowParams),
                                              ctypes.c_int, _P]),
    "sbp_adam_step_frames": (ctypes.c_int, [_P, _Balls, _Balls, _Balls, _Balls, _P, ctypes.c_int,
                                            ctypes.POINTER(_AdamParams), ctypes.c_uint, _P]),
    "sbp_reconstruct_frames": (ctypes.c_int, [_P, _P, _Balls, _P, ctypes.POINTER(_ReconParams),
                                              _P]),
    "sbp_set_frame_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
    "sbp_get_frame_tiles": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "sbp_autotune_frames": (ctypes.c_int, [_P, _Balls, _P, _P, _P, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_int)]),
    "sbp_set_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "sbp_get_tiles": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int)]),
    "sbp_autotune": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _P,
                                    ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "sbp_probe_fp32_fma": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "sbp_probe_fp32x2_fma": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "sbp_probe_issue": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)]),
    "sbp_probe_smem_atomic": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "sbp_forward_gauss": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _P]),
    "sbp_adjoint_gauss": (ctypes.c_int, [_P, _Balls, _P, ctypes.c_int, _P, _Balls, ctypes.c_uint,
                                         _P]),
    "sbp_envelope_create": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_P)]),
    "sbp_envelope_destroy": (ctypes.c_int, [_P]),
    "sbp_envelope_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), _P]),
    "sbp_envelope_faces": (ctypes.c_int, [_P, _P]),
    "sbp_envelope_classify": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_longlong, ctypes.c_double,
                                             _P, _P]),
    "sbp_envelope_sample": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_longlong,
                                           ctypes.c_longlong, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           _Balls, ctypes.c_int, _P, _P]),
    "sbp_voxelize": (ctypes.c_int, [_Balls, _P, _P, ctypes.c_int, _P, ctypes.c_double,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P, _P]),
    "sbp_conv3d_bf16": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       _P, ctypes.c_int, _P, ctypes.c_int, ctypes.c_int, _P,
                                       ctypes.c_int, _P]),
    "sbp_cnn_status": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "sbp_das_volume": (ctypes.c_int, [_P, _P, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, _P, _P]),
    "sbp_cnn_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_uint64,
                                      ctypes.POINTER(_P)]),
    "sbp_cnn_destroy": (ctypes.c_int, [_P]),
    "sbp_cnn_num_params": (ctypes.c_int, []),
    "sbp_cnn_params": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "sbp_cnn_forward": (ctypes.c_int, [_P, _P, _P, _P]),
    "sbp_cnn_train_step": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_float, ctypes.c_float, _P,
                                          _P]),
    "sbp_cnn_grad": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_float, _P, _P, _P]),
    "sbp_cnn_propose": (ctypes.c_int, [_P, _P, ctypes.c_float, ctypes.c_uint64, _P,
                                       ctypes.c_double, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_int, _Balls, ctypes.c_int, _P,
                                       _P]),
    "sbp_sync_status": (ctypes.c_int, [_P, _P]),
    "sbp_get_inside_pairs": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_longlong)]),
}


def load_library(path: str = LIB_PATH):
    """Load libslingbag.so (built by `paper_2601_00551_gb300.build`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"libslingbag is not built ({path} missing); run "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(fn: str, code: int):
    if code != SBP_OK:
        raise SlingbagError(fn, code, load_library().sbp_last_error().decode())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _on_current_device(t: torch.Tensor):
    """Every pointer handed to the library is device memory of the current
    device, where its kernels run: a host tensor or one on another GPU is
    refused here, before anything is enqueued."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor, got one on " + str(t.device))
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError(f"tensor on {t.device}, but the current device is cuda:{cur} "
                         "(select it with torch.cuda.set_device)")


def _rows(t: torch.Tensor) -> _Balls:
    if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2 or t.shape[0] != 5 \
            or not t.is_contiguous():
        raise ValueError("expected a contiguous (5, n) float32 CUDA tensor")
    _on_current_device(t)
    base, stride = t.data_ptr(), t.stride(0) * 4
    return _Balls(*(base + k * stride for k in range(5)))


def _dptr(t):
    if t is None:
        return None
    _on_current_device(t)
    return ctypes.c_void_p(t.data_ptr())


@dataclasses.dataclass
class GrowParams:
    """Growth thresholds (see sbp_grow_params in include/slingbag.h)."""
    p_min: float = 1e-3
    R_min: float = 0.02
    R_max: float = 0.3
    g_dup: float = 1e30
    seed: int = 0
    grad_mask: int = MASK_ALL
    prune_zero: bool = True
    destroy: bool = True
    split: bool = True
    duplicate: bool = False

    def c(self) -> _GrowParams:
        return _GrowParams(self.p_min, self.R_min, self.R_max, self.g_dup,
                           self.seed & ((1 << 64) - 1), self.grad_mask, int(self.prune_zero),
                           int(self.destroy), int(self.split), int(self.duplicate))


@dataclasses.dataclass
class AdamParams:
    lr: tuple = (1e-3, 1e-3, 1e-3, 1e-3, 1e-2)  # x, y, z, R, p0
    beta1: float = 0.9
    beta2: float = 0.999
    eps: float = 1e-8

    def c(self) -> _AdamParams:
        return _AdamParams((ctypes.c_float * 5)(*self.lr), self.beta1, self.beta2, self.eps)


@dataclasses.dataclass
class Stage:
    """`iterations` iterations at level `level` (see sbp_stage)."""
    level: int
    iterations: int
    grad_mask: int = MASK_ALL
    grow: bool = True
    duplicate: bool = False


def launch_count() -> int:
    """Kernels launched by libslingbag in this process so far."""
    return int(load_library().sbp_launch_count())


def probe_rates() -> dict:
    """Measured throughput of the units that bound the hot kernels
    (include/slingbag_probe.h): FP32 FMA/s (single and packed-pair
    instructions), warp instructions issued/s and
    shared-memory atomic adds/s (u32, u64, f32), on the current device."""
    lib = load_library()
    out = {}
    v = ctypes.c_double()
    _check("sbp_probe_fp32_fma", lib.sbp_probe_fp32_fma(ctypes.byref(v)))
    out["fp32_fma_per_s"] = v.value
    _check("sbp_probe_fp32x2_fma", lib.sbp_probe_fp32x2_fma(ctypes.byref(v)))
    out["fp32x2_fma_per_s"] = v.value
    _check("sbp_probe_issue", lib.sbp_probe_issue(ctypes.byref(v)))
    out["warp_inst_per_s"] = v.value
    for kind, name in enumerate(("u32", "u64", "f32")):
        _check("sbp_probe_smem_atomic", lib.sbp_probe_smem_atomic(kind, ctypes.byref(v)))
        out[f"smem_atomic_{name}_per_s"] = v.value
    return out


class SensorArray:
    """A sensor array with its sampling hierarchy (sbp_create_array)."""

    def __init__(self, pos, normal, c: float, fs_mhz: float, T: int, factors=(1,),
                 n_cap: int = 1, weight_mode: str = "clamp", device=None):
        self._lib = load_library()
        if not torch.cuda.is_available():
            raise RuntimeError("libslingbag needs a CUDA GPU")
        if device is not None:
            torch.cuda.set_device(device)
        self.device = torch.device("cuda", torch.cuda.current_device())
        pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float32).reshape(-1, 3))
        nrm = np.ascontiguousarray(np.asarray(normal, dtype=np.float32).reshape(-1, 3))
        if pos.shape != nrm.shape:
            raise ValueError("pos and normal must both be (M, 3)")
        fac = np.ascontiguousarray(np.asarray(factors, dtype=np.int32))
        self.M, self.T, self.n_cap = pos.shape[0], int(T), int(n_cap)
        self.c, self.fs = float(c), float(fs_mhz)
        self.factors = tuple(int(f) for f in fac)
        params = _Params(W_MODES[weight_mode])
        h = _P()
        torch.cuda.synchronize()
        _check("sbp_create_array", self._lib.sbp_create_array(
            pos.ctypes.data, nrm.ctypes.data, self.M, self.c, self.fs, self.T,
            fac.ctypes.data, len(fac), self.n_cap, ctypes.byref(params), ctypes.byref(h)))
        self._h = h
        self.level = 0

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sbp_destroy_array(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------ levels
    def level_info(self, k: int):
        T = ctypes.c_int()
        dt = ctypes.c_double()
        _check("sbp_level_info", self._lib.sbp_level_info(self._h, k, ctypes.byref(T),
                                                          ctypes.byref(dt)))
        return T.value, dt.value

    @property
    def Tk(self) -> int:
        return self.level_info(self.level)[0]

    def set_sampling_level(self, k: int, y_full: torch.Tensor | None = None,
                           out: torch.Tensor | None = None):
        """Select level k; with y_full (M, T) also return Downsample_{f_k}(y_full)."""
        Tk = self.level_info(k)[0]
        if y_full is not None:
            self._check_traces(y_full, self.T)
            if out is None:
                out = torch.empty((self.M, Tk), dtype=torch.float32, device=self.device)
            self._check_traces(out, Tk)
        _check("sbp_set_sampling_level", self._lib.sbp_set_sampling_level(
            self._h, k, _dptr(y_full), _dptr(out if y_full is not None else None), _stream()))
        self.level = k
        return out

    def set_tiles(self, k: int, fwd_chunk: int = 0, adj_split: int = 0):
        """Tile choice of the forward and adjoint at level k (sbp_set_tiles; 0 = default)."""
        _check("sbp_set_tiles", self._lib.sbp_set_tiles(self._h, k, fwd_chunk, adj_split))

    def get_tiles(self, k: int):
        c, sp = ctypes.c_int(), ctypes.c_int()
        _check("sbp_get_tiles", self._lib.sbp_get_tiles(self._h, k, ctypes.byref(c),
                                                        ctypes.byref(sp)))
        return c.value, sp.value

    def autotune(self, balls: torch.Tensor, n=None, G: torch.Tensor | None = None):
        """Tile autotuner at the current level (sbp_autotune); returns and keeps
        (forward balls per CTA, adjoint CTAs per ball chunk). G defaults to
        standard normal traces."""
        Tk = self.Tk
        S = torch.empty((self.M, Tk), dtype=torch.float32, device=self.device)
        if G is None:
            G = torch.randn((self.M, Tk), dtype=torch.float32, device=self.device)
        self._check_traces(G, Tk)
        nd = self._n(n, balls.shape[1])
        c, sp = ctypes.c_int(), ctypes.c_int()
        torch.cuda.synchronize()
        _check("sbp_autotune", self._lib.sbp_autotune(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], _dptr(S), _dptr(G),
            ctypes.byref(c), ctypes.byref(sp)))
        return c.value, sp.value

    def _check_traces(self, t, T):
        if t.dtype != torch.float32 or not t.is_cuda or tuple(t.shape) != (self.M, T) \
                or not t.is_contiguous():
            raise ValueError(f"expected a contiguous ({self.M}, {T}) float32 CUDA tensor")

    def _n(self, n, n_cap):
        if n is None or isinstance(n, torch.Tensor):
            if n is not None and (n.dtype != torch.int32 or not n.is_cuda):
                raise ValueError("n must be an int32 CUDA tensor")
            return n
        return torch.tensor([int(n)], dtype=torch.int32, device=self.device)

    # ----------------------------------------------------------------- hot path
    def forward(self, balls: torch.Tensor, n=None, out: torch.Tensor | None = None):
        """Traces S (M, T_k) at the current level (sbp_forward)."""
        Tk = self.Tk
        if out is None:
            out = torch.empty((self.M, Tk), dtype=torch.float32, device=self.device)
        self._check_traces(out, Tk)
        nd = self._n(n, balls.shape[1])
        _check("sbp_forward", self._lib.sbp_forward(self._h, _rows(balls), _dptr(nd),
                                                    balls.shape[1], _dptr(out), 0, _stream()))
        return out

    def residual(self, S: torch.Tensor | None, y_k: torch.Tensor, G: torch.Tensor | None = None,
                 loss: torch.Tensor | None = None, want_loss: bool = True):
        """G = 2 (S - y_k) and L = ||S - y_k||^2 (sbp_residual); S=None means S = 0."""
        Tk = self.Tk
        self._check_traces(y_k, Tk)
        if S is not None:
            self._check_traces(S, Tk)
        if G is None:
            G = torch.empty((self.M, Tk), dtype=torch.float32, device=self.device)
        if want_loss and loss is None:
            loss = torch.zeros(1, dtype=torch.float64, device=self.device)
        _check("sbp_residual", self._lib.sbp_residual(self._h, _dptr(S), _dptr(y_k), _dptr(G),
                                                      _dptr(loss if want_loss else None),
                                                      _stream()))
        return G, loss

    def adjoint(self, balls: torch.Tensor, G: torch.Tensor, n=None, mask: int = MASK_ALL,
                out: torch.Tensor | None = None):
        """Per-ball gradients (5, n_cap) in the order x, y, z, R, p0 (sbp_adjoint)."""
        self._check_traces(G, self.Tk)
        if out is None:
            out = torch.empty_like(balls)
        nd = self._n(n, balls.shape[1])
        _check("sbp_adjoint", self._lib.sbp_adjoint(self._h, _rows(balls), _dptr(nd),
                                                    balls.shape[1], _dptr(G), _rows(out),
                                                    mask, _stream()))
        return out

    def store_windows(self, balls: torch.Tensor, n=None, out: torch.Tensor | None = None):
        """Per-pair window records of the current level (sbp_store_windows):
        an int32 tensor (5, M, n_cap) whose planes 0-2 hold float32 bits."""
        if out is None:
            out = torch.empty((5, self.M, balls.shape[1]), dtype=torch.int32, device=balls.device)
        if out.dtype != torch.int32 or not out.is_cuda or not out.is_contiguous() or \
                tuple(out.shape) != (5, self.M, balls.shape[1]):
            raise ValueError("out must be a contiguous int32 CUDA tensor (5, M, n_cap)")
        nd = self._n(n, balls.shape[1])
        _check("sbp_store_windows", self._lib.sbp_store_windows(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], _dptr(out), _stream()))
        return out

    def adjoint_stored(self, balls: torch.Tensor, G: torch.Tensor, rec: torch.Tensor, n=None,
                       mask: int = MASK_ALL, out: torch.Tensor | None = None):
        """Per-ball gradients from stored window records (sbp_adjoint_stored)."""
        self._check_traces(G, self.Tk)
        if rec.dtype != torch.int32 or not rec.is_cuda or not rec.is_contiguous() or \
                tuple(rec.shape) != (5, self.M, balls.shape[1]):
            raise ValueError("rec must come from store_windows of this cloud")
        if out is None:
            out = torch.empty_like(balls)
        nd = self._n(n, balls.shape[1])
        _check("sbp_adjoint_stored", self._lib.sbp_adjoint_stored(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], _dptr(rec), _dptr(G), _rows(out),
            mask, _stream()))
        return out

    def filter_grow(self, balls: torch.Tensor, grads: torch.Tensor, n_dev: torch.Tensor,
                    mode: int = KEEP_NEG, grow: GrowParams | None = None, extra=()):
        """Filter/grow in place (sbp_filter_grow); n_dev is updated on the device."""
        ex = []
        for t in extra:
            if t.dim() == 2:
                ex.extend(t[k] for k in range(t.shape[0]))
            else:
                ex.append(t)
        for t in ex:
            if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() \
                    or t.numel() < balls.shape[1]:
                raise ValueError("extra arrays must be contiguous float32 CUDA tensors of n_cap")
        arr = (_P * max(1, len(ex)))(*[t.data_ptr() for t in ex])
        gp = grow.c() if grow is not None else None
        _check("sbp_filter_grow", self._lib.sbp_filter_grow(
            self._h, _rows(balls), _rows(grads), arr, len(ex), _dptr(n_dev), balls.shape[1],
            ctypes.byref(gp) if gp is not None else None, mode, _stream()))

    def adam_step(self, balls, grads, m, v, t: int, ap: AdamParams, n=None,
                  mask: int = MASK_ALL):
        nd = self._n(n, balls.shape[1])
        p = ap.c()
        _check("sbp_adam_step", self._lib.sbp_adam_step(
            self._h, _rows(balls), _rows(grads), _rows(m), _rows(v), _dptr(nd), balls.shape[1],
            int(t), ctypes.byref(p), mask, _stream()))

    def reconstruct(self, y_full: torch.Tensor, balls: torch.Tensor, n_dev: torch.Tensor,
                    stages, zero_grad_mode: int = KEEP_NEG, zero_grad_level: int = 0,
                    adam: AdamParams | None = None, grow: GrowParams | None = None,
                    loss_log: torch.Tensor | None = None, n_log: torch.Tensor | None = None,
                    spatial_sort: bool = False):
        """Algorithm 1 on the device (sbp_reconstruct): zero-gradient filtering
        then the given stages; balls and n_dev are updated in place. With
        spatial_sort the live cloud is first put in Morton order (sbp_sort_cloud)."""
        self._check_traces(y_full, self.T)
        if len(stages) > MAX_STAGES:
            raise ValueError(f"at most {MAX_STAGES} stages")
        rp = _ReconParams()
        rp.zero_grad_mode = -1 if zero_grad_mode is None else int(zero_grad_mode)
        rp.zero_grad_level = int(zero_grad_level)
        rp.n_stages = len(stages)
        for i, st in enumerate(stages):
            rp.stages[i] = _Stage(st.level, st.iterations, st.grad_mask, int(st.grow),
                                  int(st.duplicate))
        rp.adam = (adam or AdamParams()).c()
        rp.grow = (grow or GrowParams()).c()
        cap = 0
        if loss_log is not None:
            if loss_log.dtype != torch.float64 or not loss_log.is_cuda:
                raise ValueError("loss_log must be a float64 CUDA tensor")
            rp.loss_log_dev = loss_log.data_ptr()
            cap = loss_log.numel()
        if n_log is not None:
            if n_log.dtype != torch.int32 or not n_log.is_cuda:
                raise ValueError("n_log must be an int32 CUDA tensor")
            rp.n_log_dev = n_log.data_ptr()
            cap = n_log.numel() if loss_log is None else min(cap, n_log.numel())
        rp.log_capacity = cap
        rp.spatial_sort = int(bool(spatial_sort))
        _check("sbp_reconstruct", self._lib.sbp_reconstruct(
            self._h, _dptr(y_full), _rows(balls), _dptr(n_dev), balls.shape[1],
            ctypes.byref(rp), _stream()))
        if stages:
            self.level = stages[-1].level
        elif zero_grad_mode is not None and zero_grad_mode >= 0:
            self.level = zero_grad_level

    def sort_cloud(self, balls: torch.Tensor, n: torch.Tensor | None = None, extra=()):
        """Morton order of the live balls in place (sbp_sort_cloud); `extra`:
        float32 CUDA tensors of rows (k, n_cap) carried through the permutation."""
        nd = self._n(n, balls.shape[1])
        rows = []
        for e in extra:
            if e.dtype != torch.float32 or not e.is_cuda or not e.is_contiguous() or \
                    e.dim() != 2 or e.shape[1] != balls.shape[1]:
                raise ValueError("extra rows must be contiguous (k, n_cap) float32 CUDA tensors")
            rows += [e[r].data_ptr() for r in range(e.shape[0])]
        ptrs = (ctypes.c_void_p * max(1, len(rows)))(*rows)
        _check("sbp_sort_cloud", self._lib.sbp_sort_cloud(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], ptrs if rows else None, len(rows),
            _stream()))

    def forward_gauss(self, balls: torch.Tensor, n: torch.Tensor | None = None, out=None):
        """Gaussian-profile traces at the current level (sbp_forward_gauss);
        the R row of `balls` holds the standard deviation."""
        nd = self._n(n, balls.shape[1])
        if out is None:
            out = torch.empty((self.M, self.Tk), dtype=torch.float32, device=self.device)
        _check("sbp_forward_gauss", self._lib.sbp_forward_gauss(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], _dptr(out), _stream()))
        return out

    def adjoint_gauss(self, balls: torch.Tensor, G: torch.Tensor, n=None, mask: int = MASK_ALL,
                      out=None):
        """Gradients (5, n: x, y, z, a, p0) of the Gaussian-profile radiator."""
        nd = self._n(n, balls.shape[1])
        self._check_traces(G, self.Tk)
        if out is None:
            out = torch.empty_like(balls)
        _check("sbp_adjoint_gauss", self._lib.sbp_adjoint_gauss(
            self._h, _rows(balls), _dptr(nd), balls.shape[1], _dptr(G), _rows(out), mask,
            _stream()))
        return out

    def das_volume(self, y_full: torch.Tensor, origin, spacing: float, dims, out=None):
        """Delay-and-sum volume of [M][T] traces (sbp_das_volume):
        float32 [nz][ny][nx]."""
        self._check_traces(y_full, self.T)
        nx, ny, nz = (int(v) for v in dims)
        if out is None:
            out = torch.empty((nz, ny, nx), dtype=torch.float32, device=self.device)
        org = (ctypes.c_double * 3)(*[float(v) for v in origin])
        _check("sbp_das_volume", self._lib.sbp_das_volume(
            self._h, _dptr(y_full), org, float(spacing), nx, ny, nz, _dptr(out), _stream()))
        return out

    # ------------------------------------------------------------ batched frames
    def set_frames(self, capacities) -> np.ndarray:
        """Frame layout (sbp_set_frames): returns the F + 1 padded offsets of
        the frames in the packed cloud."""
        caps = np.ascontiguousarray(np.asarray(capacities, dtype=np.int32))
        off = np.zeros(caps.size + 1, dtype=np.int32)
        _check("sbp_set_frames", self._lib.sbp_set_frames(self._h, caps.ctypes.data, caps.size,
                                                          off.ctypes.data))
        self.frames = int(caps.size)
        self.frame_off = off
        return off

    def _check_frame_traces(self, t, T):
        shape = (self.frames, self.M, T)
        if t.dtype != torch.float32 or not t.is_cuda or tuple(t.shape) != shape \
                or not t.is_contiguous():
            raise ValueError(f"expected a contiguous {shape} float32 CUDA tensor")

    def set_sampling_level_frames(self, k: int, y_full=None, out=None):
        Tk = self.level_info(k)[0]
        if y_full is not None:
            self._check_frame_traces(y_full, self.T)
            if out is None:
                out = torch.empty((self.frames, self.M, Tk), dtype=torch.float32,
                                  device=self.device)
            self._check_frame_traces(out, Tk)
        _check("sbp_set_sampling_level_frames", self._lib.sbp_set_sampling_level_frames(
            self._h, k, _dptr(y_full), _dptr(out if y_full is not None else None), _stream()))
        self.level = k
        return out

    def forward_frames(self, balls, n_dev, out=None):
        Tk = self.Tk
        if out is None:
            out = torch.empty((self.frames, self.M, Tk), dtype=torch.float32, device=self.device)
        self._check_frame_traces(out, Tk)
        _check("sbp_forward_frames", self._lib.sbp_forward_frames(
            self._h, _rows(balls), _dptr(n_dev), _dptr(out), _stream()))
        return out

    def residual_frames(self, S, y_k, G=None, loss=None):
        Tk = self.Tk
        self._check_frame_traces(y_k, Tk)
        if G is None:
            G = torch.empty_like(y_k)
        _check("sbp_residual_frames", self._lib.sbp_residual_frames(
            self._h, _dptr(S), _dptr(y_k), _dptr(G), _dptr(loss), _stream()))
        return G

    def adjoint_frames(self, balls, n_dev, G, mask: int = MASK_ALL, out=None):
        self._check_frame_traces(G, self.Tk)
        if out is None:
            out = torch.empty_like(balls)
        _check("sbp_adjoint_frames", self._lib.sbp_adjoint_frames(
            self._h, _rows(balls), _dptr(n_dev), _dptr(G), _rows(out), mask, _stream()))
        return out

    def filter_grow_frames(self, balls, grads, n_dev, mode: int = KEEP_NEG,
                           grow: GrowParams | None = None, extra=()):
        ex = []
        for t in extra:
            ex.extend(t[k] for k in range(t.shape[0])) if t.dim() == 2 else ex.append(t)
        arr = (_P * max(1, len(ex)))(*[t.data_ptr() for t in ex])
        gp = grow.c() if grow is not None else None
        _check("sbp_filter_grow_frames", self._lib.sbp_filter_grow_frames(
            self._h, _rows(balls), _rows(grads), arr, len(ex), _dptr(n_dev),
            ctypes.byref(gp) if gp is not None else None, mode, _stream()))

    def adam_step_frames(self, balls, grads, m, v, n_dev, t: int, ap: AdamParams,
                         mask: int = MASK_ALL):
        p = ap.c()
        _check("sbp_adam_step_frames", self._lib.sbp_adam_step_frames(
            self._h, _rows(balls), _rows(grads), _rows(m), _rows(v), _dptr(n_dev), int(t),
            ctypes.byref(p), mask, _stream()))

    def reconstruct_frames(self, y_full, balls, n_dev, stages, zero_grad_mode: int = KEEP_NEG,
                           zero_grad_level: int = 0, adam: AdamParams | None = None,
                           grow: GrowParams | None = None, loss_log=None, n_log=None):
        """sbp_reconstruct_frames: all frames in lockstep; logs hold F entries
        per iteration."""
        self._check_frame_traces(y_full, self.T)
        rp = _ReconParams()
        rp.zero_grad_mode = -1 if zero_grad_mode is None else int(zero_grad_mode)
        rp.zero_grad_level = int(zero_grad_level)
        rp.n_stages = len(stages)
        for i, st in enumerate(stages):
            rp.stages[i] = _Stage(st.level, st.iterations, st.grad_mask, int(st.grow),
                                  int(st.duplicate))
        rp.adam = (adam or AdamParams()).c()
        rp.grow = (grow or GrowParams()).c()
        cap = 10 ** 9
        if loss_log is not None:
            rp.loss_log_dev = loss_log.data_ptr()
            cap = min(cap, loss_log.numel() // self.frames)
        if n_log is not None:
            rp.n_log_dev = n_log.data_ptr()
            cap = min(cap, n_log.numel() // self.frames)
        rp.log_capacity = cap if (loss_log is not None or n_log is not None) else 0
        _check("sbp_reconstruct_frames", self._lib.sbp_reconstruct_frames(
            self._h, _dptr(y_full), _rows(balls), _dptr(n_dev), ctypes.byref(rp), _stream()))
        if stages:
            self.level = stages[-1].level

    def set_frame_tiles(self, fwd_chunk: int = 0, adj_split: int = 0):
        """Tiles of the batched path (sbp_set_frame_tiles; 0 = default)."""
        _check("sbp_set_frame_tiles", self._lib.sbp_set_frame_tiles(self._h, fwd_chunk,
                                                                    adj_split))

    def get_frame_tiles(self):
        c, sp = ctypes.c_int(), ctypes.c_int()
        _check("sbp_get_frame_tiles", self._lib.sbp_get_frame_tiles(self._h, ctypes.byref(c),
                                                                    ctypes.byref(sp)))
        return c.value, sp.value

    def autotune_frames(self, balls, n_dev):
        """Tile autotuner of the batched path (sbp_autotune_frames); returns
        (forward balls per CTA, adjoint CTAs per ball chunk)."""
        Tk = self.Tk
        S = torch.empty((self.frames, self.M, Tk), dtype=torch.float32, device=self.device)
        G = torch.randn((self.frames, self.M, Tk), dtype=torch.float32, device=self.device)
        c, sp = ctypes.c_int(), ctypes.c_int()
        torch.cuda.synchronize()
        _check("sbp_autotune_frames", self._lib.sbp_autotune_frames(
            self._h, _rows(balls), _dptr(n_dev), _dptr(S), _dptr(G), ctypes.byref(c),
            ctypes.byref(sp)))
        return c.value, sp.value

    def sync_status(self) -> int:
        return int(self._lib.sbp_sync_status(self._h, _stream()))

    def inside_pairs(self) -> int:
        c = ctypes.c_longlong()
        _check("sbp_get_inside_pairs", self._lib.sbp_get_inside_pairs(self._h, _stream(),
                                                                       ctypes.byref(c)))
        return c.value


def forward_static(sensors: torch.Tensor, c: float, dt_us: float, T_k: int,
                   balls: torch.Tensor, n: torch.Tensor | None = None,
                   out: torch.Tensor | None = None, weight_mode: str = "clamp") -> torch.Tensor:
    """Traces S (M, T_k) without an array object (sbp_forward_static): the
    library allocates no device memory for the call (`out` is allocated here
    when not given). sensors: (6, M) float32 CUDA tensor, positions then unit
    normals; balls: (5, N); n: None (all N balls) or an int32 CUDA tensor
    holding the live count; M * T_k must stay within the library's static
    scratch (2^21 cells). Every tensor must sit on the current CUDA device."""
    if sensors.dim() != 2 or sensors.shape[0] != 6 or sensors.dtype != torch.float32 or \
            not sensors.is_cuda or not sensors.is_contiguous():
        raise ValueError("sensors must be a contiguous (6, M) float32 CUDA tensor")
    M = sensors.shape[1]
    if out is None:
        out = torch.empty((M, int(T_k)), dtype=torch.float32, device=sensors.device)
    if out.shape != (M, int(T_k)) or out.dtype != torch.float32 or not out.is_cuda or \
            not out.is_contiguous():
        raise ValueError(f"out must be a contiguous ({M}, {T_k}) float32 CUDA tensor")
    if n is not None and (n.dtype != torch.int32 or not n.is_cuda or n.numel() < 1):
        raise ValueError("n must be an int32 CUDA tensor")
    rows = _rows(balls)
    devs = {t.device for t in (sensors, balls, out) + ((n,) if n is not None else ())}
    if len(devs) != 1:
        raise ValueError("sensors, balls, out and n must be on one CUDA device")
    if sensors.device.index != torch.cuda.current_device():
        raise ValueError("the tensors must be on the current CUDA device "
                         f"(cuda:{torch.cuda.current_device()}), not {sensors.device}")
    lib = load_library()
    _check("sbp_forward_static", lib.sbp_forward_static(
        _dptr(sensors), M, float(c), float(dt_us), int(T_k), W_MODES[weight_mode], rows,
        _dptr(n), balls.shape[1], _dptr(out), _stream()))
    return out


class _Radiator(torch.autograd.Function):
    """Traces S = Simulate(balls) at one level, differentiable in every ball
    parameter. The forward saves only the cloud (the inputs); the backward
    recomputes each pair's geometry inside the adjoint kernel instead of
    storing per-pair windows."""

    @staticmethod
    def forward(ctx, x, y, z, R, p0, array, level):
        balls = torch.stack([x, y, z, R, p0]).contiguous()
        array.set_sampling_level(level)
        S = array.forward(balls)
        ctx.save_for_backward(balls)
        ctx.array, ctx.level = array, level
        return S

    @staticmethod
    def backward(ctx, gS):
        (balls,) = ctx.saved_tensors
        ctx.array.set_sampling_level(ctx.level)
        g = ctx.array.adjoint(balls, gS.contiguous(), mask=MASK_ALL)
        return g[0], g[1], g[2], g[3], g[4], None, None


def radiate(array: SensorArray, x, y, z, R, p0, level: int = 0) -> torch.Tensor:
    """Differentiable forward radiator: (M, T_k) traces of the balls with
    centres (x, y, z), radii R and pressures p0 (float32 CUDA vectors) at
    sampling level `level` of `array`."""
    return _Radiator.apply(x, y, z, R, p0, array, level)


class _RadiatorStored(torch.autograd.Function):
    """The same traces, but the forward also stores every pair's window
    record (20 bytes per pair) for the backward, which then reads them
    instead of recomputing the geometry: the stored-window alternative to
    _Radiator, kept to measure the trade."""

    @staticmethod
    def forward(ctx, x, y, z, R, p0, array, level):
        balls = torch.stack([x, y, z, R, p0]).contiguous()
        array.set_sampling_level(level)
        S = array.forward(balls)
        rec = array.store_windows(balls)
        ctx.save_for_backward(balls, rec)
        ctx.array, ctx.level = array, level
        return S

    @staticmethod
    def backward(ctx, gS):
        balls, rec = ctx.saved_tensors
        ctx.array.set_sampling_level(ctx.level)
        g = ctx.array.adjoint_stored(balls, gS.contiguous(), rec, mask=MASK_ALL)
        return g[0], g[1], g[2], g[3], g[4], None, None


def radiate_stored(array: SensorArray, x, y, z, R, p0, level: int = 0) -> torch.Tensor:
    """radiate() with stored per-pair windows instead of recomputation."""
    return _RadiatorStored.apply(x, y, z, R, p0, array, level)


# --------------------------------------------------------------------------
# envelope, initialisation and voxel grid (include/slingbag.h)
# --------------------------------------------------------------------------

class Envelope:
    """The array's envelope mesh (sbp_envelope_create): the convex hull of the
    sensor positions, with the ray-casting region test and the seeded
    initialisation of a point cloud inside it."""

    def __init__(self, pos, device=None):
        self._lib = load_library()
        if device is not None:
            torch.cuda.set_device(device)
        self.device = torch.device("cuda", torch.cuda.current_device())
        P = np.ascontiguousarray(np.asarray(pos, dtype=np.float32).reshape(-1, 3))
        h = _P()
        _check("sbp_envelope_create", self._lib.sbp_envelope_create(P.ctypes.data, P.shape[0],
                                                                    ctypes.byref(h)))
        self._h = h
        nf, vol = ctypes.c_int(), ctypes.c_double()
        box = np.zeros(6, dtype=np.float64)
        _check("sbp_envelope_info", self._lib.sbp_envelope_info(
            self._h, ctypes.byref(nf), ctypes.byref(vol), box.ctypes.data))
        self.n_faces, self.volume = nf.value, vol.value
        self.bbox = (box[:3].copy(), box[3:].copy())

    def faces(self) -> np.ndarray:
        tri = np.zeros((self.n_faces, 3), dtype=np.int32)
        _check("sbp_envelope_faces", self._lib.sbp_envelope_faces(self._h, tri.ctypes.data))
        return tri

    def classify(self, pts: torch.Tensor, inset: float = 0.0) -> torch.Tensor:
        """pts: (3, n) or (>=3, n) float32 CUDA rows x, y, z -> uint8 flags."""
        if pts.dtype != torch.float32 or not pts.is_cuda or pts.dim() != 2 or pts.shape[0] < 3 \
                or not pts.is_contiguous():
            raise ValueError("expected a contiguous (3+, n) float32 CUDA tensor")
        n = pts.shape[1]
        out = torch.empty(n, dtype=torch.uint8, device=pts.device)
        _check("sbp_envelope_classify", self._lib.sbp_envelope_classify(
            self._h, _dptr(pts[0]), _dptr(pts[1]), _dptr(pts[2]), n, float(inset), _dptr(out),
            _stream()))
        return out

    def sample(self, n_want: int, n_candidates: int, seed: int, inset: float = 0.0,
               R_range=(0.05, 0.2), p_range=(0.0, 1.0), first: int = 0, out=None, n_dev=None):
        """Seeded ray-casting initialisation (sbp_envelope_sample): returns the
        (5, cap) cloud tensor and its device count."""
        if out is None:
            out = torch.zeros((5, max(1, n_want)), dtype=torch.float32, device=self.device)
        if n_dev is None:
            n_dev = torch.zeros(1, dtype=torch.int32, device=self.device)
        if out.shape[1] < n_want:
            raise ValueError("out holds fewer than n_want balls")
        _check("sbp_envelope_sample", self._lib.sbp_envelope_sample(
            self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, int(first), int(n_candidates), float(inset),
            float(R_range[0]), float(R_range[1]), float(p_range[0]), float(p_range[1]),
            _rows(out), int(n_want), _dptr(n_dev), _stream()))
        return out, n_dev

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sbp_envelope_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def voxelize(balls: torch.Tensor, origin, spacing: float, dims, n_dev=None, values=None,
             out=None, scratch=None) -> torch.Tensor:
    """Point cloud -> voxel grid (sbp_voxelize): float32 [nz][ny][nx] of the
    summed values (default p0) of the balls containing each voxel centre."""
    lib = load_library()
    nx, ny, nz = (int(v) for v in dims)
    total = nx * ny * nz
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=balls.device)
    if scratch is None:
        scratch = torch.zeros(total + 1, dtype=torch.int64, device=balls.device)
    if scratch.numel() < total + 1 or scratch.dtype != torch.int64:
        raise ValueError("scratch needs nx*ny*nz + 1 int64 words")
    if values is not None and (values.dtype != torch.float32 or not values.is_cuda):
        raise ValueError("values must be a float32 CUDA tensor")
    org = (ctypes.c_double * 3)(*[float(v) for v in origin])
    _check("sbp_voxelize", lib.sbp_voxelize(
        _rows(balls), _dptr(values), _dptr(n_dev), balls.shape[1], org, float(spacing), nx, ny, nz,
        _dptr(scratch), _dptr(out), _stream()))
    return out


# --------------------------------------------------------------------------
# volume CNN (include/slingbag.h)
# --------------------------------------------------------------------------

def conv3d(x: torch.Tensor, dims, w: torch.Tensor, bias=None, relu: bool = False,
           out_f32: bool = False, out=None) -> torch.Tensor:
    """3x3x3 convolution on the tensor cores (sbp_conv3d_bf16). x: bf16
    (V, cin) channels-last for dims = (nx, ny, nz); w: bf16 (cout, kp)."""
    lib = load_library()
    nx, ny, nz = (int(v) for v in dims)
    V = nx * ny * nz
    if x.dtype != torch.bfloat16 or x.dim() != 2 or x.shape[0] != V or not x.is_contiguous():
        raise ValueError("x must be a contiguous (V, cin) bfloat16 tensor")
    if w.dtype != torch.bfloat16 or w.dim() != 2 or not w.is_contiguous():
        raise ValueError("w must be a contiguous (cout, kp) bfloat16 tensor")
    cin, (cout, kp) = x.shape[1], w.shape
    if out is None:
        out = torch.empty((V, cout), dtype=torch.float32 if out_f32 else torch.bfloat16,
                          device=x.device)
    if bias is not None and (bias.dtype != torch.float32 or bias.numel() != cout):
        raise ValueError("bias must be float32 with cout entries")
    _check("sbp_conv3d_bf16", lib.sbp_conv3d_bf16(
        _dptr(x), nx, ny, nz, cin, _dptr(w), kp, _dptr(bias), cout, int(relu), _dptr(out),
        int(out_f32), _stream()))
    return out


def cnn_status() -> int:
    lib = load_library()
    v = ctypes.c_int()
    _check("sbp_cnn_status", lib.sbp_cnn_status(_stream(), ctypes.byref(v)))
    return v.value


def pack_conv_weights(w: torch.Tensor) -> torch.Tensor:
    """(cout, 27, cin) float -> bf16 (cout, kp) with k = tap * cin + c, zero
    padded to kp = a multiple of 64."""
    cout, taps, cin = w.shape
    k = taps * cin
    kp = (k + 63) // 64 * 64
    out = torch.zeros((cout, kp), dtype=torch.bfloat16, device=w.device)
    out[:, :k] = w.reshape(cout, k).to(torch.bfloat16)
    return out


class VolumeCNN:
    """The learned proposal's volume CNN (sbp_cnn_*): three tcgen05 3x3x3
    convolutions with ReLU and a two-output head per voxel."""

    def __init__(self, dims, seed: int = 1):
        self._lib = load_library()
        self.dims = tuple(int(v) for v in dims)
        nx, ny, nz = self.dims
        self.V = nx * ny * nz
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = _P()
        _check("sbp_cnn_create", self._lib.sbp_cnn_create(nx, ny, nz, int(seed) & (2 ** 64 - 1),
                                                          ctypes.byref(h)))
        self._h = h
        self.n_params = int(self._lib.sbp_cnn_num_params())

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params, dtype=np.float32)
        _check("sbp_cnn_params", self._lib.sbp_cnn_params(self._h, out.ctypes.data, 0))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if p.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters")
        _check("sbp_cnn_params", self._lib.sbp_cnn_params(self._h, p.ctypes.data, 1))

    def _vol(self, vol):
        if vol.dtype != torch.float32 or not vol.is_cuda or vol.numel() != self.V \
                or not vol.is_contiguous():
            raise ValueError("volume must be a contiguous float32 CUDA tensor of nx*ny*nz")
        return _dptr(vol)

    def forward(self, vol: torch.Tensor) -> torch.Tensor:
        out = torch.empty((self.V, 2), dtype=torch.float32, device=self.device)
        _check("sbp_cnn_forward", self._lib.sbp_cnn_forward(self._h, self._vol(vol), _dptr(out),
                                                            _stream()))
        return out

    def train_step(self, vol, occ, p0, lr: float = 1e-3, pos_weight: float = 10.0, loss=None):
        for t in (occ, p0):
            if t.dtype != torch.float32 or not t.is_cuda or t.numel() != self.V:
                raise ValueError("targets must be float32 CUDA tensors of nx*ny*nz")
        _check("sbp_cnn_train_step", self._lib.sbp_cnn_train_step(
            self._h, self._vol(vol), _dptr(occ), _dptr(p0), float(pos_weight), float(lr),
            _dptr(loss), _stream()))

    def grad(self, vol, occ, p0, pos_weight: float = 10.0, loss=None) -> torch.Tensor:
        """The loss gradient with respect to every parameter (sbp_cnn_grad),
        as a float32 CUDA tensor of n_params; the parameters are unchanged."""
        for t in (occ, p0):
            if t.dtype != torch.float32 or not t.is_cuda or t.numel() != self.V:
                raise ValueError("targets must be float32 CUDA tensors of nx*ny*nz")
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.device)
        _check("sbp_cnn_grad", self._lib.sbp_cnn_grad(
            self._h, self._vol(vol), _dptr(occ), _dptr(p0), float(pos_weight), _dptr(loss),
            _dptr(out), _stream()))
        return out

    def propose(self, vol, origin, spacing: float, threshold: float = 0.5, seed: int = 1,
                R: float = 0.1, p_range=(0.05, 2.0), out=None, n_dev=None, per_voxel: int = 1):
        if out is None:
            out = torch.zeros((5, self.V * int(per_voxel)), dtype=torch.float32,
                              device=self.device)
        if n_dev is None:
            n_dev = torch.zeros(1, dtype=torch.int32, device=self.device)
        org = (ctypes.c_double * 3)(*[float(v) for v in origin])
        _check("sbp_cnn_propose", self._lib.sbp_cnn_propose(
            self._h, self._vol(vol), float(threshold), int(seed) & (2 ** 64 - 1), org,
            float(spacing), float(R), float(p_range[0]), float(p_range[1]), int(per_voxel),
            _rows(out), out.shape[1], _dptr(n_dev), _stream()))
        return out, n_dev

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sbp_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

