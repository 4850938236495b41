"""Thin Python binding of libgputb.so (include/gputb.h).

Argument marshalling only: every step of the path runs in the CUDA library.
PyTorch supplies device memory (tensors whose data pointers are passed
through) and the stream.  If the library is missing or cannot be loaded the
import fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgputb.so")

TB_OK = 0
TB_ERR_INVALID_ARG = 1
TB_ERR_CUDA = 2
TB_ERR_WORKSPACE = 3
TB_ERR_BOX = 4
TB_ERR_ELL_OVERFLOW = 5
TB_ERR_BOUNDS = 6
TB_ERR_NOT_FINITE = 7
TB_ERR_TIMEOUT = 8
TB_ERR_NOT_CONVERGED = 9

F32, F64 = 0, 1
KERNELS = {"jackson": 0, "lorentz": 1, "none": 2}

_c_i32, _c_i64, _c_u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
_c_dbl, _c_sz, _c_vp = ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p

# name -> (restype, argtypes); must match include/gputb.h
SIGNATURES = {
    "tb_abi_version": (_c_i32, []),
    "tb_last_error": (ctypes.c_char_p, []),
    "kpm_moments_workspace_size": (_c_sz, [_c_i64, _c_i32, _c_i32, _c_i32]),
    "tb_launch_count": (_c_i64, []),
    "tb_kpm_shape_count": (_c_i32, [_c_i32, _c_i32]),
    "tb_kpm_shape_info": (_c_i32, [_c_i32, _c_i32, _c_i32, _c_vp]),
    "tb_kpm_set_shape": (_c_i32, [_c_i64, _c_i32, _c_i32, _c_i32, _c_i32]),
    "tb_kpm_clear_shapes": (_c_i32, []),
    "tb_kpm_get_shape": (_c_i32, [_c_i64, _c_i32, _c_i32, _c_i32]),
    "tb_kpm_shape_grid": (_c_i32, [_c_i64, _c_i32, _c_i32, _c_i32, _c_i32]),
    "tb_kpm_autotune": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32, _c_i32, _c_i32,
                                 _c_vp, _c_sz, _c_vp, _c_vp, _c_vp, _c_i32]),
    "kpm_moments": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32, _c_i32,
                             _c_u64, _c_i64, _c_i32, _c_vp, _c_vp, _c_sz, _c_vp, ctypes.POINTER(_c_dbl)]),
    "kpm_moments_noalloc": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32,
                                     _c_i32, _c_u64, _c_vp, _c_vp]),
    "kpm_moments_batched_workspace_size": (_c_sz, [_c_i32, _c_vp, _c_vp, _c_i32, _c_i32, _c_i32, _c_vp]),
    "kpm_moments_batched": (_c_i32, [_c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp, _c_i32, _c_i32,
                                     _c_u64, _c_i32, _c_vp, _c_vp, _c_sz, _c_vp, ctypes.POINTER(_c_dbl)]),
    "kpm_moments_batched_autotune": (_c_i32, [_c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp,
                                              _c_i32, _c_i32, _c_i32, _c_vp, _c_sz, _c_vp, _c_vp, _c_vp, _c_i32]),
    "kpm_dos": (_c_i32, [_c_vp, _c_i32, _c_i32, _c_i32, _c_dbl, _c_dbl, _c_dbl, _c_vp, _c_i32, _c_vp, _c_vp]),
    "tb_mlp_set_variant": (_c_i32, [_c_i32]),
    "tb_sk_geometry": (_c_i32, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_i64, _c_vp, _c_dbl, _c_dbl,
                                _c_vp, _c_vp]),
    "tb_sk_bounds": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_sz, _c_vp]),
    "sk_kpm_workspace_size": (_c_sz, [_c_i64, _c_i32]),
    "sk_kpm_moments": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_i64, _c_vp, _c_dbl, _c_dbl, _c_i32, _c_u64, _c_i64,
                                _c_vp, _c_vp, _c_sz, _c_vp, ctypes.POINTER(_c_dbl)]),
    "tb_debug_wait_timeout": (_c_i32, [_c_i64, _c_vp, _c_sz, _c_vp]),
    "tb_velocity_values": (_c_i32, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp,
                                    _c_vp, _c_vp]),
    "lsqt_vac_workspace_size": (_c_sz, [_c_i64, _c_i32, _c_i32, _c_i32]),
    "lsqt_vac": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32, _c_i32, _c_u64,
                          _c_i64, _c_i32, _c_dbl, _c_vp, _c_vp, _c_sz, _c_vp, ctypes.POINTER(_c_dbl)]),
    "lsqt_correlation": (_c_i32, [_c_vp, _c_i32, _c_i32, _c_i32, _c_i32, _c_dbl, _c_dbl, _c_dbl, _c_vp, _c_i32,
                                  _c_dbl, _c_vp, _c_vp, _c_vp, _c_vp]),
    "tb_neighbors_workspace_size": (_c_sz, [_c_i64, _c_vp, _c_vp, _c_dbl, _c_i32]),
    "tb_build_neighbors": (_c_i32, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_i32, _c_vp, _c_vp, _c_i64,
                                    _c_vp, _c_vp, ctypes.POINTER(_c_i64), _c_vp, _c_sz, _c_vp]),
    "tb_build_hamiltonian_teacher": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                                              _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_i32, _c_vp,
                                              _c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_compute_descriptors": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_vp,
                                        _c_vp, _c_vp]),
    "tb_edge_features": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                                  _c_vp, _c_vp, _c_vp, _c_vp, _c_vp]),
    "tb_feature_stats": (_c_i32, [_c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_inverse_std": (_c_i32, [_c_vp, _c_vp, _c_vp, _c_i32, _c_vp]),
    "tb_copy_to_device": (_c_i32, [_c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_copy_to_host": (_c_i32, [_c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_mlp_workspace_size": (_c_sz, [_c_i64]),
    "tb_mlp_forward": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp]),
    "tb_mlp_backward": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_mlp_loss": (_c_i32, [_c_i64, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                             _c_sz, _c_vp]),
    "tb_adamw_step": (_c_i32, [_c_vp, _c_vp, _c_vp, _c_vp, _c_i64, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_vp,
                               _c_vp]),
    "tb_mlp_pack_weights": (_c_i32, [_c_vp, _c_vp, _c_vp]),
    "tb_build_hamiltonian_workspace_size": (_c_sz, [_c_i64, _c_i64]),
    "tb_build_hamiltonian_teacher_workspace_size": (_c_sz, [_c_i64, _c_i32]),
    "tb_build_hamiltonian": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_i64,
                                      _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp, _c_vp,
                                      _c_sz, _c_vp]),
    "tb_env_edge_inputs": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                                    _c_vp, _c_vp]),
    "tb_env_forward": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp,
                                _c_vp]),
    "tb_build_hamiltonian_env": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_vp, _c_vp, _c_vp, _c_vp,
                                          _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp, _c_vp, _c_sz, _c_vp]),
    "tb_env_set_variant": (_c_i32, [_c_i32]),
    "tb_build_hamiltonian_env_workspace_size": (_c_sz, [_c_i64]),
    "tb_env_backward_workspace_size": (_c_sz, [_c_i64, _c_i64]),
    "tb_env_backward": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                                 _c_vp, _c_sz, _c_vp]),
    "tb_bloch_bands": (_c_i32, [_c_i32, _c_i32, _c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp,
                                _c_i32, _c_vp, _c_vp, _c_vp, _c_vp]),
    "tb_band_loss": (_c_i32, [_c_i64, _c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp]),
    "tb_band_gradient": (_c_i32, [_c_i32, _c_i32, _c_i32, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_vp, _c_vp, _c_vp,
                                  _c_vp, _c_vp, _c_vp]),
    "tb_adamw_flat": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i64, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_dbl,
                               _c_vp]),
    "tb_spectral_bounds_workspace_size": (_c_sz, [_c_i64, _c_i32]),
    "tb_spectral_bounds": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_i32, _c_u64, _c_vp, _c_vp,
                                    _c_sz, _c_vp]),
}


class GputbError(RuntimeError):
    def __init__(self, func: str, status: int, message: str):
        super().__init__(f"{func} failed with status {status}: {message}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


ABI_VERSION = 9   # GPUTB_ABI_VERSION of include/gputb.h


def lib() -> ctypes.CDLL:
    """Load libgputb.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} not found; build it with paper_2509_06525_gb300.build.build()")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(handle, name)
            fn.restype = res
            fn.argtypes = args
        if handle.tb_abi_version() != ABI_VERSION:
            raise ImportError(f"{LIB_PATH} has ABI {handle.tb_abi_version()}, the binding expects {ABI_VERSION}; "
                              "rebuild it with paper_2509_06525_gb300.build.build(force=True)")
        _lib = handle
        load_tuned_shapes()
    return _lib


def _check(func: str, status: int):
    if status != TB_OK:
        msg = lib().tb_last_error().decode(errors="replace")
        raise GputbError(func, status, msg)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def precision_of(dtype) -> int:
    if dtype == torch.float32:
        return F32
    if dtype == torch.float64:
        return F64
    raise ValueError(f"unsupported value dtype {dtype}")


@dataclass
class SellMatrix:
    """A SELL-32 sparse matrix on the device (layout of include/gputb.h)."""
    n: int
    slice_ptr: torch.Tensor          # int64 [ceil(n/32) + 1]
    col: torch.Tensor                # int32 [nnz_padded]
    val: Optional[torch.Tensor]      # float32/float64 [nnz_padded]
    diag: Optional[torch.Tensor]     # same dtype [n] or None

    @property
    def precision(self) -> int:
        return precision_of(self.val.dtype)


KPM_DIRECT, KPM_DOUBLING = 0, 1


def kpm_moments(H: SellMatrix, a: float, b: float, M: int, R: int, seed: int,
                stream=None, workspace: Optional[torch.Tensor] = None, timing: Optional[list] = None,
                doubling: bool = False, first_vector: int = 0) -> torch.Tensor:
    """Per-vector KPM moments mu_r [R, M] (float64, device) of random vectors
    first_vector .. first_vector + R - 1.

    If `timing` is a list, the CUDA-event time (ms) of the Chebyshev-step
    launches is appended to it."""
    L = lib()
    prec = H.precision
    need = L.kpm_moments_workspace_size(H.n, M, R, prec)
    if need == 0:
        raise GputbError("kpm_moments_workspace_size", TB_ERR_INVALID_ARG, f"unsupported n={H.n} M={M} R={R}")
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, H.col.device)
    mu = torch.empty((R, M), dtype=torch.float64, device=H.col.device)
    step_ms = ctypes.c_double(0.0)
    st = L.kpm_moments(H.n, _ptr(H.slice_ptr), _ptr(H.col), _ptr(H.val), _ptr(H.diag), prec,
                       float(a), float(b), int(M), int(R), int(seed) & ((1 << 64) - 1), int(first_vector),
                       KPM_DOUBLING if doubling else KPM_DIRECT, _ptr(mu), _ptr(ws), ws.numel(), _stream(stream),
                       ctypes.byref(step_ms) if timing is not None else None)
    _check("kpm_moments", st)
    if timing is not None:
        timing.append(step_ms.value)
    return mu


class _BatchArgs:
    """Marshalled host arrays of a batch of SELL matrices (kept alive with
    the call)."""

    def __init__(self, mats, a, b):
        import numpy as np
        self.S = len(mats)
        self.prec = mats[0].precision
        if any(m.precision != self.prec for m in mats):
            raise ValueError("all snapshots must share one precision")
        self.rows = np.array([m.n for m in mats], np.int64)
        self.aa = np.ascontiguousarray(np.asarray(a, np.float64))
        self.bb = np.ascontiguousarray(np.asarray(b, np.float64))
        arr = lambda ts: (ctypes.c_void_p * self.S)(*[(t.data_ptr() if t is not None else None) for t in ts])
        self.sp, self.col = arr([m.slice_ptr for m in mats]), arr([m.col for m in mats])
        self.val, self.dg = arr([m.val for m in mats]), arr([m.diag for m in mats])
        self.dev = mats[0].col.device

    def ptrs(self):
        c = lambda x: ctypes.cast(x, ctypes.c_void_p)
        return (self.S, self.rows.ctypes.data_as(ctypes.c_void_p), c(self.sp), c(self.col), c(self.val), c(self.dg),
                self.prec, self.aa.ctypes.data_as(ctypes.c_void_p), self.bb.ctypes.data_as(ctypes.c_void_p))


_BATCH_WS = {}


def _batch_workspace(args: "_BatchArgs", M: int, R: int, stream=None) -> torch.Tensor:
    """A workspace for the batch, reused across calls of the same size so
    that the library's cached graph (keyed by the workspace) stays valid."""
    L = lib()
    need = L.kpm_moments_batched_workspace_size(args.S, ctypes.cast(args.sp, ctypes.c_void_p),
                                                args.rows.ctypes.data_as(ctypes.c_void_p), M, R, args.prec,
                                                _stream(stream))
    if need == 0:
        raise GputbError("kpm_moments_batched_workspace_size", TB_ERR_INVALID_ARG, f"unsupported R={R} M={M}")
    ws = _BATCH_WS.get(args.dev)
    if ws is None or ws.numel() < need:
        ws = _workspace(need, args.dev)
        _BATCH_WS[args.dev] = ws
    return ws


def kpm_moments_batched_autotune(mats, a, b, R: int, doubling: bool = False, reps: int = 20, stream=None):
    """Time every step shape on the folded batch; the fastest becomes the
    table entry of the batch's padded size.  Returns (best, [ms per step])."""
    args = _BatchArgs(mats, a, b)
    ws = _batch_workspace(args, 2, R, stream)
    count = kpm_shape_count(R, args.prec)
    ms = (ctypes.c_float * count)()
    best = _c_i32(-1)
    st = lib().kpm_moments_batched_autotune(*args.ptrs(), int(R), KPM_DOUBLING if doubling else KPM_DIRECT,
                                            int(reps), _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(best),
                                            ms, count)
    _check("kpm_moments_batched_autotune", st)
    return int(best.value), [float(v) for v in ms]


def kpm_moments_batched(mats, a, b, M: int, R: int, seed: int, doubling: bool = False, stream=None,
                        timing: Optional[list] = None, mu: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Moments of every snapshot in one graph launch: mu [S, R, M] (float64,
    device).  Snapshot s uses seed + s.  Pass the previous call's `mu` to
    reuse the library's cached graph of an identical call."""
    args = _BatchArgs(mats, a, b)
    ws = _batch_workspace(args, M, R, stream)
    if mu is None or mu.shape != (args.S, R, M):
        mu = torch.empty((args.S, R, M), dtype=torch.float64, device=args.dev)
    ms = ctypes.c_double(0.0)
    st = lib().kpm_moments_batched(*args.ptrs(), int(M), int(R), int(seed) & ((1 << 64) - 1),
                                   KPM_DOUBLING if doubling else KPM_DIRECT, _ptr(mu), _ptr(ws), ws.numel(),
                                   _stream(stream), ctypes.byref(ms) if timing is not None else None)
    _check("kpm_moments_batched", st)
    if timing is not None:
        timing.append(ms.value)
    return mu


class StepShape(ctypes.Structure):
    """tb_step_shape of include/gputb.h."""
    _fields_ = [("pipelined", _c_i32), ("complex_per_thread", _c_i32), ("stages", _c_i32),
                ("min_blocks", _c_i32), ("rows_per_tile", _c_i32), ("rows_per_thread", _c_i32),
                ("staged_vectors", _c_i32), ("options", _c_i32), ("band_rows", _c_i32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def _prec(dtype_or_prec) -> int:
    return dtype_or_prec if isinstance(dtype_or_prec, int) else precision_of(dtype_or_prec)


def kpm_shape_count(R: int, dtype) -> int:
    """Number of compiled Chebyshev-step shapes for (R, precision)."""
    return int(lib().tb_kpm_shape_count(int(R), _prec(dtype)))


def kpm_shape_info(R: int, dtype, shape: int) -> dict:
    out = StepShape()
    _check("tb_kpm_shape_info", lib().tb_kpm_shape_info(int(R), _prec(dtype), int(shape), ctypes.byref(out)))
    return out.as_dict()


def kpm_set_shape(n: int, R: int, dtype, mode: int, shape: int):
    """Table entry of n's size class (n > 0) or the forced entry (n = 0);
    mode 0 (direct), 1 (doubling) or -1 (both); shape -1 removes it."""
    _check("tb_kpm_set_shape", lib().tb_kpm_set_shape(int(n), int(R), _prec(dtype), int(mode), int(shape)))


def kpm_force_shape(R: int, dtype, shape: int):
    """Every call with (R, precision) uses `shape` (-1 lifts the override)."""
    kpm_set_shape(0, R, dtype, -1, shape)


def kpm_clear_shapes():
    _check("tb_kpm_clear_shapes", lib().tb_kpm_clear_shapes())


def kpm_get_shape(n: int, R: int, dtype, doubling: bool = False) -> int:
    return int(lib().tb_kpm_get_shape(int(n), int(R), _prec(dtype), KPM_DOUBLING if doubling else KPM_DIRECT))


def kpm_shape_grid(n: int, R: int, dtype, doubling: bool, shape: int) -> int:
    """CTAs of one step launch of `shape` over n rows (needs the GPU)."""
    g = int(lib().tb_kpm_shape_grid(int(n), int(R), _prec(dtype), KPM_DOUBLING if doubling else KPM_DIRECT,
                                    int(shape)))
    if g < 1:
        raise GputbError("tb_kpm_shape_grid", TB_ERR_INVALID_ARG, f"no grid for n={n} R={R} shape={shape}")
    return g


def kpm_autotune(H: SellMatrix, a: float, b: float, R: int, doubling: bool = False, reps: int = 20, stream=None,
                 record: bool = True):
    """Time every step shape of (R, H's precision) on H (tb_kpm_autotune);
    the fastest becomes the table entry of H.n's size class.  Returns
    (best shape, [ms per step of each shape]).  With `record`, the choice is
    also written to the tuning cache file (see tuned_shapes_path)."""
    L = lib()
    prec = H.precision
    count = kpm_shape_count(R, prec)
    if count == 0:
        raise GputbError("tb_kpm_autotune", TB_ERR_INVALID_ARG, f"unsupported R={R}")
    need = L.kpm_moments_workspace_size(H.n, 2, R, prec)
    ws = _workspace(need, H.col.device)
    ms = (ctypes.c_float * count)()
    best = _c_i32(-1)
    mode = KPM_DOUBLING if doubling else KPM_DIRECT
    st = L.tb_kpm_autotune(H.n, _ptr(H.slice_ptr), _ptr(H.col), _ptr(H.val), _ptr(H.diag), prec, float(a), float(b),
                           int(R), mode, int(reps), _ptr(ws), ws.numel(), _stream(stream), ctypes.byref(best), ms,
                           count)
    _check("tb_kpm_autotune", st)
    times = [float(v) for v in ms]
    if record:
        _record_tuned(H.n, R, prec, mode, int(best.value))
    return int(best.value), times


def tuned_shapes_path() -> str:
    """JSON cache of autotuned shapes: $GPUTB_TUNE_CACHE, else
    tuned_shapes.json beside the library."""
    return os.environ.get("GPUTB_TUNE_CACHE") or os.path.join(_HERE, "tuned_shapes.json")


def _gpu_name() -> str:
    return torch.cuda.get_device_name(torch.cuda.current_device()) if torch.cuda.is_available() else "none"


def _size_class(n: int) -> int:
    return max(int(n), 1).bit_length() - 1


def _record_tuned(n: int, R: int, prec: int, mode: int, shape: int):
    import json
    path = tuned_shapes_path()
    try:
        with open(path) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        data = {}
    entries = data.setdefault(_gpu_name(), {})
    key = f"p{prec}-R{R}-m{mode}-c{_size_class(n)}"
    entries[key] = {"precision": prec, "R": int(R), "mode": int(mode), "n": int(n), "shape": int(shape),
                    "desc": kpm_shape_info(R, prec, shape)}
    # a private temporary file and an atomic rename: ranks that tune at the
    # same time each leave a whole file (the last one wins); the cache is
    # best-effort, so a failed write is not an error
    tmp = f"{path}.{os.getpid()}.tmp"
    try:
        with open(tmp, "w") as fh:
            json.dump(data, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        try:
            os.remove(tmp)
        except OSError:
            pass


def load_tuned_shapes(path: Optional[str] = None) -> int:
    """Apply the cached entries of this GPU model whose shape description
    still matches the built library; returns how many were applied."""
    import json
    try:
        with open(path or tuned_shapes_path()) as fh:
            data = json.load(fh)
    except (OSError, ValueError):
        return 0
    applied = 0
    for e in data.get(_gpu_name(), {}).values():
        try:
            if kpm_shape_info(e["R"], e["precision"], e["shape"]) != e["desc"]:
                continue
            kpm_set_shape(e["n"], e["R"], e["precision"], e["mode"], e["shape"])
            applied += 1
        except (GputbError, KeyError, TypeError):
            continue
    return applied


def kpm_dos(mu_r: torch.Tensor, a: float, b: float, energy: torch.Tensor, kernel: str = "jackson",
            lam: float = 4.0, stream=None) -> torch.Tensor:
    """DOS per orbital per eV on `energy` (float64 device) from mu_r [R, M]."""
    L = lib()
    R, M = mu_r.shape
    out = torch.empty_like(energy, dtype=torch.float64)
    st = L.kpm_dos(_ptr(mu_r), R, M, KERNELS[kernel], float(lam), float(a), float(b), _ptr(energy),
                   energy.numel(), _ptr(out), _stream(stream))
    _check("kpm_dos", st)
    return out


# ------------------------------------------------------------------ s, p, d Slater-Koster model

def sk_geometry(positions: torch.Tensor, box, pbc, nb: "Neighbors", sk, stream=None) -> torch.Tensor:
    """tb_sk_geometry: [13, total] float32 planes (l, m, n, V_0..V_9)."""
    import numpy as np
    L = lib()
    b, p, bptr, pptr = _host_box(box, pbc)
    v0 = np.ascontiguousarray(np.asarray(sk.v0, np.float64).reshape(10))
    geom = torch.empty((13, max(nb.total, 1)), dtype=torch.float32, device=positions.device)
    st = L.tb_sk_geometry(_ptr(positions), nb.n, bptr, pptr, float(sk.rcut), _ptr(nb.slice_ptr), _ptr(nb.col),
                          nb.total, v0.ctypes.data_as(ctypes.c_void_p), float(sk.a_cc), float(sk.beta), _ptr(geom),
                          _stream(stream))
    _check("tb_sk_geometry", st)
    return geom


def sk_bounds(nb: "Neighbors", geom: torch.Tensor, sk, stream=None):
    """(E_min, E_max, a, b) from the Gershgorin row sums of the SK blocks."""
    import numpy as np
    L = lib()
    on = np.ascontiguousarray(np.asarray(sk.onsite, np.float64).reshape(3))
    ws = _workspace(L.sk_kpm_workspace_size(nb.n, 2), geom.device)
    out = np.zeros(4, np.float64)
    st = L.tb_sk_bounds(nb.n, _ptr(nb.slice_ptr), _ptr(nb.col), _ptr(geom), nb.total,
                        on.ctypes.data_as(ctypes.c_void_p), out.ctypes.data_as(ctypes.c_void_p), _ptr(ws),
                        ws.numel(), _stream(stream))
    _check("tb_sk_bounds", st)
    return tuple(float(v) for v in out)


def sk_kpm_moments(nb: "Neighbors", geom: torch.Tensor, sk, a: float, b: float, M: int, seed: int,
                   first_vector: int = 0, stream=None, timing: Optional[list] = None) -> torch.Tensor:
    """KPM moments [M] of the 9N-orbital SK Hamiltonian for one random vector."""
    import numpy as np
    L = lib()
    on = np.ascontiguousarray(np.asarray(sk.onsite, np.float64).reshape(3))
    ws = _workspace(L.sk_kpm_workspace_size(nb.n, M), geom.device)
    mu = torch.empty(M, dtype=torch.float64, device=geom.device)
    ms = ctypes.c_double(0.0)
    st = L.sk_kpm_moments(nb.n, _ptr(nb.slice_ptr), _ptr(nb.col), _ptr(geom), nb.total,
                          on.ctypes.data_as(ctypes.c_void_p), float(a), float(b), int(M),
                          int(seed) & ((1 << 64) - 1), int(first_vector), _ptr(mu), _ptr(ws), ws.numel(),
                          _stream(stream), ctypes.byref(ms) if timing is not None else None)
    _check("sk_kpm_moments", st)
    if timing is not None:
        timing.append(ms.value)
    return mu


def mlp_set_variant(variant: int):
    """Forward kernel of build_hamiltonian: 0 = tcgen05 (TMEM), 1 = mma.sync."""
    _check("tb_mlp_set_variant", lib().tb_mlp_set_variant(int(variant)))


def debug_wait_timeout(polls: int, stream=None):
    """Test hook: a bounded wait on an mbarrier phase that nothing completes;
    raises GputbError(TB_ERR_TIMEOUT) when it gives up."""
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    _check("tb_debug_wait_timeout", lib().tb_debug_wait_timeout(int(polls), _ptr(ws), 256, _stream(stream)))


# ------------------------------------------------------------------ conductivity (Eq. 3 (sigma))

HBAR_EV_FS = 0.6582119569


def velocity_values(positions: torch.Tensor, box, pbc, rcut: float, H: SellMatrix, direction=(1.0, 0.0, 0.0),
                    stream=None) -> torch.Tensor:
    """tb_velocity_values: SELL values H_ij (d_ij . e) of V / (i / hbar)."""
    import numpy as np
    L = lib()
    b, p, bptr, pptr = _host_box(box, pbc)
    e = np.ascontiguousarray(np.asarray(direction, np.float64).reshape(3))
    vval = torch.empty_like(H.val)
    st = L.tb_velocity_values(_ptr(positions), H.n, bptr, pptr, float(rcut), _ptr(H.slice_ptr), _ptr(H.col),
                              _ptr(H.val), H.precision, e.ctypes.data_as(ctypes.c_void_p), _ptr(vval),
                              _stream(stream))
    _check("tb_velocity_values", st)
    return vval


def lsqt_vac(H: SellMatrix, vval: torch.Tensor, a: float, b: float, M: int, R: int, seed: int, n_steps: int,
             dt: float, first_vector: int = 0, stream=None, timing: Optional[list] = None) -> torch.Tensor:
    """Per-vector VAC moments [n_steps + 1, R, M] (float64, device, A^2/fs^2)."""
    L = lib()
    need = L.lsqt_vac_workspace_size(H.n, M, R, H.precision)
    if need == 0:
        raise GputbError("lsqt_vac_workspace_size", TB_ERR_INVALID_ARG, f"unsupported n={H.n} M={M} R={R}")
    ws = _workspace(need, H.col.device)
    mu = torch.empty((n_steps + 1, R, M), dtype=torch.float64, device=H.col.device)
    ms = ctypes.c_double(0.0)
    st = L.lsqt_vac(H.n, _ptr(H.slice_ptr), _ptr(H.col), _ptr(H.val), _ptr(H.diag), _ptr(vval), H.precision,
                    float(a), float(b), int(M), int(R), int(seed) & ((1 << 64) - 1), int(first_vector), int(n_steps),
                    float(dt), _ptr(mu), _ptr(ws), ws.numel(), _stream(stream),
                    ctypes.byref(ms) if timing is not None else None)
    _check("lsqt_vac", st)
    if timing is not None:
        timing.append(ms.value)
    return mu


def lsqt_correlation(mu: torch.Tensor, a: float, b: float, energy: torch.Tensor, dt: float,
                     kernel: str = "jackson", lam: float = 4.0, stream=None):
    """(C [n_times, K], S [n_times, K]): per-orbital velocity correlation and
    its running time integral on `energy` from lsqt_vac moments."""
    L = lib()
    mu = mu.contiguous()
    n_t, R, M = mu.shape
    K = energy.numel()
    corr = torch.empty((n_t, K), dtype=torch.float64, device=mu.device)
    sig = torch.empty((n_t, K), dtype=torch.float64, device=mu.device)
    coef = torch.empty((n_t * M,), dtype=torch.float64, device=mu.device)
    st = L.lsqt_correlation(_ptr(mu), n_t, R, M, KERNELS[kernel], float(lam), float(a), float(b),
                            _ptr(energy), K, float(dt), _ptr(corr), _ptr(sig), _ptr(coef), _stream(stream))
    _check("lsqt_correlation", st)
    return corr, sig


def _host_box(box, pbc):
    import numpy as np
    b = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(9))
    p = np.ascontiguousarray(np.asarray(pbc, dtype=np.int32).reshape(3))
    return b, p, b.ctypes.data_as(ctypes.c_void_p), p.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Neighbors:
    """SELL-32 neighbour structure on the device (the Hamiltonian's pattern)."""
    n: int
    slice_ptr: torch.Tensor      # int64 [ceil(n/32)+1]
    col: torch.Tensor            # int32 [total]
    cnt: torch.Tensor            # int32 [n]
    ncount: Optional[torch.Tensor]
    total: int


def build_neighbors(positions: torch.Tensor, box, pbc, rcut: float, r_count: float = 1.8,
                    max_width: int = 16, stream=None) -> Neighbors:
    """tb_build_neighbors for device positions [N, 3] float64."""
    L = lib()
    n = positions.shape[0]
    dev = positions.device
    b, p, bptr, pptr = _host_box(box, pbc)
    need = L.tb_neighbors_workspace_size(n, bptr, pptr, float(rcut), int(max_width))
    if need == 0:
        raise GputbError("tb_neighbors_workspace_size", TB_ERR_BOX, lib().tb_last_error().decode())
    ws = _workspace(need, dev)
    n_slices = (n + 31) // 32
    slice_ptr = torch.empty(n_slices + 1, dtype=torch.int64, device=dev)
    cap = n_slices * 32 * max_width
    col = torch.empty(cap, dtype=torch.int32, device=dev)
    cnt = torch.empty(n, dtype=torch.int32, device=dev)
    ncount = torch.empty(n, dtype=torch.int32, device=dev) if r_count > 0 else None
    total = ctypes.c_int64(0)
    st = L.tb_build_neighbors(_ptr(positions), n, bptr, pptr, float(rcut), float(r_count), int(max_width),
                              _ptr(slice_ptr), _ptr(col), cap, _ptr(cnt), _ptr(ncount), ctypes.byref(total),
                              _ptr(ws), ws.numel(), _stream(stream))
    _check("tb_build_neighbors", st)
    return Neighbors(n, slice_ptr, col[:total.value], cnt, ncount, total.value)


def build_hamiltonian_teacher(positions: torch.Tensor, species: torch.Tensor, box, pbc, nb: Neighbors,
                              teacher, dtype=torch.float64, with_diag: bool = True, stream=None) -> SellMatrix:
    """tb_build_hamiltonian_teacher: teacher values in the SELL-32 pattern of nb."""
    import numpy as np
    L = lib()
    dev = positions.device
    b, p, bptr, pptr = _host_box(box, pbc)
    pref = np.ascontiguousarray(np.asarray(teacher.hop_prefactor, np.float64).reshape(9))
    onsite = np.ascontiguousarray(np.asarray(teacher.onsite, np.float64).reshape(3))
    val = torch.empty(max(nb.total, 1), dtype=dtype, device=dev)
    diag = torch.empty(nb.n, dtype=dtype, device=dev) if with_diag else None
    ws = _workspace(L.tb_build_hamiltonian_teacher_workspace_size(nb.n, precision_of(dtype)), dev)
    st = L.tb_build_hamiltonian_teacher(
        _ptr(positions), _ptr(species), nb.n, bptr, pptr, _ptr(nb.slice_ptr), _ptr(nb.col), _ptr(nb.cnt),
        _ptr(nb.ncount), pref.ctypes.data_as(ctypes.c_void_p), onsite.ctypes.data_as(ctypes.c_void_p),
        float(teacher.a_cc), float(teacher.beta), float(teacher.gamma), float(teacher.rcut), precision_of(dtype),
        _ptr(val), _ptr(diag), _ptr(ws), ws.numel(), _stream(stream))
    _check("tb_build_hamiltonian_teacher", st)
    return SellMatrix(nb.n, nb.slice_ptr, nb.col, val[:nb.total], diag)


@dataclass
class Bounds:
    emin: float
    emax: float
    a: float
    b: float
    theta_min: float
    theta_max: float
    g_min: float
    g_max: float


def spectral_bounds(H: SellMatrix, lanczos_steps: int = 64, seed: int = 7, stream=None) -> Bounds:
    import numpy as np
    L = lib()
    need = L.tb_spectral_bounds_workspace_size(H.n, lanczos_steps)
    ws = _workspace(need, H.col.device)
    out = np.zeros(8, np.float64)
    st = L.tb_spectral_bounds(H.n, _ptr(H.slice_ptr), _ptr(H.col), _ptr(H.val), _ptr(H.diag), H.precision,
                              int(lanczos_steps), int(seed), out.ctypes.data_as(ctypes.c_void_p), _ptr(ws),
                              ws.numel(), _stream(stream))
    _check("tb_spectral_bounds", st)
    return Bounds(*[float(v) for v in out])


# ------------------------------------------------------------------ learned path

N_PARAM = 6402
N_WBF16 = 6272
PARAM_OFFSETS = {"W1": (0, (64, 32)), "b1": (2048, (64,)), "W2": (2112, (64, 64)), "b2": (6208, (64,)),
                 "W3": (6272, (2, 64)), "b3": (6400, (2,))}


def pack_params(params: dict) -> "np.ndarray":
    """Flatten {W1, b1, W2, b2, W3, b3} into the library's FP32 parameter vector."""
    import numpy as np
    flat = np.zeros(N_PARAM, np.float32)
    for k, (off, shape) in PARAM_OFFSETS.items():
        flat[off:off + int(np.prod(shape))] = np.asarray(params[k], np.float32).reshape(-1)
    return flat


def unpack_params(flat) -> dict:
    import numpy as np
    flat = np.asarray(flat)
    return {k: flat[off:off + int(np.prod(shape))].reshape(shape).copy() for k, (off, shape) in PARAM_OFFSETS.items()}


class MLPModel:
    """Device state of the learned model: FP32 parameters, their BF16 weight
    copy, AdamW moments, frozen input normalisation and the descriptor
    mixing matrices."""

    def __init__(self, params: dict, cmix, eps0, mean=None, std=None, device="cuda", stream=None):
        import numpy as np
        self.p = torch.tensor(pack_params(params), device=device)
        self.wb = torch.empty(N_WBF16, dtype=torch.bfloat16, device=device)
        self.m = torch.zeros(N_PARAM, dtype=torch.float32, device=device)
        self.v = torch.zeros(N_PARAM, dtype=torch.float32, device=device)
        self.cmix = torch.tensor(np.asarray(cmix, np.float32).reshape(-1), device=device)
        self.eps0 = torch.tensor(np.asarray(eps0, np.float32), device=device)
        self.mean = None if mean is None else torch.as_tensor(mean, dtype=torch.float32, device=device)
        self.inv_std = None
        if std is not None:
            self.inv_std = inverse_std(torch.as_tensor(std, dtype=torch.float32, device=device), stream=stream)
        self.step = 0
        _check("tb_mlp_pack_weights", lib().tb_mlp_pack_weights(_ptr(self.p), _ptr(self.wb), _stream(stream)))

    def set_normalisation(self, mean: torch.Tensor, std: torch.Tensor, mask: Optional[torch.Tensor] = None):
        self.mean = mean.to(torch.float32).contiguous()
        self.inv_std = inverse_std(std.to(torch.float32).contiguous(), mask)

    def params_numpy(self) -> dict:
        return unpack_params(self.p.cpu().numpy())


def compute_descriptors(positions, species, box, pbc, rcut, nb: Neighbors, cmix: torch.Tensor,
                        stream=None) -> torch.Tensor:
    b, p, bptr, pptr = _host_box(box, pbc)
    v = torch.empty((nb.n, 8), dtype=torch.float32, device=positions.device)
    st = lib().tb_compute_descriptors(_ptr(positions), _ptr(species), nb.n, bptr, pptr, float(rcut),
                                      _ptr(nb.slice_ptr), _ptr(nb.col), _ptr(nb.cnt), _ptr(cmix), _ptr(v),
                                      _stream(stream))
    _check("tb_compute_descriptors", st)
    return v


def edge_features(positions, species, box, pbc, rcut, nb: Neighbors, cmix, v, mean=None, inv_std=None,
                  raw=True, bf16=True, stream=None):
    b, p, bptr, pptr = _host_box(box, pbc)
    dev = positions.device
    xr = torch.empty((max(nb.total, 1), 32), dtype=torch.float32, device=dev) if raw else None
    xb = torch.empty((max(nb.total, 1), 32), dtype=torch.bfloat16, device=dev) if bf16 else None
    st = lib().tb_edge_features(_ptr(positions), _ptr(species), nb.n, bptr, pptr, float(rcut), _ptr(nb.slice_ptr),
                                _ptr(nb.col), _ptr(nb.cnt), _ptr(cmix), _ptr(v), _ptr(mean), _ptr(inv_std),
                                _ptr(xr), _ptr(xb), _stream(stream))
    _check("tb_edge_features", st)
    return (xr[:nb.total] if raw else None), (xb[:nb.total] if bf16 else None)


def feature_stats(x_raw, n, slice_ptr, cnt, mask: Optional[torch.Tensor] = None, stream=None):
    """(mean, std, inv_std) of the edge inputs (tb_feature_stats); mask
    (float [32]) switches features off in inv_std."""
    dev = x_raw.device
    mean = torch.empty(32, dtype=torch.float32, device=dev)
    std = torch.empty(32, dtype=torch.float32, device=dev)
    inv = torch.empty(32, dtype=torch.float32, device=dev)
    m = None if mask is None else torch.as_tensor(mask, dtype=torch.float32, device=dev).contiguous()
    ws = _workspace(96 * 8 * 8 * 1024, dev)
    st = lib().tb_feature_stats(_ptr(x_raw), n, _ptr(slice_ptr), _ptr(cnt), _ptr(mean), _ptr(std), _ptr(inv),
                                _ptr(m), _ptr(ws), ws.numel(), _stream(stream))
    _check("tb_feature_stats", st)
    return mean, std, inv


def inverse_std(std: torch.Tensor, mask: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """tb_inverse_std: mask / max(std, 1e-6) on the device."""
    out = torch.empty_like(std)
    m = None if mask is None else torch.as_tensor(mask, dtype=torch.float32, device=std.device).contiguous()
    _check("tb_inverse_std", lib().tb_inverse_std(_ptr(std), _ptr(m), _ptr(out), std.numel(), _stream(stream)))
    return out


def copy_to_device(dst: torch.Tensor, src_host: torch.Tensor, stream=None):
    """tb_copy_to_device: a host tensor (page-locked for an asynchronous
    transfer) into a device tensor of the same size."""
    if src_host.is_cuda or not dst.is_cuda or dst.numel() * dst.element_size() != src_host.numel() * src_host.element_size():
        raise ValueError("copy_to_device: host source and device destination of equal size")
    _check("tb_copy_to_device", lib().tb_copy_to_device(_ptr(dst), ctypes.c_void_p(src_host.data_ptr()),
                                                        dst.numel() * dst.element_size(), _stream(stream)))
    return dst


def copy_to_host(dst_host: torch.Tensor, src: torch.Tensor, stream=None):
    """tb_copy_to_host: a device tensor into a host tensor (synchronises)."""
    if dst_host.is_cuda or not src.is_cuda or dst_host.numel() * dst_host.element_size() != src.numel() * src.element_size():
        raise ValueError("copy_to_host: device source and host destination of equal size")
    if not src.is_contiguous() or not dst_host.is_contiguous():
        raise ValueError("copy_to_host: contiguous tensors only")
    _check("tb_copy_to_host", lib().tb_copy_to_host(ctypes.c_void_p(dst_host.data_ptr()), _ptr(src),
                                                    src.numel() * src.element_size(), _stream(stream)))
    return dst_host


def mlp_forward(x_bf16, model: MLPModel, stream=None):
    E = x_bf16.shape[0]
    y = torch.empty((E, 2), dtype=torch.float32, device=x_bf16.device)
    st = lib().tb_mlp_forward(E, _ptr(x_bf16), _ptr(model.wb), _ptr(model.p), _ptr(y), _stream(stream))
    _check("tb_mlp_forward", st)
    return y


def mlp_backward(x_bf16, model: MLPModel, dy, stream=None, workspace=None):
    E = x_bf16.shape[0]
    need = lib().tb_mlp_workspace_size(E)
    ws = workspace if workspace is not None and workspace.numel() >= need else _workspace(need, x_bf16.device)
    grad = torch.empty(N_PARAM, dtype=torch.float32, device=x_bf16.device)
    st = lib().tb_mlp_backward(E, _ptr(x_bf16), _ptr(model.wb), _ptr(model.p), _ptr(dy), _ptr(grad), _ptr(ws),
                               ws.numel(), _stream(stream))
    _check("tb_mlp_backward", st)
    return grad


def mlp_loss(row_begin, row_end, slice_ptr, cnt, y, t_hop, eps_target, species, eps0, dy, stream=None):
    """Fills dy for the rows' elements; returns stats (device double[4])."""
    stats = torch.empty(4, dtype=torch.float64, device=y.device)
    ws = _workspace(3 * 8 * 2 * 1024, y.device)
    st = lib().tb_mlp_loss(int(row_begin), int(row_end), _ptr(slice_ptr), _ptr(cnt), _ptr(y), _ptr(t_hop),
                           _ptr(eps_target), _ptr(species), _ptr(eps0), _ptr(dy), _ptr(stats), _ptr(ws),
                           ws.numel(), _stream(stream))
    _check("tb_mlp_loss", st)
    return stats


def adamw_step(model: MLPModel, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    model.step += 1
    st = lib().tb_adamw_step(_ptr(model.p), _ptr(grad), _ptr(model.m), _ptr(model.v), model.step, float(lr),
                             float(beta1), float(beta2), float(eps), float(weight_decay), _ptr(model.wb),
                             _stream(stream))
    _check("tb_adamw_step", st)


def build_hamiltonian(positions, species, box, pbc, rcut, nb: Neighbors, model: MLPModel, v=None,
                      dtype=torch.float32, with_diag=True, stream=None) -> SellMatrix:
    """Learned H (tb_build_hamiltonian) in the SELL-32 pattern of nb."""
    L = lib()
    dev = positions.device
    if v is None:
        v = compute_descriptors(positions, species, box, pbc, rcut, nb, model.cmix, stream)
    b, p, bptr, pptr = _host_box(box, pbc)
    val = torch.empty(max(nb.total, 1), dtype=dtype, device=dev)
    diag = torch.empty(nb.n, dtype=dtype, device=dev) if with_diag else None
    ws = _workspace(L.tb_build_hamiltonian_workspace_size(nb.n, nb.total), dev)
    st = L.tb_build_hamiltonian(_ptr(positions), _ptr(species), nb.n, bptr, pptr, float(rcut), _ptr(nb.slice_ptr),
                                _ptr(nb.col), _ptr(nb.cnt), nb.total, _ptr(model.cmix), _ptr(v), _ptr(model.mean),
                                _ptr(model.inv_std), _ptr(model.wb), _ptr(model.p), _ptr(model.eps0),
                                precision_of(dtype), _ptr(val), _ptr(diag), _ptr(ws), ws.numel(), _stream(stream))
    _check("tb_build_hamiltonian", st)
    return SellMatrix(nb.n, nb.slice_ptr, nb.col, val[:nb.total], diag)


# ---------------------------------------------------------------- environment network and bands

ENV_NPARAM = 2349    # TB_ENV_NPARAM
ENV_NFEAT = 20       # TB_ENV_NFEAT


class EnvModel:
    """Device state of the environment-network model: the flat FP32
    parameter vector (layout of include/gputb.h), its AdamW moments, the
    species-pair mixing c^{Z_i Z_j} and the reference onsite energies."""

    def __init__(self, params, cmix, eps0, device="cuda"):
        import numpy as np
        flat = np.asarray(params, np.float32).reshape(-1)
        if flat.size != ENV_NPARAM:
            raise ValueError(f"expected {ENV_NPARAM} parameters, got {flat.size}")
        c = np.asarray(cmix, np.float32).reshape(3, 3, 8, 8)
        if not np.array_equal(c, c.transpose(1, 0, 2, 3)):
            raise ValueError("the environment model needs a mixing symmetric in the species pair")
        self.p = torch.tensor(flat, device=device)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.cmix = torch.tensor(c.reshape(-1), device=device)
        self.eps0 = torch.tensor(np.asarray(eps0, np.float32), device=device)
        self.step = 0


def env_edge_inputs(positions, species, box, pbc, rcut, nb: Neighbors, cmix, v, stream=None) -> torch.Tensor:
    b, p, bptr, pptr = _host_box(box, pbc)
    feat = torch.zeros((max(nb.total, 1), ENV_NFEAT), dtype=torch.float32, device=positions.device)
    _check("tb_env_edge_inputs", lib().tb_env_edge_inputs(
        _ptr(positions), _ptr(species), nb.n, bptr, pptr, float(rcut), _ptr(nb.slice_ptr), _ptr(nb.col),
        _ptr(nb.cnt), _ptr(cmix), _ptr(v), _ptr(feat), _stream(stream)))
    return feat


def env_forward(n, slice_ptr, cnt, feat, v, species, model: EnvModel, total: int, dtype=torch.float32,
                with_diag=True, stream=None):
    """(val [total], diag [n] or None) of the model from stored bond inputs."""
    val = torch.zeros(max(total, 1), dtype=dtype, device=feat.device)
    diag = torch.zeros(n, dtype=dtype, device=feat.device) if with_diag else None
    _check("tb_env_forward", lib().tb_env_forward(
        n, _ptr(slice_ptr), _ptr(cnt), _ptr(feat), _ptr(v), _ptr(species), _ptr(model.p), _ptr(model.eps0),
        precision_of(dtype), _ptr(val), _ptr(diag), _stream(stream)))
    return val, diag


def build_hamiltonian_env(positions, species, box, pbc, rcut, nb: Neighbors, model: EnvModel, v=None,
                          dtype=torch.float32, with_diag=True, stream=None) -> SellMatrix:
    """H of the environment-network model straight from positions."""
    if v is None:
        v = compute_descriptors(positions, species, box, pbc, rcut, nb, model.cmix, stream)
    b, p, bptr, pptr = _host_box(box, pbc)
    val = torch.zeros(max(nb.total, 1), dtype=dtype, device=positions.device)
    diag = torch.empty(nb.n, dtype=dtype, device=positions.device) if with_diag else None
    ws = _workspace(lib().tb_build_hamiltonian_env_workspace_size(nb.n), positions.device)
    _check("tb_build_hamiltonian_env", lib().tb_build_hamiltonian_env(
        _ptr(positions), _ptr(species), nb.n, bptr, pptr, float(rcut), _ptr(nb.slice_ptr), _ptr(nb.col),
        _ptr(nb.cnt), _ptr(model.cmix), _ptr(v), _ptr(model.p), _ptr(model.eps0), precision_of(dtype), _ptr(val),
        _ptr(diag), _ptr(ws), ws.numel(), _stream(stream)))
    return SellMatrix(nb.n, nb.slice_ptr, nb.col, val[:nb.total], diag)


def env_set_variant(variant: int):
    """Kernel of build_hamiltonian_env: 0 = tensor cores (BF16 operands,
    default), 1 = FP32 pipes (bit for bit the arithmetic of env_forward)."""
    _check("tb_env_set_variant", lib().tb_env_set_variant(int(variant)))


def env_backward(n, slice_ptr, cnt, total, feat, v, species, model: EnvModel, g_val, g_diag, grad=None,
                 workspace=None, stream=None) -> torch.Tensor:
    L = lib()
    if grad is None:
        grad = torch.empty(ENV_NPARAM, dtype=torch.float32, device=feat.device)
    need = L.tb_env_backward_workspace_size(n, total)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, feat.device)
    _check("tb_env_backward", L.tb_env_backward(
        n, _ptr(slice_ptr), _ptr(cnt), total, _ptr(feat), _ptr(v), _ptr(species), _ptr(model.p), _ptr(g_val),
        _ptr(g_diag), _ptr(grad), _ptr(workspace), workspace.numel(), _stream(stream)))
    return grad


def bloch_bands(n_cells, n_atoms, rows_per_cell, slice_ptr, col, cnt, feat, val, diag, kpts, max_sweeps=30,
                flags=None, stream=None):
    """(evals [cells, nk, n], evecs [cells, nk, n, n] complex64) of a batch
    of periodic cells (kpts: device float32 [nk, 3])."""
    n_k = kpts.shape[0]
    dev = feat.device
    evals = torch.empty((n_cells, n_k, n_atoms), dtype=torch.float32, device=dev)
    evecs = torch.empty((n_cells, n_k, n_atoms, n_atoms), dtype=torch.complex64, device=dev)
    if flags is None:
        flags = torch.zeros(1, dtype=torch.int32, device=dev)
    _check("tb_bloch_bands", lib().tb_bloch_bands(
        n_cells, n_atoms, rows_per_cell, _ptr(slice_ptr), _ptr(col), _ptr(cnt), _ptr(feat), _ptr(val), _ptr(diag),
        n_k, _ptr(kpts), max_sweeps, _ptr(evals), _ptr(evecs), _ptr(flags), _stream(stream)))
    return evals, evecs


def band_loss(evals, e_ref, weights, dLdE=None, stats=None, stream=None):
    """(dL/dE, stats = {S, sum w D^2, L} device float64 [3]) of Eq. 3."""
    nb = evals.shape[-1]
    if dLdE is None:
        dLdE = torch.empty_like(evals)
    if stats is None:
        stats = torch.empty(3, dtype=torch.float64, device=evals.device)
    _check("tb_band_loss", lib().tb_band_loss(evals.numel() // nb, nb, _ptr(evals), _ptr(e_ref), _ptr(weights),
                                              _ptr(dLdE), _ptr(stats), _stream(stream)))
    return dLdE, stats


def band_gradient(n_cells, n_atoms, rows_per_cell, slice_ptr, col, cnt, feat, kpts, evecs, dLdE, total,
                  g_val=None, g_diag=None, stream=None):
    dev = feat.device
    if g_val is None:
        g_val = torch.zeros(max(total, 1), dtype=torch.float32, device=dev)
    if g_diag is None:
        g_diag = torch.zeros(n_cells * rows_per_cell, dtype=torch.float32, device=dev)
    _check("tb_band_gradient", lib().tb_band_gradient(
        n_cells, n_atoms, rows_per_cell, _ptr(slice_ptr), _ptr(col), _ptr(cnt), _ptr(feat), kpts.shape[0],
        _ptr(kpts), _ptr(evecs), _ptr(dLdE), _ptr(g_val), _ptr(g_diag), _stream(stream)))
    return g_val, g_diag


def adamw_flat(model: EnvModel, grad, lr, beta1=0.9, beta2=0.999, eps=1e-8, weight_decay=0.0, stream=None):
    model.step += 1
    _check("tb_adamw_flat", lib().tb_adamw_flat(model.p.numel(), _ptr(model.p), _ptr(grad), _ptr(model.m),
                                                _ptr(model.v), model.step, lr, beta1, beta2, eps, weight_decay,
                                                _stream(stream)))
