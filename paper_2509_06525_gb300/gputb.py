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
    "kpm_moments": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32, _c_i32,
                             _c_u64, _c_vp, _c_vp, _c_sz, _c_vp, ctypes.POINTER(_c_dbl)]),
    "kpm_moments_noalloc": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_dbl, _c_dbl, _c_i32,
                                     _c_i32, _c_u64, _c_vp, _c_vp]),
    "kpm_dos": (_c_i32, [_c_vp, _c_i32, _c_i32, _c_i32, _c_dbl, _c_dbl, _c_dbl, _c_vp, _c_i32, _c_vp, _c_vp]),
    "tb_neighbors_workspace_size": (_c_sz, [_c_i64, _c_vp, _c_vp, _c_dbl]),
    "tb_build_neighbors": (_c_i32, [_c_vp, _c_i64, _c_vp, _c_vp, _c_dbl, _c_dbl, _c_i32, _c_vp, _c_vp, _c_i64,
                                    _c_vp, _c_vp, ctypes.POINTER(_c_i64), _c_vp, _c_sz, _c_vp]),
    "tb_build_hamiltonian_teacher": (_c_i32, [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_vp,
                                              _c_vp, _c_vp, _c_dbl, _c_dbl, _c_dbl, _c_dbl, _c_i32, _c_vp,
                                              _c_vp, _c_vp]),
    "tb_spectral_bounds_workspace_size": (_c_sz, [_c_i64, _c_i32]),
    "tb_spectral_bounds": (_c_i32, [_c_i64, _c_vp, _c_vp, _c_vp, _c_vp, _c_i32, _c_i32, _c_u64, _c_vp, _c_vp,
                                    _c_sz, _c_vp]),
}


class GputbError(RuntimeError):
    def __init__(self, func: str, status: int, message: str):
        super().__init__(f"{func} failed with status {status}: {message}")
        self.status = status


_lib: Optional[ctypes.CDLL] = None


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
        _lib = handle
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


def kpm_moments(H: SellMatrix, a: float, b: float, M: int, R: int, seed: int,
                stream=None, workspace: Optional[torch.Tensor] = None, timing: Optional[list] = None
                ) -> torch.Tensor:
    """Per-vector KPM moments mu_r [R, M] (float64, device).

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
                       float(a), float(b), int(M), int(R), int(seed) & ((1 << 64) - 1),
                       _ptr(mu), _ptr(ws), ws.numel(), _stream(stream),
                       ctypes.byref(step_ms) if timing is not None else None)
    _check("kpm_moments", st)
    if timing is not None:
        timing.append(step_ms.value)
    return mu


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
    need = L.tb_neighbors_workspace_size(n, bptr, pptr, float(rcut))
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
    st = L.tb_build_hamiltonian_teacher(
        _ptr(positions), _ptr(species), nb.n, bptr, pptr, _ptr(nb.slice_ptr), _ptr(nb.col), _ptr(nb.cnt),
        _ptr(nb.ncount), pref.ctypes.data_as(ctypes.c_void_p), onsite.ctypes.data_as(ctypes.c_void_p),
        float(teacher.a_cc), float(teacher.beta), float(teacher.gamma), float(teacher.rcut), precision_of(dtype),
        _ptr(val), _ptr(diag), _stream(stream))
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
