"""Thin Python binding of the C ABI in ``include/sft.h`` (libsft.so).

Functions keep the C names and only marshal arguments: torch CUDA tensors are
passed as raw device pointers, host arrays of pointers are built with ctypes.
Every step of the method runs in the library's CUDA kernels; if the library
cannot be loaded this module raises instead of computing anything itself.

``Decomposition`` is a convenience owner of the device buffers (factor, core
and cached-product matrices plus the workspace) that forwards to the same
calls.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import torch

from . import build as _build

SFT_OK, SFT_EINVAL, SFT_ENOMEM, SFT_ECUDA, SFT_ETIMEOUT, SFT_ENOTSUP = range(6)
SFT_FP32, SFT_BF16 = 0, 1
MAX_ORDER = 16
_STATUS = {0: "SFT_OK", 1: "SFT_EINVAL", 2: "SFT_ENOMEM", 3: "SFT_ECUDA", 4: "SFT_ETIMEOUT",
           5: "SFT_ENOTSUP"}

EXPORTED = ["sft_workspace_bytes", "sft_init", "sft_refresh_C", "sft_update_factors",
            "sft_update_core", "sft_loss", "sft_loss_async", "sft_predict", "sft_epoch", "sft_sync",
            "sft_set_stream", "sft_last_error", "sft_launch_count", "sft_destroy",
            "sft_slices_scratch_bytes", "sft_group_slices", "sft_slices_workspace_bytes",
            "sft_update_factors_slices", "sft_update_core_slices", "sft_set_slice_tiling",
            "sft_update_factors_noalloc"]


class SftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sft_config(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("J", ctypes.POINTER(ctypes.c_int32)), ("R", ctypes.c_int32),
                ("prec", ctypes.c_int32), ("deterministic", ctypes.c_int32),
                ("stream", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libsft.so (building it first if needed).  Raises on failure."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(_build.LIB_PATH):
        raise RuntimeError(f"{_build.LIB_PATH} is missing; run paper_2210_06014_gb300.build.build()")
    lib = ctypes.CDLL(_build.LIB_PATH)
    vp, i64, i32, f32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
    cfgp = ctypes.POINTER(sft_config)
    ctx = ctypes.c_void_p
    lib.sft_workspace_bytes.argtypes = [cfgp, i64]
    lib.sft_workspace_bytes.restype = ctypes.c_size_t
    lib.sft_init.argtypes = [cfgp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                             ctypes.POINTER(vp), vp, ctypes.c_size_t, ctypes.POINTER(ctx)]
    lib.sft_init.restype = ctypes.c_int
    lib.sft_refresh_C.argtypes = [ctx, i32]
    lib.sft_refresh_C.restype = ctypes.c_int
    pass_args = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, i64, f32, f32]
    lib.sft_update_factors.argtypes = pass_args
    lib.sft_update_factors.restype = ctypes.c_int
    lib.sft_update_core.argtypes = pass_args
    lib.sft_update_core.restype = ctypes.c_int
    lib.sft_loss.argtypes = [ctx, ctypes.POINTER(vp), vp, i64, ctypes.POINTER(ctypes.c_double),
                             ctypes.POINTER(ctypes.c_double)]
    lib.sft_loss.restype = ctypes.c_int
    lib.sft_loss_async.argtypes = [ctx, ctypes.POINTER(vp), vp, i64, vp]
    lib.sft_loss_async.restype = ctypes.c_int
    lib.sft_predict.argtypes = [ctx, ctypes.POINTER(vp), i64, vp]
    lib.sft_predict.restype = ctypes.c_int
    lib.sft_epoch.argtypes = [ctx, ctypes.POINTER(vp), vp, i64, ctypes.POINTER(vp),
                              ctypes.POINTER(vp), i64, i64, f32, f32, f32, f32]
    lib.sft_epoch.restype = ctypes.c_int
    lib.sft_sync.argtypes = [ctx, i64]
    lib.sft_sync.restype = ctypes.c_int
    lib.sft_set_stream.argtypes = [ctx, vp]
    lib.sft_set_stream.restype = ctypes.c_int
    lib.sft_last_error.argtypes = [ctx]
    lib.sft_last_error.restype = ctypes.c_char_p
    lib.sft_launch_count.argtypes = [ctx]
    lib.sft_launch_count.restype = i64
    lib.sft_destroy.argtypes = [ctx]
    lib.sft_destroy.restype = None
    lib.sft_slices_scratch_bytes.argtypes = [i64]
    lib.sft_slices_scratch_bytes.restype = ctypes.c_size_t
    lib.sft_group_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, ctypes.POINTER(vp),
                                     vp, vp, vp, ctypes.c_size_t]
    lib.sft_group_slices.restype = ctypes.c_int
    lib.sft_slices_workspace_bytes.argtypes = [ctx, i32, i64]
    lib.sft_slices_workspace_bytes.restype = ctypes.c_size_t
    lib.sft_update_factors_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, f32, f32,
                                              vp, ctypes.c_size_t]
    lib.sft_update_factors_slices.restype = ctypes.c_int
    lib.sft_update_core_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, i64, f32, f32]
    lib.sft_update_core_slices.restype = ctypes.c_int
    lib.sft_set_slice_tiling.argtypes = [ctx, i64, i64]
    lib.sft_set_slice_tiling.restype = ctypes.c_int
    lib.sft_update_factors_noalloc.argtypes = [
        i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), i32, i32, vp, vp,
        ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, i64, i64, f32, f32, vp]
    lib.sft_update_factors_noalloc.restype = ctypes.c_int
    _lib = lib
    return lib


# ----------------------------------------------------------------------------- marshalling


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libsft takes device tensors")
    if not t.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _ptr_array(ts: Sequence[Optional[torch.Tensor]]):
    arr = (ctypes.c_void_p * len(ts))()
    for i, t in enumerate(ts):
        arr[i] = None if t is None else t.data_ptr()
    return arr


def make_config(dims, J, R, deterministic=True, prec=SFT_FP32, stream=None):
    dims_a = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    J_a = (ctypes.c_int32 * len(J))(*[int(j) for j in J])
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
    cfg = sft_config(len(dims), dims_a, J_a, int(R), int(prec), 1 if deterministic else 0,
                     ctypes.c_void_p(stream))
    cfg._keep = (dims_a, J_a)
    return cfg


def _check(lib, ctx, status, what):
    if status != SFT_OK:
        msg = lib.sft_last_error(ctx).decode() if ctx else ""
        raise SftError(status, f"{what}: {msg}")


# ----------------------------------------------------------------------------- C-named calls


def sft_workspace_bytes(cfg: sft_config, max_batch: int) -> int:
    return int(load().sft_workspace_bytes(ctypes.byref(cfg), int(max_batch)))


def sft_init(cfg, A, B, C, workspace: torch.Tensor):
    lib = load()
    ctx = ctypes.c_void_p()
    st = lib.sft_init(ctypes.byref(cfg), _ptr_array(A), _ptr_array(B), _ptr_array(C), None,
                      _ptr(workspace), workspace.numel() * workspace.element_size(),
                      ctypes.byref(ctx))
    if st != SFT_OK:
        raise SftError(st, "sft_init")
    return ctx


def sft_refresh_C(ctx, mode: int = -1) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_refresh_C(ctx, int(mode)), "sft_refresh_C")


def sft_update_factors(ctx, mode, idx, val, perm, nnz, batch, lr, lam) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_factors(ctx, int(mode), _ptr_array(idx), _ptr(val),
                                            _ptr(perm), int(nnz), int(batch), float(lr),
                                            float(lam)), "sft_update_factors")


def sft_update_core(ctx, mode, idx, val, perm, nnz, batch, lr, lam) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_core(ctx, int(mode), _ptr_array(idx), _ptr(val), _ptr(perm),
                                         int(nnz), int(batch), float(lr), float(lam)),
           "sft_update_core")


def sft_loss(ctx, idx, val, nnz):
    lib = load()
    sse, sae = ctypes.c_double(), ctypes.c_double()
    _check(lib, ctx, lib.sft_loss(ctx, _ptr_array(idx), _ptr(val), int(nnz), ctypes.byref(sse),
                                  ctypes.byref(sae)), "sft_loss")
    return sse.value, sae.value


def sft_loss_async(ctx, idx, val, nnz, out2: torch.Tensor) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_loss_async(ctx, _ptr_array(idx), _ptr(val), int(nnz), _ptr(out2)),
           "sft_loss_async")


def sft_predict(ctx, idx, nnz, out: torch.Tensor) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_predict(ctx, _ptr_array(idx), int(nnz), _ptr(out)), "sft_predict")


def sft_epoch(ctx, idx, val, nnz, perm_factor, perm_core, batch_factor, batch_core, lr_A, lam_A,
              lr_B, lam_B) -> None:
    lib = load()
    pf = _ptr_array(perm_factor) if perm_factor is not None else None
    pc = _ptr_array(perm_core) if perm_core is not None else None
    _check(lib, ctx, lib.sft_epoch(ctx, _ptr_array(idx), _ptr(val), int(nnz), pf, pc,
                                   int(batch_factor), int(batch_core), float(lr_A), float(lam_A),
                                   float(lr_B), float(lam_B)), "sft_epoch")


def sft_sync(ctx, timeout_ms: int = -1) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_sync(ctx, int(timeout_ms)), "sft_sync")


def sft_set_stream(ctx, stream) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_stream(ctx, ctypes.c_void_p(stream)), "sft_set_stream")


def sft_launch_count(ctx) -> int:
    return int(load().sft_launch_count(ctx))


def sft_destroy(ctx) -> None:
    if ctx:
        load().sft_destroy(ctx)


def sft_slices_scratch_bytes(nnz: int) -> int:
    return int(load().sft_slices_scratch_bytes(int(nnz)))


def sft_group_slices(ctx, mode, idx, val, perm, nnz, out_idx, out_val, out_row_ptr,
                     scratch: torch.Tensor) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_group_slices(ctx, int(mode), _ptr_array(idx), _ptr(val), _ptr(perm),
                                          int(nnz), _ptr_array(out_idx), _ptr(out_val),
                                          _ptr(out_row_ptr), _ptr(scratch),
                                          scratch.numel() * scratch.element_size()),
           "sft_group_slices")


def sft_slices_workspace_bytes(ctx, mode, nnz) -> int:
    return int(load().sft_slices_workspace_bytes(ctx, int(mode), int(nnz)))


def sft_update_factors_slices(ctx, mode, sidx, sval, row_ptr, nnz, lr, lam,
                              workspace: torch.Tensor) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_factors_slices(ctx, int(mode), _ptr_array(sidx), _ptr(sval),
                                                   _ptr(row_ptr), int(nnz), float(lr), float(lam),
                                                   _ptr(workspace),
                                                   workspace.numel() * workspace.element_size()),
           "sft_update_factors_slices")


def sft_update_core_slices(ctx, mode, sidx, sval, row_ptr, nnz, batch, lr, lam) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_core_slices(ctx, int(mode), _ptr_array(sidx), _ptr(sval),
                                                _ptr(row_ptr), int(nnz), int(batch), float(lr),
                                                float(lam)), "sft_update_core_slices")


def sft_set_slice_tiling(ctx, tile: int = 0, max_direct: int = 0) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_slice_tiling(ctx, int(tile), int(max_direct)),
           "sft_set_slice_tiling")


def sft_update_factors_noalloc(dims, J, R, mode, A_mode, B_mode, C, idx, val, perm, nnz, batch,
                               lr, lam, stream=None) -> int:
    """The allocation-free factor pass; returns the sft_status code."""
    lib = load()
    dims_a = (ctypes.c_int64 * len(dims))(*[int(d) for d in dims])
    J_a = (ctypes.c_int32 * len(J))(*[int(j) for j in J])
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return int(lib.sft_update_factors_noalloc(len(dims), dims_a, J_a, int(R), int(mode),
                                              _ptr(A_mode), _ptr(B_mode), _ptr_array(C),
                                              _ptr_array(idx), _ptr(val), _ptr(perm), int(nnz),
                                              int(batch), float(lr), float(lam),
                                              ctypes.c_void_p(stream)))


class Slices:
    """The slice layout of one mode (device tensors): idx (N int32 arrays),
    val (float32) and row_ptr (I_n + 1 int32), built by sft_group_slices."""

    def __init__(self, dec: "Decomposition", mode: int, idx, val, perm=None):
        nnz = val.numel()
        dev = val.device
        self.mode = mode
        self.nnz = nnz
        self.idx = [torch.empty(nnz, dtype=torch.int32, device=dev) for _ in idx]
        self.val = torch.empty(nnz, dtype=torch.float32, device=dev)
        self.row_ptr = torch.empty(dec.dims[mode] + 1, dtype=torch.int32, device=dev)
        scratch = torch.empty(max(16, sft_slices_scratch_bytes(nnz)), dtype=torch.uint8,
                              device=dev)
        sft_group_slices(dec.ctx, mode, idx, val, perm, nnz, self.idx, self.val, self.row_ptr,
                         scratch)
        self._scratch = scratch  # kept alive until the enqueued work has run


# ----------------------------------------------------------------------------- owner object


class Decomposition:
    """Device-resident FastTucker parameters plus a libsft context.

    A[n] (I_n x J_n) and B[n] (J_n x R) are float32 torch tensors on the current
    CUDA device; C[n] = A[n] B[n] (I_n x R) is float32, or bfloat16 with
    prec = SFT_BF16; ``workspace`` is a byte tensor sized by
    sft_workspace_bytes.  All methods forward to the C ABI."""

    def __init__(self, A0: Sequence[torch.Tensor], B0: Sequence[torch.Tensor],
                 deterministic: bool = True, max_batch: int = 4096, device="cuda",
                 stream=None, prec: int = SFT_FP32):
        self.A = [a.to(device=device, dtype=torch.float32).contiguous().clone() for a in A0]
        self.B = [b.to(device=device, dtype=torch.float32).contiguous().clone() for b in B0]
        self.N = len(self.A)
        self.R = int(self.B[0].shape[1])
        self.dims = [int(a.shape[0]) for a in self.A]
        self.J = [int(a.shape[1]) for a in self.A]
        self.prec = prec
        cdt = torch.bfloat16 if prec == SFT_BF16 else torch.float32
        self.C = [torch.empty(i, self.R, device=device, dtype=cdt) for i in self.dims]
        self.cfg = make_config(self.dims, self.J, self.R, deterministic, prec, stream)
        nbytes = sft_workspace_bytes(self.cfg, max_batch)
        if nbytes == 0:
            raise SftError(SFT_EINVAL, "sft_workspace_bytes rejected the configuration")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.ctx = sft_init(self.cfg, self.A, self.B, self.C, self.workspace)
        sft_refresh_C(self.ctx, -1)

    def close(self):
        if getattr(self, "ctx", None):
            sft_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refresh(self, mode: int = -1):
        sft_refresh_C(self.ctx, mode)

    def update_factors(self, mode, idx, val, perm=None, batch=4096, lr=0.01, lam=0.01):
        sft_update_factors(self.ctx, mode, idx, val, perm, val.numel(), batch, lr, lam)

    def update_core(self, mode, idx, val, perm=None, batch=4096, lr=0.01, lam=0.01):
        sft_update_core(self.ctx, mode, idx, val, perm, val.numel(), batch, lr, lam)

    def epoch(self, idx, val, perm_factor=None, perm_core=None, batch_factor=4096,
              batch_core=4096, lr_A=0.01, lam_A=0.01, lr_B=0.01, lam_B=0.01):
        sft_epoch(self.ctx, idx, val, val.numel(), perm_factor, perm_core, batch_factor,
                  batch_core, lr_A, lam_A, lr_B, lam_B)

    def slices(self, mode, idx, val, perm=None) -> Slices:
        return Slices(self, mode, idx, val, perm)

    def set_slice_tiling(self, tile: int = 0, max_direct: int = 0):
        sft_set_slice_tiling(self.ctx, tile, max_direct)

    def update_factors_slices(self, sl: Slices, lr=0.01, lam=0.01):
        need = max(16, sft_slices_workspace_bytes(self.ctx, sl.mode, sl.nnz))
        ws = getattr(self, "_slice_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=sl.val.device)
            self._slice_ws = ws
        sft_update_factors_slices(self.ctx, sl.mode, sl.idx, sl.val, sl.row_ptr, sl.nnz, lr, lam,
                                  ws)

    def update_core_slices(self, sl: Slices, batch=None, lr=0.01, lam=0.01):
        sft_update_core_slices(self.ctx, sl.mode, sl.idx, sl.val, sl.row_ptr, sl.nnz,
                               batch or sl.nnz, lr, lam)

    def loss(self, idx, val):
        return sft_loss(self.ctx, idx, val, val.numel())

    def predict(self, idx) -> torch.Tensor:
        out = torch.empty(idx[0].numel(), dtype=torch.float32, device=idx[0].device)
        sft_predict(self.ctx, idx, idx[0].numel(), out)
        return out

    def rmse(self, idx, val) -> float:
        sse, _ = self.loss(idx, val)
        return (sse / max(1, val.numel())) ** 0.5

    def sync(self, timeout_ms: int = -1):
        sft_sync(self.ctx, timeout_ms)

    @property
    def launches(self) -> int:
        return sft_launch_count(self.ctx)
