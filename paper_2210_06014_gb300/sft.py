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
            "sft_slices_scratch_bytes", "sft_group_slices", "sft_slices_expand_rows",
            "sft_fibers_expand_coords",
            "sft_slices_workspace_bytes",
            "sft_update_factors_slices", "sft_update_core_slices", "sft_set_slice_tiling",
            "sft_update_factors_noalloc", "sft_loss_grad_C", "sft_grad_AB",
            "sft_batch_workspace_bytes", "sft_batch_create", "sft_batch_refresh",
            "sft_batch_epoch", "sft_batch_loss", "sft_batch_snapshot_bytes", "sft_batch_autotune",
            "sft_batch_sync", "sft_batch_launch_count", "sft_batch_epoch_tasks",
            "sft_batch_last_error", "sft_batch_destroy", "sft_batch_plan",
            "sft_batch_set_wait_limit", "sft_batch_hold_pass", "sft_fibers_scratch_bytes",
            "sft_group_fibers", "sft_update_factors_fibers", "sft_update_core_fibers",
            "sft_autotune_slices", "sft_set_tensor_cores", "sft_set_tc_wait_limit",
            "sft_set_long_slices", "sft_set_blocked_chains"]


class SftError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sft_batch_problem(ctypes.Structure):
    _fields_ = [("order", ctypes.c_int32), ("dims", ctypes.POINTER(ctypes.c_int64)),
                ("R", ctypes.c_int32), ("A", ctypes.POINTER(ctypes.c_void_p)),
                ("B", ctypes.POINTER(ctypes.c_void_p)), ("C", ctypes.POINTER(ctypes.c_void_p)),
                ("idx", ctypes.POINTER(ctypes.c_void_p)), ("val", ctypes.c_void_p),
                ("nnz", ctypes.c_int64), ("lr_A", ctypes.c_float), ("lambda_A", ctypes.c_float),
                ("lr_B", ctypes.c_float), ("lambda_B", ctypes.c_float)]


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
    lib.sft_slices_expand_rows.argtypes = [ctx, i32, vp, i64, vp]
    lib.sft_slices_expand_rows.restype = ctypes.c_int
    lib.sft_fibers_expand_coords.argtypes = [ctx, i32, vp, i64, vp, i64, vp]
    lib.sft_fibers_expand_coords.restype = ctypes.c_int
    lib.sft_slices_workspace_bytes.argtypes = [ctx, i32, i64]
    lib.sft_slices_workspace_bytes.restype = ctypes.c_size_t
    lib.sft_update_factors_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, f32, f32,
                                              vp, ctypes.c_size_t]
    lib.sft_update_factors_slices.restype = ctypes.c_int
    lib.sft_update_core_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, i64, f32, f32]
    lib.sft_update_core_slices.restype = ctypes.c_int
    lib.sft_set_slice_tiling.argtypes = [ctx, i64, i64]
    lib.sft_set_slice_tiling.restype = ctypes.c_int
    lib.sft_set_tensor_cores.argtypes = [ctx, i32]
    lib.sft_set_tensor_cores.restype = ctypes.c_int
    lib.sft_set_tc_wait_limit.argtypes = [ctx, i64]
    lib.sft_set_tc_wait_limit.restype = ctypes.c_int
    lib.sft_set_long_slices.argtypes = [ctx, i32]
    lib.sft_set_long_slices.restype = ctypes.c_int
    lib.sft_set_blocked_chains.argtypes = [ctx, i32]
    lib.sft_set_blocked_chains.restype = ctypes.c_int
    lib.sft_update_factors_noalloc.argtypes = [
        i32, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32), i32, i32, vp, vp,
        ctypes.POINTER(vp), ctypes.POINTER(vp), vp, vp, i64, i64, f32, f32, vp]
    lib.sft_update_factors_noalloc.restype = ctypes.c_int
    bp = ctypes.POINTER(sft_batch_problem)
    lib.sft_batch_workspace_bytes.argtypes = [i32, bp, i64]
    lib.sft_batch_workspace_bytes.restype = ctypes.c_size_t
    lib.sft_batch_create.argtypes = [i32, bp, i32, i64, i64, i32, vp, ctypes.c_size_t, vp,
                                     ctypes.POINTER(vp)]
    lib.sft_batch_create.restype = ctypes.c_int
    for name in ("sft_batch_refresh", "sft_batch_epoch"):
        getattr(lib, name).argtypes = [vp]
        getattr(lib, name).restype = ctypes.c_int
    lib.sft_batch_loss.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    lib.sft_batch_loss.restype = ctypes.c_int
    lib.sft_batch_snapshot_bytes.argtypes = [vp]
    lib.sft_batch_snapshot_bytes.restype = ctypes.c_size_t
    lib.sft_batch_autotune.argtypes = [vp, vp, ctypes.c_size_t, i32, ctypes.POINTER(i64),
                                       ctypes.POINTER(i32)]
    lib.sft_batch_autotune.restype = ctypes.c_int
    lib.sft_batch_sync.argtypes = [vp, i64]
    lib.sft_batch_sync.restype = ctypes.c_int
    lib.sft_batch_launch_count.argtypes = [vp]
    lib.sft_batch_launch_count.restype = i64
    lib.sft_batch_epoch_tasks.argtypes = [vp]
    lib.sft_batch_epoch_tasks.restype = i64
    lib.sft_batch_last_error.argtypes = [vp]
    lib.sft_batch_last_error.restype = ctypes.c_char_p
    lib.sft_batch_set_wait_limit.argtypes = [vp, i64]
    lib.sft_batch_set_wait_limit.restype = ctypes.c_int
    lib.sft_batch_hold_pass.argtypes = [vp, i32, i32]
    lib.sft_batch_hold_pass.restype = ctypes.c_int
    lib.sft_batch_plan.argtypes = [i32, bp, i32, i64, i32, vp, i64]
    lib.sft_batch_plan.restype = i64
    lib.sft_batch_destroy.argtypes = [vp]
    lib.sft_batch_destroy.restype = None
    lib.sft_fibers_scratch_bytes.argtypes = [i64]
    lib.sft_fibers_scratch_bytes.restype = ctypes.c_size_t
    lib.sft_group_fibers.argtypes = [ctx, i32, ctypes.POINTER(vp), i64, vp, ctypes.POINTER(vp),
                                     ctypes.POINTER(i64), vp, ctypes.c_size_t]
    lib.sft_group_fibers.restype = ctypes.c_int
    lib.sft_update_factors_fibers.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, vp,
                                              ctypes.POINTER(vp), i64, vp, f32, f32, vp,
                                              ctypes.c_size_t]
    lib.sft_update_factors_fibers.restype = ctypes.c_int
    lib.sft_update_core_fibers.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, i64, vp,
                                           ctypes.POINTER(vp), i64, vp, f32, f32]
    lib.sft_update_core_fibers.restype = ctypes.c_int
    lib.sft_autotune_slices.argtypes = [ctx, i32, ctypes.POINTER(vp), vp, vp, i64, vp,
                                        ctypes.POINTER(vp), i64, vp, f32, f32, vp, ctypes.c_size_t,
                                        vp, ctypes.c_size_t, ctypes.POINTER(i64)]
    lib.sft_autotune_slices.restype = ctypes.c_int
    lib.sft_loss_grad_C.argtypes = [ctx, ctypes.POINTER(vp), vp, i64, ctypes.POINTER(vp), i32, vp]
    lib.sft_loss_grad_C.restype = ctypes.c_int
    lib.sft_grad_AB.argtypes = [ctx, ctypes.POINTER(vp), vp, ctypes.POINTER(vp), ctypes.POINTER(vp)]
    lib.sft_grad_AB.restype = ctypes.c_int
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


def sft_slices_expand_rows(ctx, mode, row_ptr, nnz, out):
    """out[p] = slice of position p, from row_ptr (device tensors)."""
    lib = load()
    _check(lib, ctx, lib.sft_slices_expand_rows(ctx, int(mode), _ptr(row_ptr), int(nnz), _ptr(out)),
           "sft_slices_expand_rows")


def sft_fibers_expand_coords(ctx, mode, fid, nnz, fcoord, nfibers, out_idx):
    """out_idx[k][p] = fcoord[k][fid[p]] for k != mode (device tensors; the
    entries for `mode` may be None)."""
    lib = load()
    _check(lib, ctx, lib.sft_fibers_expand_coords(ctx, int(mode), _ptr(fid), int(nnz),
                                                  _ptr_array(fcoord), int(nfibers),
                                                  _ptr_array(out_idx)),
           "sft_fibers_expand_coords")


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


def sft_set_tensor_cores(ctx, enable: bool = True) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_tensor_cores(ctx, 1 if enable else 0), "sft_set_tensor_cores")


SFT_LONG_MAPS, SFT_LONG_SUBSLICES = 0, 1


def sft_set_long_slices(ctx, how: int) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_long_slices(ctx, int(how)), "sft_set_long_slices")


def sft_set_blocked_chains(ctx, enable: bool = True) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_blocked_chains(ctx, 1 if enable else 0), "sft_set_blocked_chains")


def sft_set_tc_wait_limit(ctx, limit_ns: int) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_set_tc_wait_limit(ctx, int(limit_ns)), "sft_set_tc_wait_limit")


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


def sft_loss_grad_C(ctx, idx, val, nnz, dC, accumulate, loss_out: torch.Tensor) -> None:
    lib = load()
    dptr = _ptr_array(dC) if dC is not None else None
    _check(lib, ctx, lib.sft_loss_grad_C(ctx, _ptr_array(idx), _ptr(val), int(nnz), dptr,
                                         int(accumulate), _ptr(loss_out)), "sft_loss_grad_C")


def sft_grad_AB(ctx, dC, scale: Optional[torch.Tensor], gA, gB) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_grad_AB(ctx, _ptr_array(dC), _ptr(scale), _ptr_array(gA),
                                     _ptr_array(gB)), "sft_grad_AB")


def sft_fibers_scratch_bytes(nnz: int) -> int:
    return int(load().sft_fibers_scratch_bytes(int(nnz)))


def sft_group_fibers(ctx, mode, sidx, nnz, fid, fcoord, scratch: torch.Tensor) -> int:
    """fcoord: list of N int32 device tensors (None for `mode`)."""
    lib = load()
    n = ctypes.c_int64()
    _check(lib, ctx, lib.sft_group_fibers(ctx, int(mode), _ptr_array(sidx), int(nnz), _ptr(fid),
                                          _ptr_array(fcoord), ctypes.byref(n), _ptr(scratch),
                                          scratch.numel() * scratch.element_size()),
           "sft_group_fibers")
    return int(n.value)


def sft_update_factors_fibers(ctx, mode, sidx, sval, row_ptr, nnz, fid, fcoord, nfibers, V, lr, lam,
                              workspace: torch.Tensor) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_factors_fibers(ctx, int(mode), _ptr_array(sidx), _ptr(sval),
                                                   _ptr(row_ptr), int(nnz), _ptr(fid),
                                                   _ptr_array(fcoord),
                                                   int(nfibers), _ptr(V), float(lr), float(lam),
                                                   _ptr(workspace),
                                                   workspace.numel() * workspace.element_size()),
           "sft_update_factors_fibers")


def sft_update_core_fibers(ctx, mode, sidx, sval, row_ptr, nnz, batch, fid, fcoord, nfibers, P, lr,
                           lam) -> None:
    lib = load()
    _check(lib, ctx, lib.sft_update_core_fibers(ctx, int(mode), _ptr_array(sidx), _ptr(sval),
                                                _ptr(row_ptr), int(nnz), int(batch), _ptr(fid),
                                                _ptr_array(fcoord), int(nfibers), _ptr(P), float(lr),
                                                float(lam)), "sft_update_core_fibers")


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
        self.fid = self.fcoord = self.V = self.P = None
        self.nfibers = 0
        self._J = dec.J[mode]
        self._R = dec.R

    # A per-fiber p table pays in the core pass only while it stays in L2: the
    # per-nonzero path gathers cached rows that are L2-resident anyway.
    CORE_FIBER_BYTES = 96 << 20

    def build_fibers(self, dec: "Decomposition", core=None) -> int:
        """Fiber ids of the layout (sft_group_fibers) and a v buffer; the factor
        pass then forms v once per fiber.  core=None: also a p buffer for the
        core pass when it is at most CORE_FIBER_BYTES; True / False force it.
        Returns the number of fibers."""
        dev = self.val.device
        self.fid = torch.empty(max(1, self.nnz), dtype=torch.int32, device=dev)
        self.fcoord = [None if k == self.mode else
                       torch.empty(max(1, self.nnz), dtype=torch.int32, device=dev)
                       for k in range(len(self.idx))]
        scratch = torch.empty(max(16, sft_fibers_scratch_bytes(self.nnz)), dtype=torch.uint8,
                              device=dev)
        try:
            self.nfibers = sft_group_fibers(dec.ctx, self.mode, self.idx, self.nnz, self.fid,
                                            self.fcoord, scratch)
        except SftError:
            self.drop_fibers()
            raise
        del scratch
        self.V = torch.empty(max(1, self.nfibers), self._J, dtype=torch.float32, device=dev)
        if core is None:
            core = self.nfibers * self._R * 4 <= self.CORE_FIBER_BYTES
        self.P = (torch.empty(max(1, self.nfibers), self._R, dtype=torch.float32, device=dev)
                  if core else None)
        return self.nfibers

    def drop_fibers(self):
        self.fid = self.fcoord = self.V = self.P = None
        self.nfibers = 0


# ----------------------------------------------------------------------------- owner object


class Decomposition:
    """Device-resident FastTucker parameters plus a libsft context.

    A[n] (I_n x J_n) and B[n] (J_n x R) are float32 torch tensors on the current
    CUDA device; C[n] = A[n] B[n] (I_n x R) is float32, or bfloat16 with
    prec = SFT_BF16; ``workspace`` is a byte tensor sized by
    sft_workspace_bytes.  ``tensor_cores`` selects the tcgen05 refresh and core
    gradient for bfloat16 C (sft_set_tensor_cores).  All methods forward to the
    C ABI."""

    def __init__(self, A0: Sequence[torch.Tensor], B0: Sequence[torch.Tensor],
                 deterministic: bool = True, max_batch: int = 4096, device="cuda",
                 stream=None, prec: int = SFT_FP32, copy: bool = True,
                 tensor_cores: bool = True):
        if copy:
            self.A = [a.to(device=device, dtype=torch.float32).contiguous().clone() for a in A0]
            self.B = [b.to(device=device, dtype=torch.float32).contiguous().clone() for b in B0]
        else:
            # bind the caller's tensors (e.g. nn.Parameters): updates happen in place
            for t in list(A0) + list(B0):
                if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
                    raise ValueError("copy=False needs contiguous float32 CUDA tensors")
            self.A = list(A0)
            self.B = list(B0)
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
        sft_set_tensor_cores(self.ctx, tensor_cores)
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

    def set_blocked_chains(self, enable: bool = True):
        """Long chains of the fiber pass in 32-position blocks (default) or not."""
        sft_set_blocked_chains(self.ctx, enable)

    def set_long_slices(self, how: int):
        """SFT_LONG_MAPS (exact, default) or SFT_LONG_SUBSLICES (B-CSF style)."""
        sft_set_long_slices(self.ctx, how)

    def update_factors_slices(self, sl: Slices, lr=0.01, lam=0.01):
        need = max(16, sft_slices_workspace_bytes(self.ctx, sl.mode, sl.nnz))
        ws = getattr(self, "_slice_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=sl.val.device)
            self._slice_ws = ws
        if sl.fid is not None:
            sft_update_factors_fibers(self.ctx, sl.mode, sl.idx, sl.val, sl.row_ptr, sl.nnz, sl.fid,
                                      sl.fcoord, sl.nfibers, sl.V, lr, lam, ws)
        else:
            sft_update_factors_slices(self.ctx, sl.mode, sl.idx, sl.val, sl.row_ptr, sl.nnz, lr,
                                      lam, ws)

    def autotune_slices(self, sl: Slices, lr=0.01, lam=0.01) -> int:
        """sft_autotune_slices for the layout's mode; returns the chosen limit on
        the length of a slice run whole (A is left unchanged)."""
        lib = load()
        need = max(16, sft_slices_workspace_bytes(self.ctx, sl.mode, sl.nnz))
        ws = getattr(self, "_slice_ws", None)
        if ws is None or ws.numel() < need:
            ws = torch.empty(need, dtype=torch.uint8, device=sl.val.device)
            self._slice_ws = ws
        scratch = torch.empty_like(self.A[sl.mode])
        out = ctypes.c_int64()
        fib = sl.fid is not None
        _check(lib, self.ctx, lib.sft_autotune_slices(
            self.ctx, int(sl.mode), _ptr_array(sl.idx), _ptr(sl.val), _ptr(sl.row_ptr),
            int(sl.nnz), _ptr(sl.fid) if fib else None,
            _ptr_array(sl.fcoord) if fib else None, int(sl.nfibers),
            _ptr(sl.V) if fib else None, float(lr), float(lam), _ptr(ws),
            ws.numel() * ws.element_size(), _ptr(scratch),
            scratch.numel() * scratch.element_size(), ctypes.byref(out)),
            "sft_autotune_slices")
        return int(out.value)

    def update_core_slices(self, sl: Slices, batch=None, lr=0.01, lam=0.01):
        if sl.fid is not None and sl.P is not None:
            sft_update_core_fibers(self.ctx, sl.mode, sl.idx, sl.val, sl.row_ptr, sl.nnz,
                                   batch or sl.nnz, sl.fid, sl.fcoord, sl.nfibers, sl.P, lr, lam)
        else:
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

    def loss_grad_C(self, idx, val, dC=None, accumulate=False):
        """Enqueue L = 1/2 sum e^2 and dL/dC^(n) for every mode.  Returns
        (out, dC): out is a device float64 pair {L, sum |e|}, dC the list of
        I_n x R float32 gradients (allocated when not given)."""
        dev = val.device
        if dC is None:
            dC = [torch.empty(i, self.R, dtype=torch.float32, device=dev) for i in self.dims]
        out = torch.empty(2, dtype=torch.float64, device=dev)
        sft_loss_grad_C(self.ctx, idx, val, val.numel(), dC, accumulate, out)
        return out, dC

    def grad_AB(self, dC, scale=None):
        """(gA, gB) = (s dC[n] B[n]^T, s A[n]^T dC[n]) for every mode; s a device
        float64 scalar tensor or None for 1."""
        gA = [torch.empty_like(a) for a in self.A]
        gB = [torch.empty_like(b) for b in self.B]
        if scale is not None:
            scale = scale.detach().to(torch.float64).reshape(1).contiguous()
        sft_grad_AB(self.ctx, dC, scale, gA, gB)
        return gA, gB

    @property
    def launches(self) -> int:
        return sft_launch_count(self.ctx)


# ----------------------------------------------------------------------------- autograd


class _SampledLossFn(torch.autograd.Function):
    """L = 1/2 sum_s (x_s - x^_s)^2 as a function of A[0..N) and B[0..N).

    The forward refreshes every C^(n) from the current A and B, then runs the
    fused loss + dL/dC pass (when any input needs a gradient) and keeps dC for
    the backward, which projects it onto A and B scaled by the incoming
    gradient.  All arithmetic runs in libsft's kernels."""

    @staticmethod
    def forward(fctx, dec, idx, val, *params):
        N = dec.N
        for n, t in enumerate(params):
            own = dec.A[n] if n < N else dec.B[n - N]
            if t.data_ptr() != own.data_ptr():
                raise ValueError("parameters are not the tensors bound to the Decomposition")
        dec.refresh(-1)
        if any(fctx.needs_input_grad[3:]):
            out, dC = dec.loss_grad_C(list(idx), val)
            fctx.dec = dec
            fctx.dC = dC
        else:
            out = torch.empty(2, dtype=torch.float64, device=val.device)
            sft_loss_grad_C(dec.ctx, list(idx), val, val.numel(), None, 0, out)
        return out[0]

    @staticmethod
    def backward(fctx, g):
        gA, gB = fctx.dec.grad_AB(fctx.dC, g)
        fctx.dC = None
        want = fctx.needs_input_grad[3:]
        N = fctx.dec.N
        grads = [gA[n] if want[n] else None for n in range(N)]
        grads += [gB[n] if want[N + n] else None for n in range(N)]
        return (None, None, None, *grads)


class SampledLoss(torch.nn.Module):
    """Differentiable sampled loss of a sparse FastTucker model.

    Parameters A[n] (I_n x J_n) and B[n] (J_n x R) are ``nn.Parameter``s whose
    storage is bound to a libsft context, so any torch optimiser can train
    them; ``forward(idx, val)`` returns L = 1/2 sum over the given nonzeros of
    (x - x^)^2 as a float64 scalar, and its backward is libsft's gradient
    (Eq. (10)/(11) without the regulariser, summed over the set)."""

    def __init__(self, A0, B0, prec: int = SFT_FP32, device="cuda"):
        super().__init__()
        self.A = torch.nn.ParameterList(
            [torch.nn.Parameter(a.to(device=device, dtype=torch.float32).contiguous().clone())
             for a in A0])
        self.B = torch.nn.ParameterList(
            [torch.nn.Parameter(b.to(device=device, dtype=torch.float32).contiguous().clone())
             for b in B0])
        self.dec = Decomposition([p.data for p in self.A], [p.data for p in self.B], prec=prec,
                                 device=device, copy=False)

    def forward(self, idx, val):
        return _SampledLossFn.apply(self.dec, tuple(idx), val, *self.A, *self.B)


# ----------------------------------------------------------------------------- batched runner


def _bcheck(lib, h, status, what):
    if status != SFT_OK:
        msg = lib.sft_batch_last_error(h).decode() if h else ""
        raise SftError(status, f"{what}: {msg}")


def sft_batch_workspace_bytes(probs, min_chunk) -> int:
    return int(load().sft_batch_workspace_bytes(len(probs), probs, int(min_chunk)))


def sft_batch_create(probs, prec, min_chunk, chunk, blocks_per_sm, workspace, stream):
    lib = load()
    h = ctypes.c_void_p()
    st = lib.sft_batch_create(len(probs), probs, int(prec), int(min_chunk), int(chunk),
                              int(blocks_per_sm), _ptr(workspace),
                              workspace.numel() * workspace.element_size(), ctypes.c_void_p(stream),
                              ctypes.byref(h))
    if st != SFT_OK:
        raise SftError(st, "sft_batch_create")
    return h


def sft_batch_refresh(h) -> None:
    lib = load()
    _bcheck(lib, h, lib.sft_batch_refresh(h), "sft_batch_refresh")


def sft_batch_epoch(h) -> None:
    lib = load()
    _bcheck(lib, h, lib.sft_batch_epoch(h), "sft_batch_epoch")


def sft_batch_loss(h, nprob):
    lib = load()
    out = (ctypes.c_double * (2 * nprob))()
    _bcheck(lib, h, lib.sft_batch_loss(h, out), "sft_batch_loss")
    return [(out[2 * i], out[2 * i + 1]) for i in range(nprob)]


def sft_batch_snapshot_bytes(h) -> int:
    return int(load().sft_batch_snapshot_bytes(h))


def sft_batch_autotune(h, scratch: torch.Tensor, epochs: int = 2):
    lib = load()
    c, b = ctypes.c_int64(), ctypes.c_int32()
    _bcheck(lib, h, lib.sft_batch_autotune(h, _ptr(scratch), scratch.numel() * scratch.element_size(),
                                           int(epochs), ctypes.byref(c), ctypes.byref(b)),
            "sft_batch_autotune")
    return int(c.value), int(b.value)


def sft_batch_sync(h, timeout_ms: int = -1) -> None:
    lib = load()
    _bcheck(lib, h, lib.sft_batch_sync(h, int(timeout_ms)), "sft_batch_sync")


def sft_batch_launch_count(h) -> int:
    return int(load().sft_batch_launch_count(h))


def sft_batch_epoch_tasks(h) -> int:
    return int(load().sft_batch_epoch_tasks(h))


def sft_batch_destroy(h) -> None:
    if h:
        load().sft_batch_destroy(h)


class sft_batch_task_info(ctypes.Structure):
    _fields_ = [("prob", ctypes.c_int32), ("kind", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("wait", ctypes.c_int32), ("done", ctypes.c_int32), ("slot", ctypes.c_int32),
                ("nslots", ctypes.c_int32), ("pad", ctypes.c_int32), ("begin", ctypes.c_int64),
                ("end", ctypes.c_int64)]


def sft_batch_plan(probs, plan: int, chunk: int, workers: int):
    """Task list of a plan as a list of dicts (host only)."""
    lib = load()
    n = int(lib.sft_batch_plan(len(probs), probs, int(plan), int(chunk), int(workers), None, 0))
    if n < 0:
        raise SftError(SFT_EINVAL, "sft_batch_plan")
    out = (sft_batch_task_info * max(1, n))()
    lib.sft_batch_plan(len(probs), probs, int(plan), int(chunk), int(workers), out, n)
    names = [f[0] for f in sft_batch_task_info._fields_]
    return [{k: getattr(out[i], k) for k in names} for i in range(n)]


def batch_problem_records(shapes):
    """ctypes records for host-side planning: shapes = [(dims, R, nnz)].  The
    device pointers are dummies (sft_batch_plan never dereferences them)."""
    arr = (sft_batch_problem * len(shapes))()
    keep = []
    for i, (dims, R, nnz) in enumerate(shapes):
        N = len(dims)
        d = (ctypes.c_int64 * N)(*dims)
        fake = (ctypes.c_void_p * N)(*([256] * N))
        keep += [d, fake]
        arr[i] = sft_batch_problem(N, d, R, fake, fake, fake, fake, 256, nnz, 0.01, 0.01, 0.01, 0.01)
    arr._keep = keep
    return arr


class Batch:
    """Many independent decompositions trained together (include/sft_batch.h).

    problems: sequence of (A0, B0, idx, val): A0[n] (I_n x R), B0[n] (R x R)
    host or device tensors (copied to float32 device tensors owned here), idx
    a list of N int32 device tensors and val a float32 device tensor (borrowed;
    keep them alive).  lr / lam (a number, or one per problem) apply to A and
    B alike."""

    def __init__(self, problems, prec: int = SFT_FP32, min_chunk: int = 2048, chunk: int = 0,
                 blocks_per_sm: int = 0, lr: float = 0.01, lam: float = 0.01, device="cuda",
                 stream=None):
        self.A, self.B, self.C, self.sets = [], [], [], []
        cdt = torch.bfloat16 if prec == SFT_BF16 else torch.float32
        arr = (sft_batch_problem * len(problems))()
        self._keep = []
        lrs = list(lr) if isinstance(lr, (list, tuple)) else [lr] * len(problems)
        lams = list(lam) if isinstance(lam, (list, tuple)) else [lam] * len(problems)
        for i, (A0, B0, idx, val) in enumerate(problems):
            A = [a.to(device=device, dtype=torch.float32).contiguous().clone() for a in A0]
            B = [b.to(device=device, dtype=torch.float32).contiguous().clone() for b in B0]
            R = int(B[0].shape[1])
            C = [torch.empty(a.shape[0], R, device=device, dtype=cdt) for a in A]
            self.A.append(A)
            self.B.append(B)
            self.C.append(C)
            self.sets.append((list(idx), val))
            dims = (ctypes.c_int64 * len(A))(*[a.shape[0] for a in A])
            pa, pb, pc, pi = _ptr_array(A), _ptr_array(B), _ptr_array(C), _ptr_array(list(idx))
            self._keep += [dims, pa, pb, pc, pi]
            arr[i] = sft_batch_problem(len(A), dims, R, pa, pb, pc, pi, val.data_ptr(), val.numel(),
                                       lrs[i], lams[i], lrs[i], lams[i])
        self._probs = arr
        self.nprob = len(problems)
        nbytes = sft_batch_workspace_bytes(arr, min_chunk)
        if nbytes == 0:
            raise SftError(SFT_EINVAL, "sft_batch_workspace_bytes rejected the problems")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=device)
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.h = sft_batch_create(arr, prec, min_chunk, chunk, blocks_per_sm, self.workspace,
                                  stream)
        sft_batch_refresh(self.h)

    def close(self):
        if getattr(self, "h", None):
            sft_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def refresh(self):
        sft_batch_refresh(self.h)

    def epoch(self):
        sft_batch_epoch(self.h)

    def loss(self):
        """[(sum e^2, sum |e|)] per problem over its own nonzeros."""
        return sft_batch_loss(self.h, self.nprob)

    def rmse(self):
        return [(s / max(1, v.numel())) ** 0.5 for (s, _), (_, v) in zip(self.loss(), self.sets)]

    def autotune(self, epochs: int = 2):
        scratch = torch.empty(max(16, sft_batch_snapshot_bytes(self.h)), dtype=torch.uint8,
                              device=self.workspace.device)
        return sft_batch_autotune(self.h, scratch, epochs)

    def sync(self, timeout_ms: int = -1):
        sft_batch_sync(self.h, timeout_ms)

    def set_wait_limit(self, polls: int):
        lib = load()
        _bcheck(lib, self.h, lib.sft_batch_set_wait_limit(self.h, int(polls)),
                "sft_batch_set_wait_limit")

    def hold_pass(self, prob: int, hold: bool = True):
        lib = load()
        _bcheck(lib, self.h, lib.sft_batch_hold_pass(self.h, int(prob), 1 if hold else 0),
                "sft_batch_hold_pass")

    @property
    def launches(self) -> int:
        return sft_batch_launch_count(self.h)

    @property
    def epoch_tasks(self) -> int:
        return sft_batch_epoch_tasks(self.h)
