"""FP64 CPU oracle of sparse FastTucker SGD (test infrastructure only).

The arithmetic lives in ``sft_oracle.c`` (plain C, double precision, single
thread).  This module compiles it with gcc and marshals numpy arrays through
ctypes.  Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it; the CUDA library never does.

Passages followed (cuFasterTucker, arXiv 2210.06014): Eq. (1) and Eq. (12) for
the model and its per-nonzero evaluation, Algorithm 3 for the cached products
C^(n) = A^(n) B^(n), Eq. (9)-(11) for the SGD steps, Algorithm 2 for the epoch
schedule, Section "Real-world accuracy" for RMSE / MAE.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sft_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "libsft_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)
_pp_d = ctypes.POINTER(_dp)
_pp_i32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_int32))
_pp_u32 = ctypes.POINTER(ctypes.POINTER(ctypes.c_uint32))


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/libsft_oracle.so`` (gcc, -O2).

    FP contraction is switched off so that x86 and Arm hosts round alike."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, i32, d = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            ip64 = ctypes.POINTER(ctypes.c_int64)
            ip32 = ctypes.POINTER(ctypes.c_int)
            fp = ctypes.POINTER(ctypes.c_float)
            up = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_refresh.argtypes = [i64, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]
            lib.orc_refresh.restype = None
            lib.orc_predict_cached.argtypes = [ctypes.c_int, ctypes.c_int, _pp_d, _pp_i32, i64, _dp]
            lib.orc_predict_cached.restype = None
            lib.orc_predict_direct.argtypes = [ctypes.c_int, ip32, ctypes.c_int, _pp_d, _pp_d,
                                               _pp_i32, i64, _dp]
            lib.orc_predict_direct.restype = None
            pass_args = [ctypes.c_int, ip64, ip32, ctypes.c_int, ctypes.c_int, _pp_d, _pp_d, _pp_d,
                         _pp_i32, fp, up, i64, i64, d, d]
            lib.orc_factor_pass.argtypes = pass_args
            lib.orc_factor_pass.restype = ctypes.c_int
            lib.orc_core_pass.argtypes = pass_args
            lib.orc_core_pass.restype = ctypes.c_int
            lib.orc_factor_pass_scaled.argtypes = pass_args + [_dp]
            lib.orc_factor_pass_scaled.restype = ctypes.c_int
            lib.orc_loss.argtypes = [ctypes.c_int, ctypes.c_int, _pp_d, _pp_i32, fp, i64, _dp, _dp]
            lib.orc_loss.restype = None
            lib.orc_loss_grad.argtypes = [ctypes.c_int, ip64, ip32, ctypes.c_int, _pp_d, _pp_d,
                                          _pp_d, _pp_i32, fp, i64, _pp_d, _pp_d]
            lib.orc_loss_grad.restype = ctypes.c_double
            lib.orc_epoch.argtypes = [ctypes.c_int, ip64, ip32, ctypes.c_int, _pp_d, _pp_d, _pp_d,
                                      _pp_i32, fp, i64, _pp_u32, _pp_u32, i64, i64, d, d, d, d]
            lib.orc_epoch.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _ptr_d(a):
    return a.ctypes.data_as(_dp)


def _ptr_array(arrs, ctype):
    arr_t = ctypes.POINTER(ctype) * len(arrs)
    return arr_t(*[a.ctypes.data_as(ctypes.POINTER(ctype)) for a in arrs])


class Model:
    """FP64 copy of the parameters: factor matrices A[n] (I_n x J_n), core
    matrices B[n] (J_n x R) and the cached products C[n] = A[n] B[n] (I_n x R),
    all row-major numpy arrays owned by this object."""

    def __init__(self, A, B):
        self.A = [_f64(a).copy() for a in A]
        self.B = [_f64(b).copy() for b in B]
        self.N = len(self.A)
        self.R = int(self.B[0].shape[1])
        self.I = np.array([a.shape[0] for a in self.A], dtype=np.int64)
        self.J = np.array([a.shape[1] for a in self.A], dtype=np.int32)
        for n in range(self.N):
            assert self.B[n].shape == (self.J[n], self.R)
        self.C = [np.zeros((int(self.I[n]), self.R)) for n in range(self.N)]
        self.refresh_all()

    def refresh(self, n: int) -> None:
        lib = _load()
        lib.orc_refresh(int(self.I[n]), int(self.J[n]), self.R, _ptr_d(self.A[n]),
                        _ptr_d(self.B[n]), _ptr_d(self.C[n]))

    def refresh_all(self) -> None:
        for n in range(self.N):
            self.refresh(n)

    # -- marshalling helpers -------------------------------------------------
    def _arrays(self):
        return (_ptr_array(self.A, ctypes.c_double), _ptr_array(self.B, ctypes.c_double),
                _ptr_array(self.C, ctypes.c_double))

    @staticmethod
    def _coo(idx, val):
        idx = [np.ascontiguousarray(i, dtype=np.int32) for i in idx]
        val = np.ascontiguousarray(val, dtype=np.float32)
        return idx, val

    # -- method ----------------------------------------------------------------
    def predict(self, idx) -> np.ndarray:
        """x^ for every nonzero through the cached products (Eq. (12))."""
        idx = [np.ascontiguousarray(i, dtype=np.int32) for i in idx]
        nnz = len(idx[0])
        out = np.empty(nnz, dtype=np.float64)
        _, _, C = self._arrays()
        _load().orc_predict_cached(self.N, self.R, C, _ptr_array(idx, ctypes.c_int32), nnz,
                                   _ptr_d(out))
        return out

    def predict_direct(self, idx) -> np.ndarray:
        """x^ recomputed without the cache, as Algorithm 1 does."""
        idx = [np.ascontiguousarray(i, dtype=np.int32) for i in idx]
        nnz = len(idx[0])
        out = np.empty(nnz, dtype=np.float64)
        A, B, _ = self._arrays()
        J = np.ascontiguousarray(self.J, dtype=np.int32)
        _load().orc_predict_direct(self.N, J.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.R,
                                   A, B, _ptr_array(idx, ctypes.c_int32), nnz, _ptr_d(out))
        return out

    def _pass(self, fn, n, idx, val, perm, batch, lr, lam, *extra):
        idx, val = self._coo(idx, val)
        nnz = len(val)
        if perm is not None:
            perm = np.ascontiguousarray(perm, dtype=np.uint32)
            assert len(perm) == nnz
            pptr = perm.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
        else:
            pptr = None
        A, B, C = self._arrays()
        J = np.ascontiguousarray(self.J, dtype=np.int32)
        rc = fn(self.N, self.I.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                J.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.R, int(n), A, B, C,
                _ptr_array(idx, ctypes.c_int32), val.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                pptr, nnz, int(batch), float(lr), float(lam), *extra)
        if rc != 0:
            raise RuntimeError(f"oracle pass failed with code {rc}")

    def factor_pass(self, n, idx, val, perm=None, batch=1, lr=0.01, lam=0.01) -> None:
        """Update A[n] over every nonzero (Eq. (9)-(10)); C[n] is NOT refreshed."""
        self._pass(_load().orc_factor_pass, n, idx, val, perm, batch, lr, lam)

    def factor_pass_scaled(self, n, idx, val, perm=None, batch=1, lr=0.01, lam=0.01):
        """factor_pass, also returning the per-entry rounding scales (S1, S2) of
        the pass (I_n x J_n each): S1 = sum over the row's samples of
        lr ((|x| + |a|.|v|) |v|_j + lam |a_j|) with |v| built from |A| |B|, and
        S2 = sum over the row's samples of |a_j| as each step read it.  They
        bound the rounding of a float32 run of the same pass; A moves exactly
        as in factor_pass."""
        In, Jn = int(self.I[n]), int(self.J[n])
        scale = np.zeros(2 * In * Jn, dtype=np.float64)
        self._pass(_load().orc_factor_pass_scaled, n, idx, val, perm, batch, lr, lam,
                   _ptr_d(scale))
        return scale[:In * Jn].reshape(In, Jn), scale[In * Jn:].reshape(In, Jn)

    def core_pass(self, n, idx, val, perm=None, batch=1, lr=0.01, lam=0.01) -> None:
        """Update B[n] over every nonzero (Eq. (9), (11)); C[n] is NOT refreshed."""
        self._pass(_load().orc_core_pass, n, idx, val, perm, batch, lr, lam)

    def loss(self, idx, val):
        """(SSE, SAE) over the given nonzeros with the cached products."""
        idx, val = self._coo(idx, val)
        sse = ctypes.c_double()
        sae = ctypes.c_double()
        _, _, C = self._arrays()
        _load().orc_loss(self.N, self.R, C, _ptr_array(idx, ctypes.c_int32),
                         val.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(val),
                         ctypes.byref(sse), ctypes.byref(sae))
        return sse.value, sae.value

    def loss_grad(self, idx, val):
        """(L, gA, gB): L = 1/2 sum e^2 over the nonzeros and its gradient with
        respect to every A[n] and B[n] (Eq. (10)/(11) without regularisation)."""
        idx, val = self._coo(idx, val)
        gA = [np.zeros_like(a) for a in self.A]
        gB = [np.zeros_like(b) for b in self.B]
        A, B, C = self._arrays()
        J = np.ascontiguousarray(self.J, dtype=np.int32)
        L = _load().orc_loss_grad(self.N, self.I.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                  J.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.R, A, B, C,
                                  _ptr_array(idx, ctypes.c_int32),
                                  val.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), len(val),
                                  _ptr_array(gA, ctypes.c_double), _ptr_array(gB, ctypes.c_double))
        return L, gA, gB

    def rmse(self, idx, val) -> float:
        sse, _ = self.loss(idx, val)
        return float(np.sqrt(sse / max(1, len(val))))

    def epoch(self, idx, val, perm_factor=None, perm_core=None, batch_factor=1, batch_core=1,
              lr_A=0.01, lam_A=0.01, lr_B=0.01, lam_B=0.01) -> None:
        """One epoch of Algorithm 2 (factor module over all modes, then core
        module over all modes, each pass followed by a refresh of its mode)."""
        idx, val = self._coo(idx, val)
        nnz = len(val)
        keep = []

        def perms(ps):
            if ps is None:
                return None
            arr = []
            for p in ps:
                if p is None:
                    arr.append(None)
                else:
                    p = np.ascontiguousarray(p, dtype=np.uint32)
                    keep.append(p)
                    arr.append(p.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)))
            return (ctypes.POINTER(ctypes.c_uint32) * self.N)(*arr)

        pf, pc = perms(perm_factor), perms(perm_core)
        A, B, C = self._arrays()
        J = np.ascontiguousarray(self.J, dtype=np.int32)
        rc = _load().orc_epoch(self.N, self.I.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                               J.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), self.R, A, B, C,
                               _ptr_array(idx, ctypes.c_int32),
                               val.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), nnz, pf, pc,
                               int(batch_factor), int(batch_core), float(lr_A), float(lam_A),
                               float(lr_B), float(lam_B))
        if rc != 0:
            raise RuntimeError(f"oracle epoch failed with code {rc}")
