"""Shared pieces of the GPU parity tests: seeded workloads, the two sides
(libsft on the GPU, the FP64 oracle on the CPU) and the error bounds.

Bounds are condition-aware: a float32 result r of a sum of products is
compared with the float64 oracle value through |r - r_ref| <= tol * S, where S
is the same sum taken over absolute values (the quantity that bounds the
rounding error of any summation order).  tol is 1e-5 for float32.
"""
from __future__ import annotations

import functools

import numpy as np
import torch

TOL32 = 1e-5


@functools.lru_cache(maxsize=None)
def small_tensor():
    """Order-3 1000x800x600, 200k nonzeros, planted J=R=8 (seed 0), CPU tensors."""
    from paper_2210_06014_gb300 import synth
    return synth.make_tensor(synth.spec_small())


def to_dev(T):
    idx = [i.cuda() for i in T.idx]
    val = T.val.cuda()
    return idx, val


def np_idx(idx):
    return [i.cpu().numpy().astype(np.int64) for i in idx]


def abs_C(A, B):
    return [np.abs(a) @ np.abs(b) for a, b in zip(A, B)]


def pred_scale(absC, idx):
    """sum_r prod_k |C|^(k)[i_k][r] per nonzero."""
    prod = None
    for k, ix in enumerate(idx):
        rows = absC[k][ix]
        prod = rows if prod is None else prod * rows
    return prod.sum(axis=1)


def factor_step_scale(A, B, n, idx, val, sel, lr, lam):
    """Per-row bound of one minibatch factor step over samples `sel`:
    lr * sum_s [(|x_s| + |a| . |v|_s) |v|_s + lam |a|], with |v|_s = |B^(n)| |p|_s."""
    absC = abs_C(A, B)
    p_abs = None
    for k in range(len(idx)):
        if k == n:
            continue
        rows = absC[k][idx[k][sel]]
        p_abs = rows if p_abs is None else p_abs * rows
    v_abs = p_abs @ np.abs(B[n]).T                    # M x J
    a_abs = np.abs(A[n][idx[n][sel]])                 # M x J
    xh_abs = np.sum(a_abs * v_abs, axis=1)
    term = (np.abs(val[sel].astype(np.float64)) + xh_abs)[:, None] * v_abs + lam * a_abs
    out = np.zeros_like(A[n])
    np.add.at(out, idx[n][sel], lr * term)
    return out


def core_step_scale(A, B, n, idx, val, sel, lr, lam):
    """Bound of one minibatch core step: lr * (sum_s |e|_s |a|_s |p|_s^T / M + lam |B|)."""
    absC = abs_C(A, B)
    p_abs = None
    for k in range(len(idx)):
        if k == n:
            continue
        rows = absC[k][idx[k][sel]]
        p_abs = rows if p_abs is None else p_abs * rows
    a_abs = np.abs(A[n][idx[n][sel]])
    xh_abs = np.sum(a_abs * (p_abs @ np.abs(B[n]).T), axis=1)
    e_abs = np.abs(val[sel].astype(np.float64)) + xh_abs
    G = (a_abs * e_abs[:, None]).T @ p_abs
    return lr * (G / len(sel) + lam * np.abs(B[n]))


def assert_within(got, want, scale, tol=TOL32, what=""):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    err = np.abs(got - want)
    bound = tol * np.asarray(scale, dtype=np.float64) + 1e-30
    bad = err > bound
    if bad.any():
        i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError(f"{what}: {bad.sum()} of {bad.size} entries beyond tol*scale; worst at "
                             f"{i}: got {got[i]!r} want {want[i]!r} scale {np.asarray(scale)[i]!r} "
                             f"(err/bound {float(err[i] / bound[i]):.3g})")


U32 = 2.0 ** -24  # unit roundoff of float32


def assert_rows_within(got, want, S1, S2, tol=TOL32, what=""):
    """Per-row, per-entry check of a whole factor pass against the oracle.

    S1, S2 come from the oracle's run of the same pass (factor_pass_scaled):
    S1 sums, over the row's samples, the magnitudes lr ((|x| + |a|.|v|)|v| +
    lam |a|) that every step's products and sums round against, and S2 sums
    |a| over the row's steps (each step's add to the row rounds against |a|).
    Errors made at one step are not amplified by later steps (each step scales
    a row by 1 - lr |v|^2 along v and by 1 - lr lam elsewhere, both at most 1
    in size at the learning rates used), so a float32 run -- element by element,
    or re-associated into products of affine maps -- stays within
    tol * S1 + 4 u * S2 of the float64 pass entry by entry (u = 2^-24; tol =
    1e-5 for float32 cached products, 2e-2 for bfloat16).  Rows a pass never
    visits must come back unchanged."""
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    bound = tol * np.asarray(S1) + 4.0 * U32 * np.asarray(S2) + 1e-30
    err = np.abs(got - want)
    ratio = err / bound
    if not (ratio <= 1.0).all():
        i = np.unravel_index(np.argmax(ratio), ratio.shape)
        bad_rows = int(np.any(ratio > 1.0, axis=1).sum())
        raise AssertionError(f"{what}: {bad_rows} rows leave their bound; worst at {i}: got "
                             f"{got[i]!r} want {want[i]!r} bound {bound[i]!r} "
                             f"(err/bound {float(ratio[i]):.3g})")
    return float(ratio.max())


def rel_fro(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    return float(np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300))


def grad_scale(A, B, idx, val):
    """Condition bounds of the summed loss gradient: with E_s = |x_s| + x^abs_s
    (a bound of |e_s|) and |p|_s the product of |C| rows of the other modes,
      dA[n][i][j] <= sum_{s: i_n(s)=i} E_s (|B^(n)| |p|_s)_j
      dB[n][j][r] <= sum_s E_s |a^(n)_{i_n(s)}|_j |p|_{s,r}
    and the loss L = 1/2 sum e^2 moves by at most sum_s E_s x^abs_s per unit
    of relative rounding."""
    absC = abs_C(A, B)
    N = len(A)
    xh_abs = pred_scale(absC, idx)
    E = np.abs(val.astype(np.float64)) + xh_abs
    sA, sB = [], []
    for n in range(N):
        p_abs = None
        for k in range(N):
            if k == n:
                continue
            rows = absC[k][idx[k]]
            p_abs = rows if p_abs is None else p_abs * rows
        v_abs = p_abs @ np.abs(B[n]).T
        out = np.zeros_like(A[n], dtype=np.float64)
        np.add.at(out, idx[n], E[:, None] * v_abs)
        sA.append(out)
        sB.append((np.abs(A[n][idx[n]]) * E[:, None]).T @ p_abs)
    return sA, sB, float(np.sum(E * xh_abs))


def stable_lr(T, cap=0.01, c=0.5):
    """A learning rate for per-element SGD that stays stable on tensor T at
    its initial parameters: one step scales a row along v by 1 - lr |v|^2, so
    lr is kept below c / max_s |v_s|^2 (over every nonzero and mode), and at
    most `cap`.  The products of N - 1 cached rows are heavy-tailed, so this
    matters from order 5 or R = 32 on."""
    A = [a.double() for a in T.A0]
    B = [b.double() for b in T.B0]
    C = [a @ b for a, b in zip(A, B)]
    vmax = 0.0
    N = len(A)
    for n in range(N):
        p = None
        for k in range(N):
            if k != n:
                rows = C[k][T.idx[k].long()]
                p = rows if p is None else p * rows
        v = p @ B[n].T
        vmax = max(vmax, float((v * v).sum(1).max()))
    return min(cap, c / vmax) if vmax > 0 else cap
