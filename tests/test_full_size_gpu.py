"""Parity at the benchmark's full size, on sampled rows.

The ratings workload that bench.py times (480000 x 17800 x 2200, 100M
nonzeros, J = R = 16, float32 cached products) is built on the device with
the same slice layouts, fiber tables and autotuned chain lengths, and one
factor pass is run per mode.  The oracle cannot run a 90M-nonzero pass in
seconds, but during a factor pass of mode n a row of A^(n) depends only on
its own slice's nonzeros, taken in layout order, and on the other modes'
cached rows (Algorithm 4; Eq. (10)).  So sampled rows -- the longest slices
(heads run as chains, then affine maps over thousands of pieces), slices just
below and just above the chain limit, and random ones -- are recomputed in
float64 from the same starting parameters, and compared entry by entry with
the per-row rounding bound of the other slice tests.
"""
import numpy as np
import pytest
import torch

from parity_util import assert_rows_within

pytestmark = pytest.mark.gpu

LR, LAM = 0.01, 0.01


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


@pytest.fixture(scope="module")
def ratings_full():
    from paper_2210_06014_gb300 import synth
    return synth.make_tensor(synth.spec_ratings(), device="cuda")


def sample_rows(lengths, limit, rng):
    """Rows of the slices to check: the three longest, three just at or below
    the chain limit, three just above it, and five at random among the
    non-empty ones."""
    nz = np.flatnonzero(lengths > 0)
    order = nz[np.argsort(lengths[nz])]
    rows = list(order[-3:])
    below = nz[(lengths[nz] <= limit) & (lengths[nz] > limit // 2)]
    above = nz[(lengths[nz] > limit) & (lengths[nz] <= 2 * limit)]
    for pool in (below, above):
        if len(pool):
            rows += list(rng.choice(pool, size=min(3, len(pool)), replace=False))
    rows += list(rng.choice(nz, size=min(5, len(nz)), replace=False))
    return sorted(set(int(r) for r in rows))


@pytest.mark.parametrize("n", [0, 1, 2])
def test_full_size_factor_pass_sampled_rows(sft, oracle_mod, ratings_full, n):
    T = ratings_full
    N = len(T.idx)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=False, max_batch=4096)
    sl = dec.slices(n, T.idx, T.val, None)
    sl._scratch = None
    nf = sl.build_fibers(dec)
    if nf > T.nnz // 2:  # bench.py's fiber rule
        sl.drop_fibers()
    limit = dec.autotune_slices(sl, lr=LR, lam=LAM)  # restores A^(n)
    dec.sync(600_000)
    A0 = [a.cpu().numpy() for a in dec.A]
    B0 = [b.cpu().numpy() for b in dec.B]
    dec.update_factors_slices(sl, lr=LR, lam=LAM)
    dec.sync(600_000)
    got = dec.A[n].cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))

    row_ptr = sl.row_ptr.cpu().numpy().astype(np.int64)
    lengths = np.diff(row_ptr)
    lim = int(min(limit, lengths.max()))
    rows = sample_rows(lengths, max(lim, 1), np.random.default_rng(1234 + n))
    # the sampled slices' nonzeros, slice after slice, each in layout order
    pos = np.concatenate([np.arange(row_ptr[r], row_ptr[r + 1]) for r in rows])
    pos_t = torch.from_numpy(pos).cuda()
    sub_idx = [sl.idx[k][pos_t].cpu().numpy() for k in range(N)]
    sub_val = sl.val[pos_t].cpu().numpy()
    assert np.all(sub_idx[n] == np.repeat(rows, lengths[rows]))

    ref = oracle_mod.Model([a.astype(np.float32) for a in A0], [b.astype(np.float32) for b in B0])
    S1, S2 = ref.factor_pass_scaled(n, sub_idx, sub_val, perm=None, batch=1, lr=LR, lam=LAM)
    want = ref.A[n]
    worst = assert_rows_within(got[rows], want[rows], S1[rows], S2[rows],
                               what=f"full-size mode {n} rows {rows}")
    print(f"mode {n}: chain limit {limit}, longest slice {int(lengths.max())}, "
          f"{len(rows)} rows / {len(pos)} nonzeros checked, worst err/bound {worst:.3g}")
    # the rows were really moved by the pass
    assert np.any(np.abs(got[rows] - A0[n][rows]) > 0)
