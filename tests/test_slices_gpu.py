"""GPU parity of the slice-layout passes (CSF slices of one mode) against the
FP64 oracle, through the C ABI.

The factor pass on a slice layout runs every slice element by element in visit
order; since slices of one mode do not interact during a factor pass, it must
equal the oracle's element-by-element pass (batch 1) over the permutation
that built the layout.  Long slices split into affine maps are forced on with
small tiles.  The core pass over the layout is compared with the oracle's core
pass over the same order.
"""
import functools

import numpy as np
import pytest
import torch

from parity_util import (TOL32, assert_rows_within, assert_within, core_step_scale, np_idx,
                         rel_fro, small_tensor, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


def perm_of(seed, epoch, phase, mode, n):
    from paper_2210_06014_gb300 import synth
    return synth.pass_permutation(seed, epoch, phase, mode, n)


def slice_order(idx_np, n, perm):
    """Storage indices in slice order: sort visit positions by (i_n, position)."""
    rows = idx_np[n][perm]
    pos = np.arange(len(perm))
    order = np.lexsort((pos, rows))
    return perm[order], rows[order]


@pytest.fixture(scope="module")
def skewed():
    """A small Netflix-shaped tensor: Zipf(1.1) user / item modes (heavy slices)."""
    from paper_2210_06014_gb300 import synth
    spec = synth.spec_ratings(nnz=400_000, dims=(20_000, 3_000, 500))
    return synth.make_tensor(spec)


def test_group_slices_layout(sft):
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    for n in range(3):
        perm = perm_of(5, 0, 0, n, T.nnz)
        sl = dec.slices(n, idx, val, perm.cuda())
        dec.sync(60_000)
        order, rows = slice_order(ix, n, perm.numpy().astype(np.int64))
        for k in range(3):
            assert np.array_equal(sl.idx[k].cpu().numpy(), ix[k][order])
        assert np.array_equal(sl.val.cpu().numpy(), T.val.numpy()[order])
        want_ptr = np.searchsorted(rows, np.arange(T.spec.dims[n] + 1), side="left")
        assert np.array_equal(sl.row_ptr.cpu().numpy(), want_ptr)


def test_expand_rows_equals_layout(sft, skewed):
    """sft_slices_expand_rows rebuilds a layout's own-mode coordinate array from
    row_ptr: the same int32 array sft_group_slices wrote (Zipf slices of tens of
    thousands of nonzeros, empty slices, and a layout whose bad coordinates
    sit after the last slice as -1)."""
    T = skewed
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0)
    for n in range(3):
        sl = dec.slices(n, idx, val, None)
        out = torch.full_like(sl.idx[n], 12345)
        sft.sft_slices_expand_rows(dec.ctx, n, sl.row_ptr, sl.nnz, out)
        dec.sync(60_000)
        assert torch.equal(out, sl.idx[n]), n
    # a coordinate out of range: moved behind the last slice by the layout
    bad = [t.clone() for t in idx]
    bad[0][::97] = T.spec.dims[0] + 5
    sl = dec.slices(0, bad, val, None)
    out = torch.full_like(sl.idx[0], 12345)
    sft.sft_slices_expand_rows(dec.ctx, 0, sl.row_ptr, sl.nnz, out)
    with pytest.raises(sft.SftError):
        dec.sync(60_000)  # the layout build reports the bad coordinates
    assert torch.equal(out, sl.idx[0])
    assert int((out == -1).sum()) == len(range(0, T.nnz, 97))


def test_fibers_expand_coords_equals_layout(sft, skewed):
    """sft_fibers_expand_coords rebuilds a layout's other-mode coordinate arrays
    from fid and fcoord: the same int32 arrays sft_group_slices wrote, for every
    mode of a Zipf tensor; a position outside every fiber (fid -1, as
    sft_group_fibers marks bad data, or fid >= nfibers) gets -1."""
    T = skewed
    idx, val = to_dev(T)
    N = len(idx)
    dec = sft.Decomposition(T.A0, T.B0)
    for n in range(N):
        sl = dec.slices(n, idx, val, None)
        sl.build_fibers(dec)
        out = [None if k == n else torch.full_like(sl.idx[k], 12345) for k in range(N)]
        sft.sft_fibers_expand_coords(dec.ctx, n, sl.fid, sl.nnz, sl.fcoord, sl.nfibers, out)
        dec.sync(60_000)
        for k in range(N):
            if k != n:
                assert torch.equal(out[k], sl.idx[k]), (n, k)
    # positions outside every fiber
    fid = sl.fid.clone()
    fid[::89] = -1
    fid[5::131] = sl.nfibers
    out = [torch.full_like(sl.idx[k], 12345) for k in range(N - 1)] + [None]
    sft.sft_fibers_expand_coords(dec.ctx, N - 1, fid, sl.nnz, sl.fcoord, sl.nfibers, out)
    dec.sync(60_000)
    badpos = (fid < 0) | (fid >= sl.nfibers)
    assert int(badpos.sum()) > 0
    for k in range(N - 1):
        assert torch.equal(out[k][~badpos], sl.idx[k][~badpos]), k
        assert bool((out[k][badpos] == -1).all()), k


@pytest.mark.parametrize("tiling", [(0, 0), (64, -1), (64, 1 << 30), (7, -1), (64, 300), (32, 40)])
def test_factor_slices_equal_sequential_pass(sft, oracle_mod, tiling):
    """Slice pass == oracle element-by-element pass over the same permutation,
    for every mode and with the long-slice maps forced on or off."""
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    dec.set_slice_tiling(*tiling)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        perm = perm_of(7, 0, 0, n, T.nnz)
        A0 = dec.A[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, perm.cuda())
        dec.update_factors_slices(sl, lr=0.05, lam=0.01)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(),
                                        perm=perm.numpy().astype(np.uint32), batch=1, lr=0.05,
                                        lam=0.01)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert_rows_within(got, ref.A[n], S1, S2, what=f"tiling {tiling} A^({n})")
        assert rel_fro(got - A0, ref.A[n] - A0) < 1e-4, n
        assert rel_fro(got, ref.A[n]) < TOL32, n
        # keep both sides on the same parameters for the next mode
        dec.A[n].copy_(torch.from_numpy(ref.A[n].astype(np.float32)))
        dec.refresh(n)
        ref.A[n] = ref.A[n].astype(np.float32).astype(np.float64)
        ref.refresh(n)


def test_factor_slices_skewed_tensor(sft, oracle_mod, skewed):
    """Heavy Zipf slices (tens of thousands of nonzeros) go through the map
    path; the pass still equals the sequential oracle pass."""
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    counts = np.bincount(ix[0], minlength=T.spec.dims[0])
    assert counts.max() > 10_000
    for n in range(3):
        A0 = dec.A[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, None)
        dec.update_factors_slices(sl, lr=0.01, lam=0.01)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(), perm=None, batch=1, lr=0.01,
                                        lam=0.01)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        worst = assert_rows_within(got, ref.A[n], S1, S2, what=f"skewed A^({n})")
        print(f"skewed mode {n}: worst err/bound {worst:.3g}")
        assert rel_fro(got - A0, ref.A[n] - A0) < 1e-4, n
        assert rel_fro(got, ref.A[n]) < TOL32, n


HIGH_ORDER = {
    # name: (order, dim, nnz, J, lr) -- planted std(x) ~ 1 (synth.spec_order).
    # Per-element SGD is stable while lr |v|^2 < 2; the products of 7 cached
    # rows are heavy-tailed (max |v|^2 ~ 6e3 on the order-8 J=32 case), so lr
    # is chosen under 2 / max |v|^2 (the oracle diverges too above it).
    "order5_J16": (5, 60, 30_011, 16, 0.002),
    "order8_J32": (8, 30, 20_003, 32, 1e-4),
    "order8_J8": (8, 12, 40_000, 8, 0.002),
}


@functools.lru_cache(maxsize=None)
def high_order_tensor(name):
    from paper_2210_06014_gb300 import synth
    order, dim, nnz, J, _ = HIGH_ORDER[name]
    return synth.make_tensor(synth.spec_order(order, dim, nnz, J, seed=4))


@pytest.mark.parametrize("tiling", [(0, 0), (32, 1 << 30)])
@pytest.mark.parametrize("name", list(HIGH_ORDER))
def test_high_order_slice_passes(sft, oracle_mod, name, tiling):
    """Orders 5 and 8 (the 7-other-mode kernels): the element-by-element factor
    pass of every mode equals the oracle's sequential pass, with the long
    slices as maps (automatic tiling) or as chains, and a whole-pass core step
    per mode matches the oracle."""
    T = high_order_tensor(name)
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    N = len(ix)
    lr = HIGH_ORDER[name][4]
    dec = sft.Decomposition(T.A0, T.B0)
    dec.set_slice_tiling(*tiling)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(N):
        perm = perm_of(11, 0, 0, n, T.nnz)
        A0 = dec.A[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, perm.cuda())
        dec.update_factors_slices(sl, lr=lr, lam=0.01)
        dec.refresh(n)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(),
                                        perm=perm.numpy().astype(np.uint32), batch=1, lr=lr,
                                        lam=0.01)
        ref.refresh(n)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got)), n
        assert_rows_within(got, ref.A[n], S1, S2, what=f"{name} {tiling} A^({n})")
        # A row takes L = nnz / I_n dependent float32 steps on average; the
        # slice path re-associates them (maps, products of maps), so its
        # rounding is bounded by a small multiple of L u (u = 2^-24) relative
        # to the row, i.e. tol * |A| / |dA| relative to the increment.
        tol = 4 * (T.nnz / T.spec.dims[n]) * 2.0 ** -24
        inc = np.linalg.norm(ref.A[n] - A0)
        assert rel_fro(got, ref.A[n]) < tol, (n, rel_fro(got, ref.A[n]), tol)
        assert rel_fro(got - A0, ref.A[n] - A0) < tol * np.linalg.norm(ref.A[n]) / inc, n
    # the core steps start from the same parameters on both sides
    for n in range(N):
        dec.A[n].copy_(torch.from_numpy(ref.A[n].astype(np.float32)))
        ref.A[n] = ref.A[n].astype(np.float32).astype(np.float64)
    dec.refresh(-1)
    ref.refresh_all()
    for n in range(N):
        B0 = dec.B[n].cpu().numpy().astype(np.float64)
        A_now = [a.copy() for a in ref.A]
        B_now = [b.copy() for b in ref.B]
        sl = dec.slices(n, idx, val, None)
        dec.update_core_slices(sl, batch=T.nnz, lr=0.5, lam=0.01)
        dec.refresh(n)
        dec.sync(60_000)
        ref.core_pass(n, ix, T.val.numpy(), batch=T.nnz, lr=0.5, lam=0.01)
        ref.refresh(n)
        got = dec.B[n].cpu().numpy().astype(np.float64)
        scale = core_step_scale(A_now, B_now, n, ix, T.val.numpy(), np.arange(T.nnz), 0.5, 0.01)
        assert_within(got - B0, ref.B[n] - B0, scale + 1e-2 * np.abs(ref.B[n]),
                      what=f"{name} core step B^({n})")
        # keep both sides on the same B for the next mode
        dec.B[n].copy_(torch.from_numpy(ref.B[n].astype(np.float32)))
        ref.B[n] = ref.B[n].astype(np.float32).astype(np.float64)
        dec.refresh(n)
        ref.refresh(n)


@pytest.mark.parametrize("n", [0, 1, 2])
def test_core_slices_one_step_gradient(sft, oracle_mod, n):
    """Whole-pass core step on the layout (Algorithm 5) with lr = 1: B moves by
    G / nnz - lam B."""
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    lr, lam = 1.0, 0.01
    dec = sft.Decomposition(T.A0, T.B0)
    B_before = dec.B[n].cpu().numpy().astype(np.float64)
    sl = dec.slices(n, idx, val, None)
    dec.update_core_slices(sl, batch=T.nnz, lr=lr, lam=lam)
    dec.sync(60_000)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    ref.core_pass(n, ix, T.val.numpy(), batch=T.nnz, lr=lr, lam=lam)
    got = dec.B[n].cpu().numpy().astype(np.float64) - B_before
    want = ref.B[n] - B_before
    scale = core_step_scale(ref.A, [b.numpy().astype(np.float64) for b in T.B0], n, ix,
                            T.val.numpy(), np.arange(T.nnz), lr, lam)
    assert_within(got, want, scale + 1e-2 * np.abs(ref.B[n]), what=f"step B^({n})")
    assert rel_fro(got, want) < TOL32


def test_core_slices_minibatches(sft, oracle_mod):
    """Minibatches of 4096 consecutive layout positions, the last one ragged."""
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    n = 1
    perm = perm_of(9, 0, 1, n, T.nnz)
    dec = sft.Decomposition(T.A0, T.B0)
    sl = dec.slices(n, idx, val, perm.cuda())
    dec.update_core_slices(sl, batch=4096, lr=0.05, lam=0.01)
    dec.sync(60_000)
    order, _ = slice_order(ix, n, perm.numpy().astype(np.int64))
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    ref.core_pass(n, ix, T.val.numpy(), perm=order.astype(np.uint32), batch=4096, lr=0.05,
                  lam=0.01)
    B0 = T.B0[n].numpy().astype(np.float64)
    got = dec.B[n].cpu().numpy().astype(np.float64)
    assert rel_fro(got - B0, ref.B[n] - B0) < 1e-4
    assert rel_fro(got, ref.B[n]) < TOL32


def _slice_epochs(sft, oracle_mod, T, epochs, lr=0.01, core_batch=4096):
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    xv = T.val.numpy()
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    got, want = [], []
    N = len(ix)
    for ep in range(epochs):
        pf = [perm_of(0, ep, 0, n, T.nnz) for n in range(N)]
        pc = [perm_of(0, ep, 1, n, T.nnz) for n in range(N)]
        for n in range(N):
            sl = dec.slices(n, idx, val, pf[n].cuda())
            dec.update_factors_slices(sl, lr=lr, lam=0.01)
            dec.refresh(n)
        for n in range(N):
            sl = dec.slices(n, idx, val, pc[n].cuda())
            dec.update_core_slices(sl, batch=core_batch, lr=lr, lam=0.01)
            dec.refresh(n)
        got.append(dec.rmse(idx, val))
        core_orders = [slice_order(ix, n, pc[n].numpy().astype(np.int64))[0].astype(np.uint32)
                       for n in range(N)]
        ref.epoch(ix, xv, [p.numpy().astype(np.uint32) for p in pf], core_orders,
                  batch_factor=1, batch_core=core_batch, lr_A=lr, lam_A=0.01, lr_B=lr,
                  lam_B=0.01)
        want.append(ref.rmse(ix, xv))
    return np.array(got), np.array(want), dec, ref


def test_slice_epochs_rmse(sft, oracle_mod):
    """5 epochs of Algorithm 2 on slice layouts (factor rows element by
    element, core minibatches of 4096): training RMSE within 1 % per epoch."""
    T = small_tensor()
    got, want, dec, ref = _slice_epochs(sft, oracle_mod, T, 5)
    np.testing.assert_allclose(got, want, rtol=0.01)
    for n in range(3):
        assert rel_fro(dec.A[n].cpu().numpy(), ref.A[n]) < 1e-4
        assert rel_fro(dec.B[n].cpu().numpy(), ref.B[n]) < 1e-4


def test_slice_epochs_skewed_rmse(sft, oracle_mod, skewed):
    """Two epochs on the Zipf tensor with one core update per pass: the slice
    path stays finite and tracks the oracle (the minibatch and Hogwild rules
    diverge here at this learning rate)."""
    got, want, _, _ = _slice_epochs(sft, oracle_mod, skewed, 2, lr=0.01, core_batch=skewed.nnz)
    assert np.all(np.isfinite(want))
    np.testing.assert_allclose(got, want, rtol=0.01)


def test_slices_bitwise_reproducible(sft, skewed):
    T = skewed
    idx, val = to_dev(T)
    outs = []
    for _ in range(2):
        dec = sft.Decomposition(T.A0, T.B0)
        for n in range(3):
            sl = dec.slices(n, idx, val, None)
            dec.update_factors_slices(sl, lr=0.01, lam=0.01)
            dec.refresh(n)
            dec.update_core_slices(sl, lr=0.01, lam=0.01)
            dec.refresh(n)
        dec.sync(60_000)
        outs.append([t.clone() for t in dec.A + dec.B])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


# ----------------------------------------------------------------------------- bfloat16 cached products

TOL_BF16 = 2e-2


def test_bf16_refresh_and_predictions(sft, oracle_mod):
    """C stored in bfloat16: C and predictions within 2e-2 of the float64 oracle
    (condition-aware); the measured worst ratio is printed as the result's error."""
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    from parity_util import abs_C, pred_scale
    absC = abs_C(ref.A, ref.B)
    worst = 0.0
    for n in range(3):
        got = dec.C[n].float().cpu().numpy()
        assert_within(got, ref.C[n], absC[n], tol=TOL_BF16, what=f"bf16 C^({n})")
        worst = max(worst, float(np.max(np.abs(got - ref.C[n]) / (absC[n] + 1e-30))))
    ix = np_idx(T.idx)
    xh = dec.predict(idx).cpu().numpy()
    scale = pred_scale(absC, ix)
    assert_within(xh, ref.predict(ix), scale, tol=TOL_BF16, what="bf16 x^")
    print(f"bf16: worst |C err|/|A||B| = {worst:.3e}, "
          f"worst |x^ err|/scale = {float(np.max(np.abs(xh - ref.predict(ix)) / scale)):.3e}")


@pytest.mark.parametrize("fibers", [False, True])
def test_bf16_slice_passes(sft, oracle_mod, fibers):
    """One factor pass (element by element) and one whole-pass core step per mode
    with bfloat16 cached products track the float64 oracle within 2e-2; with
    fibers the v table itself is stored in bfloat16."""
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16)
    dec.set_slice_tiling(64, 128)  # heads, maps and chains all in use
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        A0 = dec.A[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, None)
        if fibers:
            sl.build_fibers(dec)
        dec.update_factors_slices(sl, lr=0.05, lam=0.01)
        dec.refresh(n)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(), batch=1, lr=0.05, lam=0.01)
        ref.refresh(n)
        dec.sync(60_000)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        worst = assert_rows_within(got, ref.A[n], S1, S2, tol=TOL_BF16, what=f"bf16 A^({n})")
        print(f"bf16 factor pass mode {n}: worst err/bound {worst:.3g}")
        assert rel_fro(got - A0, ref.A[n] - A0) < TOL_BF16, n
    for n in range(3):
        B0 = dec.B[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, None)
        dec.update_core_slices(sl, batch=T.nnz, lr=1.0, lam=0.01)
        dec.refresh(n)
        ref.core_pass(n, ix, T.val.numpy(), batch=T.nnz, lr=1.0, lam=0.01)
        ref.refresh(n)
        dec.sync(60_000)
        got = dec.B[n].cpu().numpy().astype(np.float64)
        assert rel_fro(got - B0, ref.B[n] - B0) < TOL_BF16, n


def test_bf16_epochs_rmse(sft, oracle_mod, skewed):
    """Two epochs on the Zipf tensor with bfloat16 cached products: training RMSE
    within 1 % of the float64 oracle per epoch."""
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    xv = T.val.numpy()
    dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    lays = [dec.slices(n, idx, val, None) for n in range(3)]
    for ep in range(2):
        for n in range(3):
            dec.update_factors_slices(lays[n], lr=0.01, lam=0.01)
            dec.refresh(n)
        for n in range(3):
            dec.update_core_slices(lays[n], lr=0.01, lam=0.01)
            dec.refresh(n)
        ref.epoch(ix, xv, None, None, batch_factor=1, batch_core=T.nnz)
        got, want = dec.rmse(idx, val), ref.rmse(ix, xv)
        assert abs(got / want - 1) < 0.01, (ep, got, want)


# ----------------------------------------------------------------------------- fiber-shared v


@functools.lru_cache(maxsize=None)
def dense_small(order=3, dims=(30, 20, 10), nnz=3000, J=8, seed=5):
    """A small, dense-ish tensor: every fiber of every mode holds several nonzeros."""
    from paper_2210_06014_gb300 import synth
    spec = synth.TensorSpec(f"dense{order}", dims, nnz, (J,) * order, J, ("uniform",) * order,
                            values="planted", planted_sigma=0.4, noise_sigma=0.01, seed=seed)
    return synth.make_tensor(spec)


def test_fiber_layout(sft):
    """fid groups exactly the positions that share the other modes' coordinates,
    fcoord holds each fiber's tuple, and the count is the number of distinct
    tuples."""
    T = dense_small()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0)
    for n in range(3):
        sl = dec.slices(n, idx, val, None)
        nf = sl.build_fibers(dec)
        sidx = [i.cpu().numpy().astype(np.int64) for i in sl.idx]
        others = [k for k in range(3) if k != n]
        tup = np.stack([sidx[k] for k in others], axis=1)
        uniq, inv = np.unique(tup, axis=0, return_inverse=True)
        assert nf == len(uniq)
        fid = sl.fid.cpu().numpy()[:T.nnz]
        assert fid.min() >= 0 and fid.max() < nf
        # same tuple <-> same fiber id
        pairs = set(zip(inv.ravel().tolist(), fid.tolist()))
        assert len(pairs) == nf
        fc = np.stack([sl.fcoord[k].cpu().numpy()[:nf] for k in others], axis=1)
        assert np.array_equal(fc[fid], tup)


@pytest.mark.parametrize("case", ["dense_tiled", "dense_maps", "dense_chains", "small", "order5",
                                  "bf16"])
def test_fiber_pass_equals_row_pass(sft, case):
    """The factor pass with v formed once per fiber gives the same bits as the
    per-nonzero path (same operations in the same order), for every mode."""
    prec = sft.SFT_BF16 if case == "bf16" else sft.SFT_FP32
    tiling = {"dense_tiled": (0, 0), "dense_maps": (32, -1), "dense_chains": (32, 1 << 30),
              "small": (0, 0), "order5": (32, -1), "bf16": (32, -1)}[case]
    if case == "small":
        T = small_tensor()
    elif case == "order5":
        T = high_order_tensor("order5_J16")
    else:
        T = dense_small()
    idx, val = to_dev(T)
    N = len(idx)
    outs = []
    for use_fibers in (False, True):
        dec = sft.Decomposition(T.A0, T.B0, prec=prec)
        dec.set_slice_tiling(*tiling)
        dec.set_blocked_chains(False)  # element by element on both sides
        for n in range(N):
            sl = dec.slices(n, idx, val, None)
            if use_fibers:
                sl.build_fibers(dec)
            dec.update_factors_slices(sl, lr=0.002, lam=0.01)
            dec.refresh(n)
        dec.sync(60_000)
        outs.append([a.clone() for a in dec.A])
    for n, (a, b) in enumerate(zip(*outs)):
        if case == "bf16":
            # with bfloat16 cached products the fiber table stores v rounded to
            # bfloat16 (the per-nonzero path keeps v in float32): one bfloat16
            # rounding of v apart, far inside the 2e-2 bfloat16 bound
            assert rel_fro(b.cpu().numpy(), a.cpu().numpy()) < 2e-3, (case, n)
            continue
        assert torch.equal(a, b), (case, n, (a - b).abs().max().item())


def test_fiber_pass_on_skewed_tensor_matches_oracle(sft, oracle_mod, skewed):
    """Zipf slices (maps) with fibers: equal to the element-by-element oracle pass."""
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        A0 = dec.A[n].cpu().numpy().astype(np.float64)
        sl = dec.slices(n, idx, val, None)
        nf = sl.build_fibers(dec)
        assert 0 < nf <= T.nnz
        dec.update_factors_slices(sl, lr=0.01, lam=0.01)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(), perm=None, batch=1, lr=0.01,
                                        lam=0.01)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert_rows_within(got, ref.A[n], S1, S2, what=f"fibers skewed A^({n})")
        assert rel_fro(got - A0, ref.A[n] - A0) < 1e-4, n
        assert rel_fro(got, ref.A[n]) < TOL32, n


@pytest.mark.parametrize("case", ["dense", "small_batches", "order5", "bf16"])
def test_fiber_core_pass_equals_row_pass(sft, case):
    """The core pass with p read from the per-fiber table gives the same bits as
    the per-nonzero path, whole-pass and in minibatches."""
    prec = sft.SFT_BF16 if case == "bf16" else sft.SFT_FP32
    T = {"dense": dense_small(), "small_batches": small_tensor(),
         "order5": high_order_tensor("order5_J16"), "bf16": dense_small()}[case]
    batch = 4096 if case == "small_batches" else None
    idx, val = to_dev(T)
    N = len(idx)
    outs = []
    for use_fibers in (False, True):
        dec = sft.Decomposition(T.A0, T.B0, prec=prec)
        for n in range(N):
            sl = dec.slices(n, idx, val, None)
            if use_fibers:
                sl.build_fibers(dec, core=True)
            dec.update_core_slices(sl, batch=batch, lr=0.5, lam=0.01)
            dec.refresh(n)
        dec.sync(60_000)
        outs.append([b.clone() for b in dec.B])
    for n, (a, b) in enumerate(zip(*outs)):
        assert torch.equal(a, b), (case, n, (a - b).abs().max().item())


@pytest.mark.parametrize("tiling", [(0, 0), (64, -1), (64, 1 << 30), (0, 8192)])
def test_fiber_passes_read_no_other_coordinates(sft, skewed, tiling):
    """With fiber tables for both passes, a mode's factor and core passes read
    the other modes only through fid / fcoord (Eq. (12)-(13)): replacing the
    layout's other-mode coordinate arrays by different in-range values leaves
    every bit of A and B unchanged, on the tiled, map, chain and blocked-chain
    paths."""
    T = skewed
    idx, val = to_dev(T)
    N = len(idx)
    outs = []
    for scramble in (False, True):
        dec = sft.Decomposition(T.A0, T.B0)
        dec.set_slice_tiling(*tiling)
        for n in range(N):
            sl = dec.slices(n, idx, val, None)
            sl.build_fibers(dec, core=True)
            if scramble:
                for k in range(N):
                    if k != n:
                        sl.idx[k].copy_(torch.roll(sl.idx[k], 7919))
            dec.update_factors_slices(sl, lr=0.01, lam=0.01)
            dec.refresh(n)
            dec.update_core_slices(sl, lr=0.01, lam=0.01)
            dec.refresh(n)
        dec.sync(60_000)
        outs.append([t.clone() for t in list(dec.A) + list(dec.B)])
    for q, (a, b) in enumerate(zip(*outs)):
        assert torch.equal(a, b), (tiling, q, (a - b).abs().max().item())


@pytest.mark.parametrize("fibers", [False, True])
def test_slice_autotune_leaves_A_and_keeps_parity(sft, oracle_mod, skewed, fibers):
    """sft_autotune_slices restores A^(n) after its trials, returns one of its
    candidates, and the pass it selects still equals the sequential oracle."""
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        sl = dec.slices(n, idx, val, None)
        if fibers:
            sl.build_fibers(dec)
        A0 = dec.A[n].clone()
        L = dec.autotune_slices(sl, lr=0.01, lam=0.01)
        dec.sync(60_000)
        assert torch.equal(dec.A[n], A0)
        W = max(32, min(2048, T.nnz // (torch.cuda.get_device_properties(0).multi_processor_count * 1024)))
        pows = [1024 << k for k in range(7)]
        assert L in (W, 2 * W, 1 << 40) or L in pows or L in [3 * p // 2 for p in pows[:-1]]
        dec.update_factors_slices(sl, lr=0.01, lam=0.01)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(), perm=None, batch=1, lr=0.01,
                                        lam=0.01)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert_rows_within(got, ref.A[n], S1, S2, what=f"autotuned (fibers={fibers}) A^({n})")
        A0n = A0.cpu().numpy().astype(np.float64)
        assert rel_fro(got - A0n, ref.A[n] - A0n) < 1e-4, n
        assert rel_fro(got, ref.A[n]) < TOL32, n


def test_subslice_mode_epochs_rmse(sft, oracle_mod):
    """Long slices as concurrent sub-slices (SFT_LONG_SUBSLICES, the paper's
    B-CSF manner; Hogwild within a row): with short tiles every slice of the
    small tensor is long and cut into sub-slices of at most 32 nonzeros.  Only
    the per-epoch training RMSE is checked (within 1 % of the oracle's
    element-by-element epochs), as for every Hogwild path."""
    T = small_tensor()
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    xv = T.val.numpy()
    dec = sft.Decomposition(T.A0, T.B0)
    dec.set_slice_tiling(32, 64)
    dec.set_long_slices(sft.SFT_LONG_SUBSLICES)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    lays = [dec.slices(n, idx, val, None) for n in range(3)]
    for lay in lays:
        lay.build_fibers(dec)
    got, want = [], []
    for ep in range(3):
        for n in range(3):
            dec.update_factors_slices(lays[n], lr=0.01, lam=0.01)
            dec.refresh(n)
        for n in range(3):
            dec.update_core_slices(lays[n], lr=0.01, lam=0.01)
            dec.refresh(n)
        ref.epoch(ix, xv, None, None, batch_factor=1, batch_core=T.nnz)
        got.append(dec.rmse(idx, val))
        want.append(ref.rmse(ix, xv))
    print("sub-slice epochs rmse gpu", got, "oracle", want)
    np.testing.assert_allclose(got, want, rtol=0.01)


@pytest.mark.parametrize("tiling", [(64, 1 << 30), (0, 8192), (32, 4100)])
def test_blocked_chains_match_oracle(sft, oracle_mod, skewed, tiling):
    """Chains of 4096 or more nonzeros run 32 at a time (Gram block on the tensor
    cores + triangular solve): every row within the per-row rounding bound of
    the oracle's sequential pass.  (64, 1 << 30): every crossing slice whole
    (the Zipf heads of the user and item modes hold 10k+ nonzeros); (0, 8192):
    heads of 8192 before the maps; (32, 4100): heads of 4100 (not a multiple
    of 32) before the maps."""
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    dec.set_slice_tiling(*tiling)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        sl = dec.slices(n, idx, val, None)
        sl.build_fibers(dec)
        dec.update_factors_slices(sl, lr=0.01, lam=0.01)
        dec.refresh(n)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(), perm=None, batch=1, lr=0.01,
                                        lam=0.01)
        ref.refresh(n)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        worst = assert_rows_within(got, ref.A[n], S1, S2, what=f"blocked {tiling} A^({n})")
        print(f"blocked chains {tiling} mode {n}: worst err/bound {worst:.3g}")


def test_csf_order_pass_matches_oracle(sft, oracle_mod, skewed):
    """Slices laid out in the B-CSF traversal order (each slice sorted by the
    other modes' coordinates, synth.csf_order) with fibers, blocked chains and
    maps: every row within the per-row bound of the oracle's sequential pass
    over the same order."""
    from paper_2210_06014_gb300 import synth
    T = skewed
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    for n in range(3):
        order = synth.csf_order(idx, n)
        sl = dec.slices(n, idx, val, order)
        sl.build_fibers(dec)
        dec.update_factors_slices(sl, lr=0.01, lam=0.01)
        dec.refresh(n)
        dec.sync(60_000)
        S1, S2 = ref.factor_pass_scaled(n, ix, T.val.numpy(),
                                        perm=order.cpu().numpy().astype(np.uint32), batch=1,
                                        lr=0.01, lam=0.01)
        ref.refresh(n)
        got = dec.A[n].cpu().numpy().astype(np.float64)
        assert_rows_within(got, ref.A[n], S1, S2, what=f"csf order A^({n})")
