"""GPU parity of libsft against the FP64 oracle, through the C ABI.

Inputs are identical on both sides (seeded synthetic tensors, float32 initial
parameters, the same visit permutations).  Float32 results are checked with
condition-aware bounds at tol = 1e-5 (predictions, one-step factor and core
gradients), whole runs by the per-epoch training RMSE within 1 %.
"""
import numpy as np
import pytest
import torch

from parity_util import (TOL32, abs_C, assert_within, core_step_scale, factor_step_scale,
                         np_idx, pred_scale, rel_fro, small_tensor, to_dev,
                         assert_rows_within)

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


def rand_params(rng, dims, J, R, scale=0.4):
    A = [torch.from_numpy(rng.normal(0, scale, (i, j)).astype(np.float32)) for i, j in zip(dims, J)]
    B = [torch.from_numpy(rng.normal(0, scale, (j, R)).astype(np.float32)) for j in J]
    return A, B


def rand_coo(rng, dims, nnz):
    total = int(np.prod([float(d) for d in dims]))
    if total < 1e15:
        flat = rng.choice(int(total), size=nnz, replace=False)
        idx = [torch.from_numpy(i.astype(np.int32)) for i in np.unravel_index(flat, dims)]
    else:
        idx = [torch.from_numpy(rng.integers(0, d, nnz).astype(np.int32)) for d in dims]
    val = torch.from_numpy(rng.normal(0, 1, nnz).astype(np.float32))
    return idx, val


# ----------------------------------------------------------------------------- refresh


@pytest.mark.parametrize("J,R", [(8, 8), (16, 16), (32, 32), (4, 8), (32, 4), (8, 32), (16, 4)])
def test_refresh_parity(sft, oracle_mod, J, R):
    rng = np.random.default_rng(J * 100 + R)
    dims = (1031, 517, 77)  # ragged against every tile size
    A, B = rand_params(rng, dims, (J,) * 3, R)
    dec = sft.Decomposition(A, B)
    torch.cuda.synchronize()
    ref = oracle_mod.Model([a.numpy() for a in A], [b.numpy() for b in B])
    absC = abs_C(ref.A, ref.B)
    for n in range(3):
        assert_within(dec.C[n].cpu().numpy(), ref.C[n], absC[n], what=f"C^({n})")


# ----------------------------------------------------------------------------- prediction / loss


def test_predict_and_loss_parity(sft, oracle_mod):
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    xh = dec.predict(idx).cpu().numpy()
    ix = np_idx(T.idx)
    want = ref.predict(ix)
    scale = pred_scale(abs_C(ref.A, ref.B), ix)
    assert_within(xh, want, scale, what="x^")
    sse, sae = dec.loss(idx, val)
    rsse, rsae = ref.loss(ix, T.val.numpy())
    e = T.val.numpy().astype(np.float64) - want
    assert abs(sse - rsse) <= TOL32 * float(np.sum(2 * np.abs(e) * scale) + 1e-30)
    assert abs(sae - rsae) <= TOL32 * float(np.sum(scale) + 1e-30)


# ----------------------------------------------------------------------------- factor step


@pytest.mark.parametrize("n", [0, 1, 2])
def test_factor_one_batch_gradient(sft, oracle_mod, n):
    """One deterministic minibatch of 4096 with lr = 1: the row moves equal the
    negative batch gradient of Eq. (10) summed per row."""
    T = small_tensor()
    idx, val = to_dev(T)
    M, lr, lam = 4096, 1.0, 0.01
    perm = perm_of(0, 0, 0, n, T.nnz)
    sel = perm[:M].numpy().astype(np.int64)
    sub_idx = [i[perm[:M].long()].contiguous() for i in idx]
    sub_val = val[perm[:M].long()].contiguous()
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    A0 = [a.numpy().astype(np.float64) for a in T.A0]
    dec.update_factors(n, sub_idx, sub_val, None, batch=M, lr=lr, lam=lam)
    dec.sync(60_000)
    ref = oracle_mod.Model(A0, [b.numpy() for b in T.B0])
    ix = np_idx(T.idx)
    ref.factor_pass(n, [i[sel] for i in ix], T.val.numpy()[sel], batch=M, lr=lr, lam=lam)
    got = dec.A[n].cpu().numpy().astype(np.float64) - A0[n]
    want = ref.A[n] - A0[n]
    scale = factor_step_scale(A0, ref.B, n, ix, T.val.numpy(), sel, lr, lam)
    touched = np.zeros(A0[n].shape[0], bool)
    touched[ix[n][sel]] = True
    # the stored row is rounded to float32 once: allow one rounding of |a'|
    assert_within(got, want, scale + 1e-2 * np.abs(ref.A[n]), what=f"step A^({n})")
    assert np.all(got[~touched] == 0.0), "rows outside the batch moved"
    assert rel_fro(got, want) < TOL32


def test_factor_pass_perm_ragged(sft, oracle_mod):
    """A full deterministic factor pass through a permutation (49 minibatches of
    4096, the last 3392) agrees with the oracle pass."""
    T = small_tensor()
    idx, val = to_dev(T)
    n = 1
    perm = perm_of(0, 0, 0, n, T.nnz)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    A0 = dec.A[n].cpu().numpy().astype(np.float64)
    dec.update_factors(n, idx, val, perm.cuda(), batch=4096, lr=0.05, lam=0.01)
    dec.sync(60_000)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    S1, S2 = ref.factor_pass_scaled(n, np_idx(T.idx), T.val.numpy(),
                                    perm=perm.numpy().astype(np.uint32), batch=4096, lr=0.05,
                                    lam=0.01)
    got = dec.A[n].cpu().numpy().astype(np.float64)
    assert_rows_within(got, ref.A[n], S1, S2, what="ragged minibatch pass")
    assert rel_fro(got - A0, ref.A[n] - A0) < 1e-4
    assert rel_fro(got, ref.A[n]) < TOL32


# ----------------------------------------------------------------------------- core step


@pytest.mark.parametrize("n,M", [(0, 4096), (1, 4096), (2, 1000), (2, "all")])
def test_core_one_batch_gradient(sft, oracle_mod, n, M):
    """The first core minibatch with lr = 1: B moves by G / M_b - lam B
    (Eq. (11), Algorithm 5 when the batch is the whole tensor)."""
    T = small_tensor()
    idx, val = to_dev(T)
    lr, lam = 1.0, 0.01
    perm = perm_of(0, 0, 1, n, T.nnz)
    M = T.nnz if M == "all" else M
    sel = perm[:M].numpy().astype(np.int64)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    B_before = dec.B[n].cpu().numpy().astype(np.float64)
    dec.update_core(n, idx, val, perm.cuda(), batch=M, lr=lr, lam=lam) if M == T.nnz else \
        dec.update_core(n, [i[perm[:M].long()].contiguous() for i in idx],
                        val[perm[:M].long()].contiguous(), None, batch=M, lr=lr, lam=lam)
    dec.sync(60_000)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    ix = np_idx(T.idx)
    ref.core_pass(n, [i[sel] for i in ix], T.val.numpy()[sel], batch=M, lr=lr, lam=lam)
    got = dec.B[n].cpu().numpy().astype(np.float64) - B_before
    want = ref.B[n] - B_before
    scale = core_step_scale(ref.A, [b.numpy().astype(np.float64) for b in T.B0], n, ix,
                            T.val.numpy(), sel, lr, lam)
    assert_within(got, want, scale + 1e-2 * np.abs(ref.B[n]), what=f"step B^({n})")
    assert rel_fro(got, want) < TOL32


# ----------------------------------------------------------------------------- whole epochs


def _run_epochs(sft, oracle_mod, T, epochs, deterministic, batch_factor_gpu, batch_factor_ref,
                batch_core, lr=0.01):
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=deterministic)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    ix = np_idx(T.idx)
    xv = T.val.numpy()
    N = len(ix)
    got, want = [], []
    for ep in range(epochs):
        pf = [perm_of(0, ep, 0, n, T.nnz) for n in range(N)]
        pc = [perm_of(0, ep, 1, n, T.nnz) for n in range(N)]
        dec.epoch(idx, val, [p.cuda() for p in pf], [p.cuda() for p in pc],
                  batch_factor=batch_factor_gpu, batch_core=batch_core, lr_A=lr, lr_B=lr)
        ref.epoch(ix, xv, [p.numpy().astype(np.uint32) for p in pf],
                  [p.numpy().astype(np.uint32) for p in pc], batch_factor=batch_factor_ref,
                  batch_core=batch_core, lr_A=lr, lr_B=lr)
        got.append(dec.rmse(idx, val))
        want.append(ref.rmse(ix, xv))
    return np.array(got), np.array(want), dec, ref


def test_ten_epochs_deterministic_rmse(sft, oracle_mod):
    """10 epochs of Algorithm 2 on the 200k-nonzero planted tensor, minibatch
    4096, lr = lambda = 0.01: training RMSE per epoch within 1 % of the oracle."""
    T = small_tensor()
    got, want, dec, ref = _run_epochs(sft, oracle_mod, T, 10, True, 4096, 4096, 4096)
    np.testing.assert_allclose(got, want, rtol=0.01)
    for n in range(3):
        assert rel_fro(dec.A[n].cpu().numpy(), ref.A[n]) < 1e-4
        assert rel_fro(dec.B[n].cpu().numpy(), ref.B[n]) < 1e-4


def test_ten_epochs_hogwild_rmse(sft, oracle_mod):
    """Hogwild factor rows (every nonzero applies its own step at once) track
    the oracle's element-by-element rule (batch 1) within 1 % per epoch."""
    T = small_tensor()
    got, want, _, _ = _run_epochs(sft, oracle_mod, T, 10, False, 1, 1, 4096)
    np.testing.assert_allclose(got, want, rtol=0.01)


def test_deterministic_mode_is_bitwise_reproducible(sft):
    T = small_tensor()
    idx, val = to_dev(T)
    outs = []
    for _ in range(2):
        dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
        pf = [perm_of(3, 0, 0, n, T.nnz).cuda() for n in range(3)]
        pc = [perm_of(3, 0, 1, n, T.nnz).cuda() for n in range(3)]
        dec.epoch(idx, val, pf, pc, batch_factor=4096, batch_core=4096)
        dec.sync(60_000)
        outs.append([t.clone() for t in dec.A + dec.B + dec.C] + [torch.tensor(dec.loss(idx, val))])
    for a, b in zip(*outs):
        assert torch.equal(a, b)


# ----------------------------------------------------------------------------- other orders / ranks


@pytest.mark.parametrize("dims,J,R,lr", [
    ((300, 200), (8, 8), 8, 0.01),
    ((60, 50, 40, 30), (16, 8, 16, 32), 16, 0.002),
    ((40,) * 8, (8,) * 8, 32, 0.0005),
    ((500, 400, 300), (4, 4, 4), 4, 0.01),
    ((100, 90, 80, 70, 60), (32, 16, 8, 4, 32), 16, 0.002),
])
def test_other_orders_one_epoch(sft, oracle_mod, dims, J, R, lr):
    """One deterministic epoch at orders 2..8 and mixed ranks, ragged batches."""
    rng = np.random.default_rng(len(dims) * 7 + R)
    nnz = 5000
    idx, val = rand_coo(rng, dims, nnz)
    # entry std per mode so that every C entry has std R^(-1/(2N)) and x^ has std ~1
    N = len(dims)
    A = [torch.from_numpy(rng.normal(0, (R ** (-0.5 / N) / np.sqrt(j)) ** 0.5, (i, j))
                          .astype(np.float32)) for i, j in zip(dims, J)]
    B = [torch.from_numpy(rng.normal(0, (R ** (-0.5 / N) / np.sqrt(j)) ** 0.5, (j, R))
                          .astype(np.float32)) for j in J]
    from types import SimpleNamespace
    T = SimpleNamespace(idx=idx, val=val, A0=A, B0=B, nnz=nnz)
    got, want, dec, ref = _run_epochs(sft, oracle_mod, T, 1, True, 777, 777, 1000, lr=lr)
    assert np.all(np.isfinite(want)), "the oracle run diverged: the case is mis-set"
    np.testing.assert_allclose(got, want, rtol=1e-4)
    for n in range(len(dims)):
        assert rel_fro(dec.A[n].cpu().numpy(), ref.A[n]) < 1e-4
        assert rel_fro(dec.B[n].cpu().numpy(), ref.B[n]) < 1e-4


# ----------------------------------------------------------------------------- edge cases


def test_empty_and_tiny_sets(sft, oracle_mod):
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    A_before = [a.clone() for a in dec.A]
    empty_idx = [i[:0] for i in idx]
    dec.update_factors(0, empty_idx, val[:0], None, batch=16)
    dec.update_core(0, empty_idx, val[:0], None, batch=16)
    assert dec.loss(empty_idx, val[:0]) == (0.0, 0.0)
    dec.sync(10_000)
    assert all(torch.equal(a, b) for a, b in zip(A_before, dec.A))
    # batch 1 (element-by-element) and a batch larger than the set
    sub = [i[:37].contiguous() for i in idx]
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    six = [i[:37].numpy() for i in T.idx]
    dec.update_factors(2, sub, val[:37].contiguous(), None, batch=1, lr=0.5, lam=0.01)
    ref.factor_pass(2, six, T.val.numpy()[:37], batch=1, lr=0.5, lam=0.01)
    dec.update_core(1, sub, val[:37].contiguous(), None, batch=4096, lr=0.5, lam=0.01)
    ref.core_pass(1, six, T.val.numpy()[:37], batch=4096, lr=0.5, lam=0.01)
    dec.sync(10_000)
    assert rel_fro(dec.A[2].cpu().numpy(), ref.A[2]) < TOL32
    assert rel_fro(dec.B[1].cpu().numpy(), ref.B[1]) < TOL32


def test_bad_data_is_flagged_not_faulted(sft):
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=False)
    bad = [i[:100].clone() for i in idx]
    bad[1][17] = 10_000_000  # out of range for mode 1
    A_before = [a.clone() for a in dec.A]
    dec.update_factors(0, bad, val[:100].contiguous(), None)
    with pytest.raises(sft.SftError) as ei:
        dec.sync(10_000)
    assert ei.value.status == sft.SFT_EINVAL
    # the flag is cleared and the good samples were applied
    dec.sync(10_000)
    assert not torch.equal(A_before[0], dec.A[0])
    perm = torch.arange(100, dtype=torch.int32, device="cuda")
    perm[5] = 1000
    dec.update_core(0, [i[:100].contiguous() for i in idx], val[:100].contiguous(), perm, batch=64)
    with pytest.raises(sft.SftError):
        dec.sync(10_000)


def test_unsupported_requests(sft):
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True, max_batch=4096)
    with pytest.raises(sft.SftError) as ei:
        dec.update_factors(0, idx, val, None, batch=8192)
    assert ei.value.status == sft.SFT_ENOTSUP
    with pytest.raises(sft.SftError) as ei:
        dec.update_factors(5, idx, val, None, batch=64)
    assert ei.value.status == sft.SFT_EINVAL
    dec.sync(10_000)
