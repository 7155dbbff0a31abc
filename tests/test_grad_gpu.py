"""GPU parity of the sampled-loss gradient (sft_loss_grad_C + sft_grad_AB and
the autograd module on top of them) against the FP64 oracle's loss_grad.

The oracle gradient is pinned on the CPU by central differences; here the
float32 CUDA result must match it within 1e-5 of the condition bound of each
entry (the same sum over absolute values), and the incoming-gradient scale,
the accumulate flag, the loss-only mode and the bad-index flag are exercised.
"""
import math

import numpy as np
import pytest
import torch

from parity_util import TOL32, assert_within, grad_scale

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


CASES = {
    # name: (dims, J, R, nnz)
    "order3_J8": ((300, 200, 100), (8, 8, 8), 8, 20_000),
    "order4_J32": ((500, 400, 300, 200), (32, 32, 32, 32), 32, 30_000),
    "order5_mixed": ((90, 80, 70, 60, 50), (4, 8, 16, 8, 4), 16, 25_003),
    "order9_J16": ((40,) * 9, (16,) * 9, 16, 12_001),
}


def make_case(name, seed=0):
    dims, J, R, nnz = CASES[name]
    N = len(dims)
    rng = np.random.default_rng(seed)
    sig = [math.sqrt(R ** (-1.0 / (2 * N)) / math.sqrt(j)) for j in J]
    A = [rng.normal(0, s, (I, j)).astype(np.float32) for I, j, s in zip(dims, J, sig)]
    B = [rng.normal(0, s, (j, R)).astype(np.float32) for j, s in zip(J, sig)]
    idx = [rng.integers(0, I, nnz).astype(np.int32) for I in dims]
    val = rng.normal(0, 1, nnz).astype(np.float32)
    return A, B, idx, val


def dev(A, B, idx, val):
    return ([torch.from_numpy(a) for a in A], [torch.from_numpy(b) for b in B],
            [torch.from_numpy(i).cuda() for i in idx], torch.from_numpy(val).cuda())


@pytest.mark.parametrize("name", list(CASES))
def test_loss_grad_matches_oracle(sft, oracle_mod, name):
    A, B, idx, val = make_case(name)
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    out, dC = dec.loss_grad_C(didx, dval)
    gA, gB = dec.grad_AB(dC)
    dec.sync(60_000)
    L_ref, gA_ref, gB_ref = oracle_mod.Model(A, B).loss_grad(idx, val)
    ix = [i.astype(np.int64) for i in idx]
    sA, sB, sL = grad_scale([a.astype(np.float64) for a in A], [b.astype(np.float64) for b in B],
                            ix, val)
    L = out.cpu().numpy()
    assert abs(L[0] - L_ref) <= TOL32 * sL + 1e-12, (L[0], L_ref)
    for n in range(len(A)):
        assert_within(gA[n].cpu().numpy(), gA_ref[n], sA[n], what=f"{name} dL/dA[{n}]")
        assert_within(gB[n].cpu().numpy(), gB_ref[n], sB[n], what=f"{name} dL/dB[{n}]")


def test_sum_abs_residual_and_loss_only(sft, oracle_mod):
    A, B, idx, val = make_case("order3_J8", seed=3)
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    out_g, _ = dec.loss_grad_C(didx, dval)
    out_l = torch.empty(2, dtype=torch.float64, device="cuda")
    sft.sft_loss_grad_C(dec.ctx, didx, dval, dval.numel(), None, 0, out_l)
    dec.sync(60_000)
    pred = oracle_mod.Model(A, B).predict(idx)
    e = val.astype(np.float64) - pred
    got_g, got_l = out_g.cpu().numpy(), out_l.cpu().numpy()
    assert got_l[0] == got_g[0] and got_l[1] == got_g[1]
    assert abs(got_g[1] - np.abs(e).sum()) <= 1e-5 * np.abs(e).sum()
    assert abs(got_g[0] - 0.5 * (e * e).sum()) <= 1e-5 * (e * e).sum()


def test_scale_and_accumulate(sft):
    A, B, idx, val = make_case("order4_J32", seed=5)
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    _, dC = dec.loss_grad_C(didx, dval)
    gA1, gB1 = dec.grad_AB(dC)
    s = torch.tensor([-2.5], dtype=torch.float64, device="cuda")
    gA2, gB2 = dec.grad_AB(dC, s)
    # a second pass added onto the first doubles dC up to rounding
    dC2 = [d.clone() for d in dC]
    dec.loss_grad_C(didx, dval, dC=dC2, accumulate=True)
    dec.sync(60_000)
    for n in range(4):
        torch.testing.assert_close(gA2[n], -2.5 * gA1[n], rtol=1e-6, atol=0)
        torch.testing.assert_close(gB2[n], -2.5 * gB1[n], rtol=1e-6, atol=1e-12)
        scale = dC[n].abs().max().item()
        assert (dC2[n] - 2 * dC[n]).abs().max().item() <= 1e-5 * scale


def test_empty_set_gives_zero(sft):
    A, B, idx, val = make_case("order3_J8")
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    out, dC = dec.loss_grad_C([i[:0] for i in didx], dval[:0])
    gA, gB = dec.grad_AB(dC)
    dec.sync(60_000)
    assert out.cpu().tolist() == [0.0, 0.0]
    for n in range(3):
        assert gA[n].abs().max().item() == 0.0 and gB[n].abs().max().item() == 0.0


def test_bad_coordinate_is_flagged(sft):
    A, B, idx, val = make_case("order3_J8")
    idx = [i.copy() for i in idx]
    idx[1][17] = CASES["order3_J8"][0][1]  # one past the end: the kernel skips it
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    dec.loss_grad_C(didx, dval)
    with pytest.raises(sft.SftError, match="out of range"):
        dec.sync(60_000)


def test_autograd_module(sft, oracle_mod):
    """SampledLoss: forward value, .grad of every parameter after backward of a
    scaled loss, loss-only forward under no_grad, and that torch.optim.SGD on
    it lowers the loss."""
    A, B, idx, val = make_case("order4_J32", seed=9)
    tA, tB, didx, dval = dev(A, B, idx, val)
    mod = sft.SampledLoss(tA, tB)
    L = mod(didx, dval)
    (3.0 * L).backward()
    L_ref, gA_ref, gB_ref = oracle_mod.Model(A, B).loss_grad(idx, val)
    ix = [i.astype(np.int64) for i in idx]
    sA, sB, sL = grad_scale([a.astype(np.float64) for a in A], [b.astype(np.float64) for b in B],
                            ix, val)
    assert abs(L.item() - L_ref) <= TOL32 * sL
    for n in range(4):
        assert_within(mod.A[n].grad.cpu().numpy(), 3.0 * gA_ref[n], 3.0 * sA[n], what=f"A[{n}].grad")
        assert_within(mod.B[n].grad.cpu().numpy(), 3.0 * gB_ref[n], 3.0 * sB[n], what=f"B[{n}].grad")
    with torch.no_grad():
        L0 = mod(didx, dval).item()
    assert L0 == L.item()
    opt = torch.optim.SGD(mod.parameters(), lr=2e-4)
    losses = []
    for _ in range(5):
        opt.zero_grad()
        loss = mod(didx, dval)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    with torch.no_grad():
        losses.append(mod(didx, dval).item())
    assert all(b < a for a, b in zip(losses, losses[1:])), losses


def test_gradient_against_central_differences(sft, oracle_mod):
    """Independent of the oracle's gradient code: entries of the CUDA gradient
    against central differences (h = 1e-3, float64) of the oracle's loss on a
    1000-nonzero subset."""
    A, B, idx, val = make_case("order4_J32", seed=21)
    idx = [i[:1000] for i in idx]
    val = val[:1000]
    tA, tB, didx, dval = dev(A, B, idx, val)
    dec = sft.Decomposition(tA, tB)
    _, dC = dec.loss_grad_C(didx, dval)
    gA, gB = dec.grad_AB(dC)
    dec.sync(60_000)
    ix = [i.astype(np.int64) for i in idx]
    A64 = [a.astype(np.float64) for a in A]
    B64 = [b.astype(np.float64) for b in B]
    sA, sB, _ = grad_scale(A64, B64, ix, val)

    def loss(As, Bs):
        sse, _ = oracle_mod.Model(As, Bs).loss(idx, val)
        return 0.5 * sse

    h = 1e-3
    rng = np.random.default_rng(2)
    for n in range(4):
        for _ in range(3):
            i = int(ix[n][rng.integers(0, 1000)])  # a row the subset touches
            j = int(rng.integers(0, A[n].shape[1]))
            Ap = [a.copy() for a in A64]; Am = [a.copy() for a in A64]
            Ap[n][i, j] += h; Am[n][i, j] -= h
            fd = (loss(Ap, B64) - loss(Am, B64)) / (2 * h)
            got = float(gA[n][i, j])
            assert abs(got - fd) <= 1e-4 * sA[n][i, j] + 1e-5 * abs(fd), (n, i, j, got, fd)
            j, r = int(rng.integers(0, B[n].shape[0])), int(rng.integers(0, B[n].shape[1]))
            Bp = [b.copy() for b in B64]; Bm = [b.copy() for b in B64]
            Bp[n][j, r] += h; Bm[n][j, r] -= h
            fd = (loss(A64, Bp) - loss(A64, Bm)) / (2 * h)
            got = float(gB[n][j, r])
            assert abs(got - fd) <= 1e-4 * sB[n][j, r] + 1e-5 * abs(fd), (n, j, r, got, fd)


def test_bf16_cached_products_gradient(sft, oracle_mod):
    """With C stored in bfloat16 the gradient stays within 2e-2 of the float64
    oracle (condition-aware)."""
    A, B, idx, val = make_case("order4_J32", seed=6)
    tA, tB, didx, dval = dev(A, B, idx, val)
    mod = sft.SampledLoss(tA, tB, prec=sft.SFT_BF16)
    L = mod(didx, dval)
    L.backward()
    L_ref, gA_ref, gB_ref = oracle_mod.Model(A, B).loss_grad(idx, val)
    ix = [i.astype(np.int64) for i in idx]
    sA, sB, sL = grad_scale([a.astype(np.float64) for a in A], [b.astype(np.float64) for b in B],
                            ix, val)
    assert abs(L.item() - L_ref) <= 2e-2 * sL
    for n in range(4):
        assert_within(mod.A[n].grad.cpu().numpy(), gA_ref[n], sA[n], tol=2e-2, what=f"bf16 A[{n}]")
        assert_within(mod.B[n].grad.cpu().numpy(), gB_ref[n], sB[n], tol=2e-2, what=f"bf16 B[{n}]")
