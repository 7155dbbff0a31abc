"""GPU checks of the batched runner (include/sft_batch.h): many independent
decompositions trained by one persistent kernel per epoch, against the FP64
oracle run problem by problem."""
import functools

import numpy as np
import pytest
import torch

from parity_util import TOL32, abs_C, assert_within, pred_scale, stable_lr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


@functools.lru_cache(maxsize=None)
def problems(count=6, seed=3):
    from paper_2210_06014_gb300 import synth
    specs = synth.spec_batch(count, seed=seed, dims=(40, 3000), nnz=(3_000, 60_000))
    return [synth.make_tensor(s) for s in specs]


def dev_problems(Ts):
    return [(T.A0, T.B0, [i.cuda() for i in T.idx], T.val.cuda()) for T in Ts]


def oracles(oracle_mod, Ts):
    return [oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0]) for T in Ts]


def test_batch_covers_orders_and_ranks():
    Ts = problems()
    assert len({T.spec.order for T in Ts}) >= 3 and len({T.spec.R for T in Ts}) >= 3


def test_batch_refresh_and_loss(sft, oracle_mod):
    Ts = problems()
    b = sft.Batch(dev_problems(Ts))
    losses = b.loss()
    for T, ref, C, (sse, sae) in zip(Ts, oracles(oracle_mod, Ts), b.C, losses):
        absC = abs_C(ref.A, ref.B)
        for n in range(T.spec.order):
            assert_within(C[n].cpu().numpy(), ref.C[n], absC[n], what=f"{T.spec.name} C^({n})")
        ix = [i.numpy().astype(np.int64) for i in T.idx]
        want_sse, want_sae = ref.loss(ix, T.val.numpy())
        e_scale = np.abs(T.val.numpy().astype(np.float64)) + pred_scale(absC, ix)
        assert abs(sse - want_sse) <= TOL32 * 2 * np.sum(e_scale * pred_scale(absC, ix)) + 1e-9
        assert abs(sae - want_sae) <= TOL32 * np.sum(pred_scale(absC, ix)) + 1e-9


def _epochs(sft, oracle_mod, prec, epochs):
    Ts = problems()
    lrs = [stable_lr(T) for T in Ts]
    b = sft.Batch(dev_problems(Ts), prec=prec, min_chunk=1024, lr=lrs)
    refs = oracles(oracle_mod, Ts)
    got, want = [], []
    for _ in range(epochs):
        b.epoch()
        got.append(b.rmse())
        row = []
        for T, ref, lr in zip(Ts, refs, lrs):
            ix = [i.numpy().astype(np.int64) for i in T.idx]
            ref.epoch(ix, T.val.numpy(), None, None, batch_factor=1, batch_core=T.nnz, lr_A=lr,
                      lam_A=0.01, lr_B=lr, lam_B=0.01)
            row.append(ref.rmse(ix, T.val.numpy()))
        want.append(row)
    return np.array(got), np.array(want), b


def test_batch_epochs_track_the_oracle(sft, oracle_mod):
    """Three epochs of every problem (Hogwild factor rows, one core update per
    pass): training RMSE within 1 % of the oracle's sequential epochs."""
    got, want, b = _epochs(sft, oracle_mod, sft.SFT_FP32, 3)
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=0.01)
    assert b.launches == 1 + 3 + 3  # refresh, 3 epochs, 3 losses: one graph each


def test_batch_bf16_epochs(sft, oracle_mod):
    got, want, _ = _epochs(sft, oracle_mod, sft.SFT_BF16, 2)
    np.testing.assert_allclose(got, want, rtol=0.02)


def test_batch_autotune_leaves_the_model_unchanged(sft):
    Ts = problems()
    b = sft.Batch(dev_problems(Ts), min_chunk=512, lr=[stable_lr(T) for T in Ts])
    b.epoch()
    b.sync(60_000)
    before = [[t.clone() for t in A + B] for A, B in zip(b.A, b.B)]
    loss0 = b.loss()
    chunk, bps = b.autotune(epochs=1)
    assert chunk in (512, 1024, 2048, 4096) and bps >= 1
    after = [[t.clone() for t in A + B] for A, B in zip(b.A, b.B)]
    assert all(bool(torch.isfinite(t).all()) for x in before for t in x)
    for x, y in zip(before, after):
        for s, t in zip(x, y):
            assert torch.equal(s, t)
    assert b.loss() == loss0  # C was refreshed from the restored A, B


def test_batch_bad_coordinate_is_reported(sft):
    Ts = problems()
    probs = dev_problems(Ts)
    A0, B0, idx, val = probs[1]
    idx = [i.clone() for i in idx]
    idx[0][5] = Ts[1].spec.dims[0]
    probs[1] = (A0, B0, idx, val)
    b = sft.Batch(probs)
    with pytest.raises(sft.SftError, match="out of range"):
        b.loss()


def test_batch_wait_timeout_is_reported_and_recoverable(sft):
    """A pass that can never complete (held on the host) makes the tasks after
    it give up after the poll limit: the epoch reports SFT_ETIMEOUT, and after
    the hold is lifted the same handle runs epochs normally."""
    Ts = problems()
    b = sft.Batch(dev_problems(Ts), lr=[stable_lr(T) for T in Ts])
    b.set_wait_limit(4000)  # a few ms of polling
    b.hold_pass(2)
    b.epoch()
    with pytest.raises(sft.SftError, match="SFT_ETIMEOUT"):
        b.sync(60_000)
    b.hold_pass(2, False)
    b.set_wait_limit(1 << 24)
    b.refresh()
    b.epoch()
    b.sync(60_000)
    assert all(np.isfinite(r) for r in b.rmse())
