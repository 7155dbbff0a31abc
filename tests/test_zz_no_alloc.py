"""The allocation-free factor pass (sft_update_factors_noalloc) against the
workspace entry point (sft_update_factors, deterministic minibatch rule).

The no-allocation call serves callers that cannot allocate device memory (a
plugin inside an application that owns all device memory, a loop that must not
allocate); it keeps its scratch in a fixed array inside the library.  This file
sorts last so that a run stopping at the first failure has run every other
test first; it passes alone in a fresh process too.
"""
import functools

import numpy as np
import pytest
import torch

from parity_util import TOL32, rel_fro, small_tensor, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


@functools.lru_cache(maxsize=None)
def tensor_for(J):
    """J = R = 8: the 200k-nonzero planted tensor (48 full minibatches of 4096
    and a ragged 3392); J = R = 32: 20k nonzeros (4 full minibatches and a
    ragged 3616), which fills the J = 32 row-sum region of the fixed scratch."""
    if J == 8:
        return small_tensor()
    from paper_2210_06014_gb300 import synth
    sigma = (J ** (-1.0 / 6) / J ** 0.5) ** 0.5
    spec = synth.TensorSpec(f"noalloc-order3-300x200x100-20k-J{J}R{J}", (300, 200, 100), 20_000,
                            (J,) * 3, J, ("uniform",) * 3, planted_sigma=sigma, noise_sigma=0.01,
                            seed=2)
    return synth.make_tensor(spec)


@pytest.mark.parametrize("J", [8, 32])
def test_noalloc_factor_pass_matches_workspace_entry_point(sft, J):
    from paper_2210_06014_gb300 import synth
    T = tensor_for(J)
    assert T.nnz % 4096 != 0  # the last minibatch is ragged
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)  # the existing entry point
    A_free = [a.clone() for a in dec.A]                         # operands of the new one
    n, batch, lam = 1, 4096, 0.01
    lr = 0.05 if J == 8 else 2e-4  # the minibatch rule sums ~14 steps per row at J = 32
    for call in range(2):  # two calls in a row: the second starts from the first's result
        perm = synth.pass_permutation(11, call, 0, n, T.nnz).cuda()
        dec.update_factors(n, idx, val, perm, batch=batch, lr=lr, lam=lam)
        st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, n, A_free[n], dec.B[n], dec.C,
                                            idx, val, perm, T.nnz, batch, lr, lam)
        assert st == sft.SFT_OK
        dec.sync(60_000)
        got = A_free[n].cpu().numpy().astype(np.float64)
        want = dec.A[n].cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(got))
        assert rel_fro(got, want) < TOL32, call
        np.testing.assert_allclose(got, want, rtol=TOL32, atol=TOL32 * np.abs(want).max())
    # the other factor matrices are untouched
    for k in range(3):
        if k != n:
            assert torch.equal(A_free[k], dec.A[k])
    # a minibatch larger than the fixed scratch is refused without any work
    before = A_free[n].clone()
    st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, n, A_free[n], dec.B[n], dec.C, idx,
                                        val, None, T.nnz, 8192, lr, lam)
    assert st == sft.SFT_ENOTSUP
    torch.cuda.synchronize()
    assert torch.equal(before, A_free[n])
    # a non-finite step size is refused before any launch
    st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, n, A_free[n], dec.B[n], dec.C, idx,
                                        val, None, T.nnz, batch, float("inf"), lam)
    assert st == sft.SFT_EINVAL
    torch.cuda.synchronize()
    assert torch.equal(before, A_free[n])


def test_noalloc_bad_permutation_entry_is_skipped_and_reported(sft):
    """A permutation entry equal to nnz is bad data: both entry points skip that
    sample, the no-allocation call reports SFT_EINVAL after its wait, and the
    factor matrices agree with the workspace path run on the same data."""
    from paper_2210_06014_gb300 import synth
    T = small_tensor()
    idx, val = to_dev(T)
    n, batch, lr, lam = 2, 4096, 0.05, 0.01
    perm = synth.pass_permutation(12, 0, 0, n, T.nnz).clone()
    perm[5000] = T.nnz  # out of range
    perm = perm.cuda()
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    A_free = dec.A[n].clone()
    dec.update_factors(n, idx, val, perm, batch=batch, lr=lr, lam=lam)
    with pytest.raises(sft.SftError) as ex:
        dec.sync(60_000)
    assert ex.value.status == sft.SFT_EINVAL
    st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, n, A_free, dec.B[n], dec.C, idx,
                                        val, perm, T.nnz, batch, lr, lam)
    assert st == sft.SFT_EINVAL
    got = A_free.cpu().numpy().astype(np.float64)
    want = dec.A[n].cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(got))
    np.testing.assert_allclose(got, want, rtol=TOL32, atol=TOL32 * np.abs(want).max())
    # the flag was cleared: a clean call on the same data succeeds
    st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, n, A_free, dec.B[n], dec.C, idx,
                                        val, None, T.nnz, batch, lr, lam)
    assert st == sft.SFT_OK


def test_noalloc_refuses_stream_capture(sft):
    """The call synchronises, so on a stream that is being captured it returns
    SFT_ENOTSUP before enqueuing anything (the capture stays valid)."""
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)
    A_free = dec.A[0].clone()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        g.capture_begin()
        st = sft.sft_update_factors_noalloc(dec.dims, dec.J, dec.R, 0, A_free, dec.B[0], dec.C,
                                            idx, val, None, T.nnz, 4096, 0.05, 0.01,
                                            stream=s.cuda_stream)
        g.capture_end()
    assert st == sft.SFT_ENOTSUP
    torch.cuda.synchronize()
    assert torch.equal(A_free, dec.A[0])
