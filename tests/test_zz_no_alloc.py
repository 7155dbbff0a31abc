"""The allocation-free factor pass (sft_update_factors_noalloc) against the
workspace entry point (sft_update_factors, deterministic minibatch rule).

The no-allocation call serves callers that cannot allocate device memory (a
plugin inside an application that owns all device memory, a loop that must not
allocate); it keeps its scratch in a fixed array inside the library.  This file
sorts last so that a run stopping at the first failure has run every other
test first; it passes alone in a fresh process too.
"""
import numpy as np
import pytest
import torch

from parity_util import TOL32, rel_fro, small_tensor, to_dev

pytestmark = pytest.mark.gpu


def test_noalloc_factor_pass_matches_workspace_entry_point():
    from paper_2210_06014_gb300 import build, sft, synth
    build.build()
    sft.load()
    T = small_tensor()
    idx, val = to_dev(T)
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True)  # the existing entry point
    A_free = [a.clone() for a in dec.A]                         # operands of the new one
    n, batch, lr, lam = 1, 4096, 0.05, 0.01
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
