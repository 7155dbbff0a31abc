"""Tensor-core (tcgen05) kernels of the bfloat16 configuration, through the C ABI.

* The refresh C^(n) = A^(n) B^(n) (Algorithm 3) by kind::tf32 MMAs on tiles of
  A^(n) copied by TMA, rounded to bfloat16: within 2e-2 of the FP64 oracle
  (condition-aware), and within a couple of bfloat16 steps of the float32
  CUDA-core refresh of the same call (sft_set_tensor_cores(ctx, 0)).
* The minibatch core gradient G = sum_s e_s a p_s^T (Eq. (11), Algorithm 5) by
  kind::f16 MMAs on bfloat16 operands with a float32 accumulator: one core
  step within 2e-2 of the oracle's, and within the operand-rounding bound of
  the CUDA-core kernel on the same bfloat16 cached products.
* Whole epochs of Algorithm 2 on the COO path in bfloat16 (tensor-core refresh
  and core passes): training RMSE within 1 % of the oracle per epoch.

Shapes cover several 128-row tiles with a ragged tail, a tile of 5 rows, more
tiles than CTAs (grid-stride), spans of several 64-nonzero MMA batches with a
ragged last batch (both operand buffers reused).
"""
import numpy as np
import pytest
import torch

from parity_util import abs_C, assert_within, core_step_scale, np_idx, rel_fro, to_dev

pytestmark = pytest.mark.gpu

TOL_BF16 = 2e-2


@pytest.fixture(scope="module")
def sft():
    from paper_2210_06014_gb300 import build, sft as mod
    build.build()
    mod.load()
    return mod


def rand_params(rng, dims, J, R, scale=0.4):
    A = [torch.from_numpy(rng.normal(0, scale, (i, j)).astype(np.float32)) for i, j in zip(dims, J)]
    B = [torch.from_numpy(rng.normal(0, scale, (j, R)).astype(np.float32)) for j in J]
    return A, B


def planted(J, R, dims=(300, 200, 100), nnz=20_000, seed=0):
    from paper_2210_06014_gb300 import synth
    sigma = (R ** (-1.0 / (2 * len(dims))) / J ** 0.5) ** 0.5  # std(x) about 1
    spec = synth.TensorSpec(f"tc-order3-{dims}-{nnz}-J{J}R{R}", dims, nnz, (J,) * len(dims), R,
                            ("uniform",) * len(dims), planted_sigma=sigma, noise_sigma=0.01,
                            seed=seed)
    return synth.make_tensor(spec)


# ----------------------------------------------------------------------------- refresh


@pytest.mark.parametrize("J,R,dims", [
    (8, 16, (1031, 517, 77)), (16, 16, (1031, 517, 77)), (32, 16, (1031, 517, 77)),
    (8, 32, (1031, 517, 77)), (16, 32, (1031, 517, 77)), (32, 32, (1031, 517, 77)),
    (16, 16, (480_000, 128, 5)),  # 3750 tiles > CTAs; exactly one tile; a 5-row tile
])
def test_tc_refresh_parity(sft, oracle_mod, J, R, dims):
    rng = np.random.default_rng(J * 1000 + R + len(str(dims)))
    A, B = rand_params(rng, dims, (J,) * 3, R)
    tc = sft.Decomposition(A, B, prec=sft.SFT_BF16, tensor_cores=True)
    cc = sft.Decomposition(A, B, prec=sft.SFT_BF16, tensor_cores=False)
    tc.sync(60_000)
    cc.sync(60_000)
    ref = oracle_mod.Model([a.numpy() for a in A], [b.numpy() for b in B])
    absC = abs_C(ref.A, ref.B)
    worst = 0.0
    for n in range(3):
        got = tc.C[n].float().cpu().numpy().astype(np.float64)
        other = cc.C[n].float().cpu().numpy().astype(np.float64)
        assert_within(got, ref.C[n], absC[n], tol=TOL_BF16, what=f"tensor-core C^({n})")
        # tf32 operands and bfloat16 rounding on both sides: a bfloat16 step of
        # the value plus the operand rounding of sum |a||b|
        bound = 2.0 ** -7 * np.abs(other) + 2.0 ** -8 * absC[n] + 1e-30
        err = np.abs(got - other)
        assert (err <= bound).all(), (n, float(np.max(err / bound)))
        worst = max(worst, float(np.max(np.abs(got - ref.C[n]) / (absC[n] + 1e-30))))
    print(f"tensor-core refresh J={J} R={R} dims={dims}: worst |C err| / |A||B| = {worst:.3e}")


# ----------------------------------------------------------------------------- core gradient


@pytest.mark.parametrize("J,R,n,M", [(16, 16, 0, 4096), (32, 32, 1, 4096), (8, 16, 2, 1000),
                                     (16, 32, 0, "all"), (4, 16, 1, 333), (32, 16, 2, "all")])
def test_tc_core_one_batch(sft, oracle_mod, J, R, n, M):
    """The first core minibatch with lr = 1: B moves by G / M_b - lam B."""
    T = planted(J, R)
    idx, val = to_dev(T)
    lr, lam = 1.0, 0.01
    M = T.nnz if M == "all" else M
    sel = np.arange(M, dtype=np.int64)
    sub_idx = [i[:M].contiguous() for i in idx]
    sub_val = val[:M].contiguous()
    steps = {}
    for tcores in (True, False):
        dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16, tensor_cores=tcores)
        B_before = dec.B[n].cpu().numpy().astype(np.float64)
        dec.update_core(n, sub_idx, sub_val, None, batch=M, lr=lr, lam=lam)
        dec.sync(60_000)
        steps[tcores] = dec.B[n].cpu().numpy().astype(np.float64) - B_before
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    ix = np_idx(T.idx)
    ref.core_pass(n, [i[sel] for i in ix], T.val.numpy()[sel], batch=M, lr=lr, lam=lam)
    want = ref.B[n] - np.asarray(T.B0[n], dtype=np.float64)
    scale = core_step_scale(ref.A, [b.numpy().astype(np.float64) for b in T.B0], n, ix,
                            T.val.numpy(), sel, lr, lam)
    assert_within(steps[True], want, scale, tol=TOL_BF16, what=f"tensor-core step B^({n})")
    # same bfloat16 cached products on both GPU paths: only the operand rounding
    # of e*a and p (2^-8 relative each) separates them
    assert_within(steps[True], steps[False], scale, tol=2.0 ** -6, what="tensor vs CUDA cores")
    print(f"tensor-core core step J={J} R={R} M={M}: rel err vs oracle "
          f"{rel_fro(steps[True], want):.3e}, vs CUDA cores {rel_fro(steps[True], steps[False]):.3e}")


def test_tc_core_large_whole_pass(sft):
    """A whole-pass core step over 4M nonzeros (608 blocks of about 6.6k
    nonzeros each, about 100 MMA batches per block) agrees with the CUDA-core
    kernel on the same bfloat16 cached products, in every mode."""
    from paper_2210_06014_gb300 import synth
    spec = synth.TensorSpec("tc-large-order3-200000x20000x2000-4M-J16R16", (200_000, 20_000, 2_000),
                            4_000_000, (16, 16, 16), 16, ("zipf", "zipf", "uniform"),
                            planted_sigma=0.4, noise_sigma=0.01)
    T = synth.make_tensor(spec)
    idx, val = to_dev(T)
    for n in range(3):
        steps = {}
        for tcores in (True, False):
            dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16, tensor_cores=tcores)
            B_before = dec.B[n].clone()
            dec.update_core(n, idx, val, None, batch=T.nnz, lr=1.0, lam=0.01)
            dec.sync(120_000)
            steps[tcores] = (dec.B[n] - B_before).double().cpu().numpy()
            dec.close()
        assert rel_fro(steps[True], steps[False]) < 1e-2, n


def test_tc_epochs_rmse(sft, oracle_mod):
    """Three epochs of Algorithm 2 on the COO path with bfloat16 cached products
    (tensor-core refresh and core gradient, minibatch 4096): training RMSE per
    epoch within 1 % of the float64 oracle."""
    from paper_2210_06014_gb300 import synth
    T = planted(16, 16, dims=(1000, 800, 600), nnz=200_000)
    idx, val = to_dev(T)
    ix = np_idx(T.idx)
    xv = T.val.numpy()
    dec = sft.Decomposition(T.A0, T.B0, deterministic=True, prec=sft.SFT_BF16)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    got, want = [], []
    for ep in range(3):
        pf = [synth.pass_permutation(0, ep, 0, n, T.nnz) for n in range(3)]
        pc = [synth.pass_permutation(0, ep, 1, n, T.nnz) for n in range(3)]
        dec.epoch(idx, val, [p.cuda() for p in pf], [p.cuda() for p in pc], batch_factor=4096,
                  batch_core=4096)
        ref.epoch(ix, xv, [p.numpy().astype(np.uint32) for p in pf],
                  [p.numpy().astype(np.uint32) for p in pc], batch_factor=4096, batch_core=4096)
        got.append(dec.rmse(idx, val))
        want.append(ref.rmse(ix, xv))
    print("tensor-core epochs rmse gpu", got, "oracle", want)
    np.testing.assert_allclose(got, want, rtol=0.01)


# ----------------------------------------------------------------------------- bounded waits


def test_tc_wait_expiry_is_reported_and_recoverable(sft, oracle_mod):
    """The expiry path of the tensor-core kernels' bounded waits, made to run on
    a normal launch: with a wait limit of 0 every block gives up at its first
    wait on its own TMA copy / MMA, flags it, drains what it issued (full 2 s
    bound), frees its tensor memory and returns.  sft_sync reports
    SFT_ETIMEOUT for the refresh and for the core pass; with the default limit
    restored, the same context refreshes C and takes a core step that match
    the oracle again.  Nothing faults or hangs: every wait stays bounded."""
    T = planted(16, 16, dims=(1031, 517, 77), nnz=20_000, seed=3)
    idx, val = to_dev(T)
    n, lr, lam = 1, 1.0, 0.01
    dec = sft.Decomposition(T.A0, T.B0, prec=sft.SFT_BF16, tensor_cores=True)
    dec.sync(60_000)
    B_keep = [b.clone() for b in dec.B]
    sft.sft_set_tc_wait_limit(dec.ctx, 0)
    dec.refresh(-1)
    with pytest.raises(sft.SftError) as ex:
        dec.sync(60_000)
    assert ex.value.status == sft.SFT_ETIMEOUT
    dec.update_core(n, idx, val, None, batch=4096, lr=lr, lam=lam)
    with pytest.raises(sft.SftError) as ex:
        dec.sync(60_000)
    assert ex.value.status == sft.SFT_ETIMEOUT
    # back to the default limit: the context is usable and the results are right
    sft.sft_set_tc_wait_limit(dec.ctx, 2_000_000_000)
    for k in range(3):
        dec.B[k].copy_(B_keep[k])
    dec.refresh(-1)
    dec.sync(60_000)
    ref = oracle_mod.Model([a.numpy() for a in T.A0], [b.numpy() for b in T.B0])
    absC = abs_C(ref.A, ref.B)
    for k in range(3):
        assert_within(dec.C[k].float().cpu().numpy(), ref.C[k], absC[k], tol=TOL_BF16,
                      what=f"C^({k}) after the expired waits")
    M = 4096
    sub_idx = [i[:M].contiguous() for i in idx]
    sub_val = val[:M].contiguous()
    B_before = dec.B[n].cpu().numpy().astype(np.float64)
    dec.update_core(n, sub_idx, sub_val, None, batch=M, lr=lr, lam=lam)
    dec.sync(60_000)
    got = dec.B[n].cpu().numpy().astype(np.float64) - B_before
    ix = np_idx(T.idx)
    sel = np.arange(M)
    ref.core_pass(n, [i[sel] for i in ix], T.val.numpy()[sel], batch=M, lr=lr, lam=lam)
    want = ref.B[n] - np.asarray(T.B0[n], dtype=np.float64)
    scale = core_step_scale(ref.A, [b.numpy().astype(np.float64) for b in T.B0], n, ix,
                            T.val.numpy(), sel, lr, lam)
    assert_within(got, want, scale, tol=TOL_BF16, what="core step after the expired waits")
