"""Pins of the FP64 oracle against facts that do not come from the oracle.

Each test fixes one part of the oracle with something independent of its own
code: the dense Tucker reconstruction (Definition "n-Mode Tensor-Matrix
product" with the Kruskal core of Eq. (1)), the matricised form Eq. (3) built
from explicit Kronecker / Khatri-Rao products, central finite differences of
the per-element objectives Eq. (7)/(8) and of the minibatch objective Eq. (9),
textbook special cases (CP-SGD, matrix-factorisation SGD), gauge invariances of
the model, and recovery of a planted low-rank tensor.
"""
import itertools

import os

import numpy as np
import pytest

# ----------------------------------------------------------------------------- helpers


def rand_model(rng, I, J, R, scale=0.5):
    A = [rng.normal(0, scale, (i, j)) for i, j in zip(I, J)]
    B = [rng.normal(0, scale, (j, R)) for j in J]
    return A, B


def all_coords(I):
    coords = np.array(list(itertools.product(*[range(i) for i in I])), dtype=np.int32)
    return [coords[:, k].copy() for k in range(len(I))]


def rand_coo(rng, I, nnz):
    """nnz distinct coordinates drawn uniformly, values N(0,1) (float32)."""
    total = int(np.prod(I))
    flat = rng.choice(total, size=nnz, replace=False)
    idx = list(np.unravel_index(flat, I))
    idx = [i.astype(np.int32) for i in idx]
    val = rng.normal(0, 1, nnz).astype(np.float32)
    return idx, val


def dense_tucker(A, B):
    """X^ = G x_1 A1 ... x_N AN with G = sum_r b1_r o ... o bN_r (brute force)."""
    N, R = len(A), B[0].shape[1]
    G = np.zeros([b.shape[0] for b in B])
    for r in range(R):
        outer = B[0][:, r]
        for k in range(1, N):
            outer = np.multiply.outer(outer, B[k][:, r])
        G += outer
    X = G
    for k in range(N):
        # (X x_k A)_{..i_k..} = sum_{j_k} X_{..j_k..} A[i_k, j_k]
        X = np.moveaxis(np.tensordot(A[k], X, axes=([1], [k])), 0, k)
    return X


def kron_chain(mats):
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def khatri_rao_chain(mats):
    out = mats[0]
    for m in mats[1:]:
        cols = [np.kron(out[:, r], m[:, r]) for r in range(out.shape[1])]
        out = np.stack(cols, axis=1)
    return out


def unfold(X, n):
    """Mode-n matricisation: column j = sum_{k != n} i_k prod_{m < k, m != n} I_m
    (0-based; Definition "n-Mode Tensor Matricization")."""
    N = X.ndim
    others = [k for k in range(N) if k != n]
    # Fortran order over the remaining modes makes i_k with the smallest k fastest
    return np.transpose(X, [n] + others).reshape(X.shape[n], -1, order="F")


# ----------------------------------------------------------------------------- generator pins


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_rows(name):
    """Non-comment rows of a fixture under tests/golden/, split on whitespace."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_splitmix64_reference_outputs():
    """SplitMix64 with state 0: the first outputs of the published generator
    (tests/golden/splitmix64_state0.txt)."""
    from paper_2210_06014_gb300 import synth
    want = [int(r[0], 16) for r in golden_rows("splitmix64_state0.txt")]
    got = [int(v) & ((1 << 64) - 1) for v in synth.bits(0, len(want)).tolist()]
    assert got == want


def test_ratings_stand_in_has_the_netflix_shape():
    """The synthetic ratings tensor stands in for the paper's Netflix tensor
    (table "Real World Datasets", tests/golden/real_world_datasets.txt): mode
    lengths within 1 %, total nonzeros within 1 % of |Omega| + |Gamma|, and
    integer ratings inside the printed value range."""
    from paper_2210_06014_gb300 import synth
    rows = {r[0]: r[1:] for r in golden_rows("real_world_datasets.txt")}
    I1, I2, I3, omega, gamma = (int(x) for x in rows["netflix"][:5])
    vmax, vmin = float(rows["netflix"][5]), float(rows["netflix"][6])
    spec = synth.spec_ratings()
    for got, want in zip(spec.dims, (I1, I2, I3)):
        assert abs(got - want) <= 0.01 * want, (got, want)
    assert abs(spec.nnz - (omega + gamma)) <= 0.01 * (omega + gamma)
    T = synth.make_tensor(synth.spec_ratings(nnz=200_000))
    vals = np.concatenate([T.val.numpy(), T.test_val.numpy()])
    assert vals.min() >= vmin and vals.max() <= vmax
    assert np.all(vals == np.round(vals))


def test_generator_distinct_and_in_range():
    from paper_2210_06014_gb300 import synth
    T = synth.make_tensor(synth.spec_small())
    assert T.nnz == 200_000
    keys = np.zeros(T.nnz, dtype=np.int64)
    for i, I in zip(T.idx, T.spec.dims):
        a = i.numpy().astype(np.int64)
        assert a.min() >= 0 and a.max() < I
        keys = keys * I + a
    assert len(np.unique(keys)) == T.nnz


# ----------------------------------------------------------------------------- refresh (Algorithm 3)


def test_refresh_is_the_matrix_product(oracle_mod):
    rng = np.random.default_rng(1)
    A, B = rand_model(rng, (37, 5, 11), (3, 7, 4), 6)
    m = oracle_mod.Model(A, B)
    for n in range(3):
        np.testing.assert_allclose(m.C[n], A[n] @ B[n], rtol=1e-13, atol=1e-14)


# ----------------------------------------------------------------------------- prediction (Eq. (1), (3), (12))


@pytest.mark.parametrize("I,J,R", [((4, 3, 5), (2, 3, 2), 3), ((3, 2, 4, 3), (2, 2, 3, 2), 4),
                                   ((5, 6), (3, 2), 2)])
def test_predictions_match_dense_tucker(oracle_mod, I, J, R):
    rng = np.random.default_rng(2)
    A, B = rand_model(rng, I, J, R)
    m = oracle_mod.Model(A, B)
    idx = all_coords(I)
    X = dense_tucker(A, B)
    want = X[tuple(idx)]
    np.testing.assert_allclose(m.predict(idx), want, rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(m.predict_direct(idx), want, rtol=1e-12, atol=1e-13)


def test_predictions_match_matricised_form(oracle_mod):
    """Eq. (3): X^(n) = A^(n) B^(n) Q^(n)T S^(n)T, Q = Khatri-Rao and S =
    Kronecker products over the other modes in descending mode order."""
    rng = np.random.default_rng(3)
    I, J, R = (4, 3, 5, 2), (2, 3, 2, 2), 3
    A, B = rand_model(rng, I, J, R)
    m = oracle_mod.Model(A, B)
    idx = all_coords(I)
    X = np.zeros(I)
    X[tuple(idx)] = m.predict(idx)
    N = len(I)
    for n in range(N):
        others = [k for k in reversed(range(N)) if k != n]
        Q = khatri_rao_chain([B[k] for k in others])
        S = kron_chain([A[k] for k in others])
        Xn = A[n] @ B[n] @ Q.T @ S.T
        np.testing.assert_allclose(unfold(X, n), Xn, rtol=1e-12, atol=1e-13)


def test_kronecker_product_identity():
    """Eq. (12): (a_N kron ... kron a_1)(b_N kron ... kron b_1) = prod_k a_k . b_k,
    the identity behind the cached products."""
    rng = np.random.default_rng(4)
    a = [rng.normal(size=j) for j in (3, 2, 4)]
    b = [rng.normal(size=j) for j in (3, 2, 4)]
    lhs = kron_chain(a[::-1]) @ kron_chain(b[::-1])
    rhs = np.prod([x @ y for x, y in zip(a, b)])
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_gauge_and_column_permutation_invariance(oracle_mod):
    rng = np.random.default_rng(5)
    I, J, R = (6, 5, 4), (3, 3, 2), 4
    A, B = rand_model(rng, I, J, R)
    idx = all_coords(I)
    base = oracle_mod.Model(A, B).predict(idx)
    A2, B2 = [a.copy() for a in A], [b.copy() for b in B]
    for n in range(3):
        M = rng.normal(size=(J[n], J[n])) + 3 * np.eye(J[n])
        A2[n] = A[n] @ M
        B2[n] = np.linalg.solve(M, B[n])
    np.testing.assert_allclose(oracle_mod.Model(A2, B2).predict(idx), base, rtol=1e-10, atol=1e-12)
    perm = rng.permutation(R)
    B3 = [b[:, perm] for b in B]
    np.testing.assert_allclose(oracle_mod.Model(A, B3).predict(idx), base, rtol=1e-12, atol=1e-13)


def test_loss_sums(oracle_mod):
    rng = np.random.default_rng(6)
    I, J, R = (5, 4, 3), (2, 2, 3), 2
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 25)
    m = oracle_mod.Model(A, B)
    X = dense_tucker(A, B)
    e = val.astype(np.float64) - X[tuple(idx)]
    sse, sae = m.loss(idx, val)
    assert abs(sse - np.sum(e * e)) <= 1e-12 * np.sum(e * e)
    assert abs(sae - np.sum(np.abs(e))) <= 1e-12 * np.sum(np.abs(e))


# ----------------------------------------------------------------------------- factor step (Eq. (7), (9), (10))


def _objective_factor_batch(A, B, n, idx, val, rows_sel, lam):
    """sum over the batch of 1/2 e_s^2 + 1/2 lam ||a_{i_n(s)}||^2 (per occurrence),
    evaluated by the dense reconstruction."""
    X = dense_tucker(A, B)
    e = val.astype(np.float64)[rows_sel] - X[tuple(i[rows_sel] for i in idx)]
    reg = sum(np.sum(A[n][idx[n][s]] ** 2) for s in rows_sel)
    return 0.5 * np.sum(e * e) + 0.5 * lam * reg


@pytest.mark.parametrize("batch", [1, "all"])
def test_factor_step_is_minus_gradient(oracle_mod, batch):
    """One factor minibatch step equals lr times minus the gradient of the
    batch objective (central differences, h = 1e-6).  With batch = 1 this is
    Eq. (10); with the whole tensor as one batch it checks the summing of
    duplicate rows and the per-occurrence regulariser."""
    rng = np.random.default_rng(7)
    I, J, R = (4, 5, 3), (2, 3, 2), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 1 if batch == 1 else 18)
    lr, lam, n, h = 0.05, 0.1, 1, 1e-6
    m = oracle_mod.Model(A, B)
    m.factor_pass(n, idx, val, batch=1 if batch == 1 else len(val), lr=lr, lam=lam)
    step = (m.A[n] - A[n]) / lr
    sel = np.arange(len(val))
    grad = np.zeros_like(A[n])
    for i in range(I[n]):
        for j in range(J[n]):
            Ap, Am = [a.copy() for a in A], [a.copy() for a in A]
            Ap[n][i, j] += h
            Am[n][i, j] -= h
            grad[i, j] = (_objective_factor_batch(Ap, B, n, idx, val, sel, lam)
                          - _objective_factor_batch(Am, B, n, idx, val, sel, lam)) / (2 * h)
    np.testing.assert_allclose(step, -grad, rtol=1e-6, atol=1e-8)


def test_factor_pass_distinct_rows_equals_sequential(oracle_mod):
    """When no row repeats inside a minibatch the minibatch rule and the
    element-by-element rule of Algorithm 4 coincide (rows are independent)."""
    rng = np.random.default_rng(8)
    I, J, R = (30, 4, 5), (3, 2, 2), 3
    A, B = rand_model(rng, I, J, R)
    n = 0
    # 4 batches of 6 samples, each batch with distinct mode-0 rows
    rows = np.concatenate([rng.permutation(30)[:6] for _ in range(4)]).astype(np.int32)
    idx = [rows, rng.integers(0, 4, 24).astype(np.int32), rng.integers(0, 5, 24).astype(np.int32)]
    val = rng.normal(size=24).astype(np.float32)
    m1, m6 = oracle_mod.Model(A, B), oracle_mod.Model(A, B)
    m1.factor_pass(n, idx, val, batch=1, lr=0.1, lam=0.05)
    m6.factor_pass(n, idx, val, batch=6, lr=0.1, lam=0.05)
    np.testing.assert_allclose(m6.A[n], m1.A[n], rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3])
def test_identity_core_reduces_to_cp_sgd(oracle_mod, N):
    """J_n = R and B^(n) = I: the model is CP (N = 2: matrix factorisation) and
    the factor step is plain CP-SGD, written here from its textbook form."""
    rng = np.random.default_rng(9)
    R = 3
    I = (7, 6, 5)[:N]
    U = [rng.normal(0, 0.6, (i, R)) for i in I]
    B = [np.eye(R) for _ in range(N)]
    idx, val = rand_coo(rng, I, 40)
    perm = rng.permutation(40).astype(np.uint32)
    lr, lam = 0.07, 0.02
    for n in range(N):
        m = oracle_mod.Model(U, B)
        m.factor_pass(n, idx, val, perm=perm, batch=1, lr=lr, lam=lam)
        W = [u.copy() for u in U]
        for s in perm:
            co = [idx[k][s] for k in range(N)]
            other = np.ones(R)
            for k in range(N):
                if k != n:
                    other *= W[k][co[k]]
            a = W[n][co[n]]
            e = float(val[s]) - float(a @ other)
            W[n][co[n]] = a + lr * (e * other - lam * a)
        np.testing.assert_allclose(m.A[n], W[n], rtol=1e-12, atol=1e-14)


# ----------------------------------------------------------------------------- core step (Eq. (8), (9), (11))


@pytest.mark.parametrize("batch", [1, 5, "all"])
def test_core_step_is_minus_gradient(oracle_mod, batch):
    """The first core minibatch step equals lr times minus the gradient of
    (1/M) sum_s 1/2 e_s^2 + 1/2 lam ||B||^2 (central differences)."""
    rng = np.random.default_rng(10)
    I, J, R = (4, 3, 5), (2, 3, 2), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 12)
    M = len(val) if batch == "all" else batch
    lr, lam, n, h = 0.05, 0.1, 2, 1e-6
    m = oracle_mod.Model(A, B)
    sub_idx = [i[:M] for i in idx]
    sub_val = val[:M]
    m.core_pass(n, sub_idx, sub_val, batch=M, lr=lr, lam=lam)
    step = (m.B[n] - B[n]) / lr

    def f(Bk):
        X = dense_tucker(A, Bk)
        e = sub_val.astype(np.float64) - X[tuple(sub_idx)]
        return 0.5 * np.mean(e * e) + 0.5 * lam * np.sum(Bk[n] ** 2)

    grad = np.zeros_like(B[n])
    for j in range(J[n]):
        for r in range(R):
            Bp, Bm = [b.copy() for b in B], [b.copy() for b in B]
            Bp[n][j, r] += h
            Bm[n][j, r] -= h
            grad[j, r] = (f(Bp) - f(Bm)) / (2 * h)
    np.testing.assert_allclose(step, -grad, rtol=1e-6, atol=1e-8)


def test_core_batches_are_sequential(oracle_mod):
    """Two core minibatches = two separate single-batch passes (the second one
    sees the core matrix moved by the first)."""
    rng = np.random.default_rng(11)
    I, J, R = (6, 5, 4), (2, 3, 2), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 20)
    m = oracle_mod.Model(A, B)
    m.core_pass(1, idx, val, batch=10, lr=0.05, lam=0.01)
    m2 = oracle_mod.Model(A, B)
    m2.core_pass(1, [i[:10] for i in idx], val[:10], batch=10, lr=0.05, lam=0.01)
    m2.core_pass(1, [i[10:] for i in idx], val[10:], batch=10, lr=0.05, lam=0.01)
    np.testing.assert_allclose(m.B[1], m2.B[1], rtol=1e-14, atol=1e-16)


# ----------------------------------------------------------------------------- whole iteration (Algorithm 2)


def _written_out_epoch(m, idx, val, pf, pc, bf, bc, lr_A, lam_A, lr_B, lam_B, variant="alg2"):
    """Algorithm 2's loop body written out from the separately pinned passes:
    for every mode a factor pass then a refresh of that mode's cached product,
    then for every mode a core pass then a refresh.  The other variants are
    plausible misreadings, kept to show that the test tensor tells them apart."""
    N = m.N
    if variant == "core_first":
        for n in range(N):
            m.core_pass(n, idx, val, perm=pc[n], batch=bc, lr=lr_B, lam=lam_B)
            m.refresh(n)
        for n in range(N):
            m.factor_pass(n, idx, val, perm=pf[n], batch=bf, lr=lr_A, lam=lam_A)
            m.refresh(n)
        return
    for n in range(N):
        m.factor_pass(n, idx, val, perm=pf[n], batch=bf, lr=lr_A, lam=lam_A)
        if variant == "no_factor_refresh":
            continue
        m.refresh((n + 1) % N if variant == "wrong_mode_refresh" else n)
    if variant == "no_factor_refresh":
        m.refresh_all()
    for n in range(N):
        m.core_pass(n, idx, val, perm=pc[n], batch=bc, lr=lr_B, lam=lam_B)
        m.refresh(n)


def test_epoch_follows_algorithm2_schedule(oracle_mod):
    """orc_epoch equals Algorithm 2 written out pass by pass (factor module
    over every mode, each followed by a refresh of that mode; then the core
    module likewise), with a distinct permutation per pass, to 1e-14.  The
    misreadings (modules swapped, a refresh of the wrong mode, no refresh after
    the factor passes) move the parameters by far more on the same input, so
    the comparison would catch them."""
    rng = np.random.default_rng(21)
    I, J, R = (7, 6, 5), (3, 2, 3), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 60)
    pf = [rng.permutation(60).astype(np.uint32) for _ in range(3)]
    pc = [rng.permutation(60).astype(np.uint32) for _ in range(3)]
    args = dict(bf=4, bc=8, lr_A=0.05, lam_A=0.01, lr_B=0.07, lam_B=0.02)
    got = oracle_mod.Model(A, B)
    for _ in range(2):  # two epochs: the second starts from the first's result
        got.epoch(idx, val, pf, pc, batch_factor=args["bf"], batch_core=args["bc"],
                  lr_A=args["lr_A"], lam_A=args["lam_A"], lr_B=args["lr_B"], lam_B=args["lam_B"])
    want = oracle_mod.Model(A, B)
    for _ in range(2):
        _written_out_epoch(want, idx, val, pf, pc, **args)
    for n in range(3):
        np.testing.assert_allclose(got.A[n], want.A[n], rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(got.B[n], want.B[n], rtol=1e-14, atol=1e-16)
        np.testing.assert_allclose(got.C[n], want.C[n], rtol=1e-14, atol=1e-16)
    for variant in ("core_first", "wrong_mode_refresh", "no_factor_refresh"):
        wrong = oracle_mod.Model(A, B)
        for _ in range(2):
            _written_out_epoch(wrong, idx, val, pf, pc, variant=variant, **args)
        diff = max(float(np.abs(wrong.A[n] - want.A[n]).max()) for n in range(3))
        diff = max(diff, max(float(np.abs(wrong.B[n] - want.B[n]).max()) for n in range(3)))
        assert diff > 1e-6, variant


def test_factor_pass_rounding_scale(oracle_mod):
    """The rounding scales returned with a factor pass are the sums they are
    documented to be, re-derived here by stepping the pass in numpy (batch 1):
    S1 = sum_s lr((|x| + |a|.|v|)|v| + lam |a|) with |v| = |B^(n)| prod |A||B|
    rows, S2 = sum_s |a| at each step; the pass itself is unchanged."""
    rng = np.random.default_rng(22)
    I, J, R = (5, 4, 3), (2, 3, 2), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 30)
    n, lr, lam = 1, 0.1, 0.02
    m = oracle_mod.Model(A, B)
    S1, S2 = m.factor_pass_scaled(n, idx, val, batch=1, lr=lr, lam=lam)
    plain = oracle_mod.Model(A, B)
    plain.factor_pass(n, idx, val, batch=1, lr=lr, lam=lam)
    np.testing.assert_array_equal(m.A[n], plain.A[n])
    a = A[n].copy()
    C = [x @ y for x, y in zip(A, B)]
    absC = [np.abs(x) @ np.abs(y) for x, y in zip(A, B)]
    w1, w2 = np.zeros_like(a), np.zeros_like(a)
    for s in range(len(val)):
        i = idx[n][s]
        p = np.ones(R)
        pa = np.ones(R)
        for k in range(3):
            if k != n:
                p *= C[k][idx[k][s]]
                pa *= absC[k][idx[k][s]]
        v = B[n] @ p
        va = np.abs(B[n]) @ pa
        e = float(val[s]) - a[i] @ v
        w1[i] += lr * ((abs(float(val[s])) + np.abs(a[i]) @ va) * va + lam * np.abs(a[i]))
        w2[i] += np.abs(a[i])
        a[i] = a[i] + lr * (e * v - lam * a[i])
    np.testing.assert_allclose(S1, w1, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(S2, w2, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m.A[n], a, rtol=1e-12, atol=1e-15)


@pytest.mark.slow
def test_planted_recovery(oracle_mod):
    """A noise-free planted J=R=3 model on a well-sampled 30x30x30 tensor is
    fitted: the training RMSE falls below 5% of std(x) (Algorithm 2 with
    per-element factor steps and small core minibatches)."""
    rng = np.random.default_rng(12)
    I, J, R = (30, 30, 30), (3, 3, 3), 3
    sigma = np.sqrt(R ** (-1 / 6) / np.sqrt(3))
    Ap = [rng.normal(0, sigma, (i, j)) for i, j in zip(I, J)]
    Bp = [rng.normal(0, sigma, (j, R)) for j in J]
    total = int(np.prod(I))
    flat = rng.choice(total, size=6000, replace=False)
    idx = [i.astype(np.int32) for i in np.unravel_index(flat, I)]
    val = dense_tucker(Ap, Bp)[tuple(idx)].astype(np.float32)
    A0 = [rng.normal(0, sigma, (i, j)) for i, j in zip(I, J)]
    B0 = [rng.normal(0, sigma, (j, R)) for j in J]
    m = oracle_mod.Model(A0, B0)
    std = float(np.std(val.astype(np.float64)))
    hist = []
    for ep in range(200):
        pf = [rng.permutation(len(val)).astype(np.uint32) for _ in range(3)]
        pc = [rng.permutation(len(val)).astype(np.uint32) for _ in range(3)]
        m.epoch(idx, val, pf, pc, batch_factor=1, batch_core=64, lr_A=0.02, lam_A=1e-4,
                lr_B=0.02, lam_B=1e-4)
        hist.append(m.rmse(idx, val))
        if hist[-1] < 0.05 * std:
            break
    assert hist[-1] < 0.05 * std, (std, hist[::20])


# ----------------------------------------------------------------------------- loss gradient


def test_loss_gradient_is_central_difference(oracle_mod):
    """dL/dA and dL/dB of L = 1/2 sum e^2 match central differences of the
    dense-reconstruction loss (h = 1e-6) for every entry of every matrix."""
    rng = np.random.default_rng(13)
    I, J, R = (4, 3, 5), (2, 3, 2), 3
    A, B = rand_model(rng, I, J, R)
    idx, val = rand_coo(rng, I, 20)
    m = oracle_mod.Model(A, B)
    L, gA, gB = m.loss_grad(idx, val)

    def f(As, Bs):
        X = dense_tucker(As, Bs)
        e = val.astype(np.float64) - X[tuple(idx)]
        return 0.5 * np.sum(e * e)

    assert abs(L - f(A, B)) <= 1e-12 * abs(L)
    h = 1e-6
    for n in range(3):
        for i in range(I[n]):
            for j in range(J[n]):
                Ap, Am = [a.copy() for a in A], [a.copy() for a in A]
                Ap[n][i, j] += h
                Am[n][i, j] -= h
                fd = (f(Ap, B) - f(Am, B)) / (2 * h)
                assert abs(gA[n][i, j] - fd) <= 1e-7 * (1 + abs(fd))
        for j in range(J[n]):
            for r in range(R):
                Bp, Bm = [b.copy() for b in B], [b.copy() for b in B]
                Bp[n][j, r] += h
                Bm[n][j, r] -= h
                fd = (f(A, Bp) - f(A, Bm)) / (2 * h)
                assert abs(gB[n][j, r] - fd) <= 1e-7 * (1 + abs(fd))
