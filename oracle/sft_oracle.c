/*
 * sft_oracle.c -- plain FP64 reference of sparse FastTucker SGD as defined in
 * "cuFasterTucker: A Stochastic Optimization Strategy for Parallel Sparse
 * FastTucker Decomposition on GPU Platform" (arXiv 2210.06014).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA library, and the CUDA library never calls it.
 *
 * Everything is single-threaded, unblocked and computed in double precision,
 * in the order the paper states, so that each function can be read against the
 * paper by eye:
 *
 *   model            Eq. (1): X^ = (sum_r b1_r o ... o bN_r) x_1 A1 ... x_N AN,
 *                    evaluated per nonzero through Eq. (12):
 *                    x^ = sum_r prod_k (a^(k)_{i_k} . b^(k)_{:,r})
 *   cached products  Section "Reusable Intermediate Variables", Algorithm 3:
 *                    C^(n) = A^(n) B^(n)
 *   SGD rule         Eq. (9)
 *   factor gradient  Eq. (10): -(x - a v) v^T + lambda_A a,  v = B^(n) p
 *   core gradient    Eq. (11): -(x - a v) a^T p_r + lambda_B b_{:,r}
 *   epoch schedule   Algorithm 2
 *   RMSE / MAE       Section "Real-world accuracy"
 *
 * Readings of the paper taken here (the paper is garbled or silent on them):
 *   - update signs follow Eq. (10)/(11): a += lr (e v - lambda a),
 *     B += lr (G / M_b - lambda B) with G = sum_s e_s a_s p_s^T
 *     (Algorithm 4 and 5 print the descent step with a wrong sign);
 *   - the factor 2 of the squared loss is absorbed into the learning rate;
 *   - factor rows: within one minibatch every prediction uses the factor
 *     matrix as it stood at the start of the minibatch; the per-sample terms
 *     (e v - lambda a) of a row are summed in sample order and applied once;
 *     no 1/M scaling (Algorithm 4 updates per element with no averaging, and
 *     batch = 1 reproduces that exactly);
 *   - core matrices: the batch gradient is divided by the true size M_b of the
 *     batch (Eq. (9)); batch = nnz reproduces Algorithm 5's single update
 *     per mode pass;
 *   - regularisation is applied per occurrence (Eq. (7)/(8) are per element);
 *   - the sample order is a caller-supplied permutation (NULL = identity).
 *
 * Index arrays are int32 structure-of-arrays idx[k][s]; values are float32,
 * the storage format of the GPU path.  They are widened to int64 / double on
 * read, which is exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAX_ORDER 16

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };

/* Algorithm 3 / Section "Reusable Intermediate Variables":
 * C[i][r] = sum_j A[i][j] * B[j][r], every row i, every r. */
void orc_refresh(int64_t I, int J, int R, const double *A, const double *B, double *C)
{
    for (int64_t i = 0; i < I; ++i) {
        for (int r = 0; r < R; ++r) {
            double acc = 0.0;
            for (int j = 0; j < J; ++j)
                acc += A[i * J + j] * B[(int64_t)j * R + r];
            C[i * R + r] = acc;
        }
    }
}

static int64_t sample_index(const uint32_t *perm, int64_t pos)
{
    return perm ? (int64_t)perm[pos] : pos;
}

/* Eq. (12) with the cached products: x^ = sum_r prod_k C^(k)[i_k][r]. */
static double predict_cached(int N, int R, const double *const *C,
                             const int32_t *const *idx, int64_t s)
{
    double xh = 0.0;
    for (int r = 0; r < R; ++r) {
        double prod = 1.0;
        for (int k = 0; k < N; ++k)
            prod *= C[k][(int64_t)idx[k][s] * R + r];
        xh += prod;
    }
    return xh;
}

void orc_predict_cached(int N, int R, const double *const *C, const int32_t *const *idx,
                        int64_t nnz, double *out)
{
    for (int64_t s = 0; s < nnz; ++s)
        out[s] = predict_cached(N, R, C, idx, s);
}

/* The cache-free way of Algorithm 1: every a^(k)_{i_k} . b^(k)_{:,r} is
 * recomputed for every nonzero (the FastTucker cost the paper removes). */
void orc_predict_direct(int N, const int *J, int R, const double *const *A,
                        const double *const *B, const int32_t *const *idx,
                        int64_t nnz, double *out)
{
    for (int64_t s = 0; s < nnz; ++s) {
        double xh = 0.0;
        for (int r = 0; r < R; ++r) {
            double prod = 1.0;
            for (int k = 0; k < N; ++k) {
                const double *a = A[k] + (int64_t)idx[k][s] * J[k];
                double dot = 0.0;
                for (int j = 0; j < J[k]; ++j)
                    dot += a[j] * B[k][(int64_t)j * R + r];
                prod *= dot;
            }
            xh += prod;
        }
        out[s] = xh;
    }
}

/* p_r = prod_{k != n} C^(k)[i_k][r]  (the s^(n) q^(n)_{:,r} of Eq. (12)). */
static void hadamard_others(int N, int R, int n, const double *const *C,
                            const int32_t *const *idx, int64_t s, double *p)
{
    for (int r = 0; r < R; ++r) {
        double prod = 1.0;
        for (int k = 0; k < N; ++k) {
            if (k == n)
                continue;
            prod *= C[k][(int64_t)idx[k][s] * R + r];
        }
        p[r] = prod;
    }
}

/* v = B^(n) p, the shared intermediate B^(n) Q^(n)T s^(n)T of Eq. (10). */
static void core_times(int J, int R, const double *B, const double *p, double *v)
{
    for (int j = 0; j < J; ++j) {
        double acc = 0.0;
        for (int r = 0; r < R; ++r)
            acc += B[(int64_t)j * R + r] * p[r];
        v[j] = acc;
    }
}

/* |c^(k)_i|_r bound: sum_j |A^(k)[i][j]| |B^(k)[j][r]| (the magnitude a float32
 * refresh of that row rounds against), used only by the rounding scale below. */
static void abs_cached_row(int J, int R, const double *A, const double *B, int64_t i, double *out)
{
    for (int r = 0; r < R; ++r) {
        double acc = 0.0;
        for (int j = 0; j < J; ++j)
            acc += fabs(A[i * J + j]) * fabs(B[(int64_t)j * R + r]);
        out[r] = acc;
    }
}

/* One factor pass over mode n (Algorithm 2, factor module; Eq. (9)-(10)).
 * For each minibatch (consecutive slice of the permutation, the last one
 * shorter):
 *   (i)  with A^(n) as it stood at the start of the batch, every sample s
 *        computes p_s, v_s = B^(n) p_s, x^_s = a_{i_n} . v_s, e_s = x_s - x^_s
 *        and its term t_s = e_s v_s - lambda a_{i_n};
 *   (ii) the terms of each row are summed in sample order and the row moves by
 *        lr times that sum.
 * C^(n) itself is not read (it is stale while A^(n) moves).
 *
 * scale (optional, I_n x J_n, accumulated into) receives, per row and entry,
 * the magnitudes that bound the rounding of a lower-precision run of the same
 * pass: S1 = sum over the row's samples of lr ((|x| + |a|.|v|) |v|_j + lambda |a_j|)
 * with |v| = |B^(n)| |p| and |p| = prod_{k != n} |A^(k)| |B^(k)| rows, and
 * S2 = sum over the row's samples of |a_j| (the row as each step reads it).
 * scale[0 .. I_n J_n) holds S1, scale[I_n J_n .. 2 I_n J_n) holds S2.  It
 * does not change the pass. */
static int factor_pass_impl(int N, const int64_t *I, const int *J, int R, int n,
                            double *const *A, const double *const *B, const double *const *C,
                            const int32_t *const *idx, const float *val, const uint32_t *perm,
                            int64_t nnz, int64_t batch, double lr, double lam, double *scale)
{
    if (N < 2 || N > ORC_MAX_ORDER || n < 0 || n >= N || batch < 1 || nnz < 0)
        return ORC_EINVAL;
    const int Jn = J[n];
    const int64_t In = I[n];
    double *An = A[n];
    const double *Bn = B[n];
    double *p = malloc(sizeof(double) * R);
    double *v = malloc(sizeof(double) * Jn);
    double *pa = malloc(sizeof(double) * R);
    double *ca = malloc(sizeof(double) * R);
    double *va = malloc(sizeof(double) * Jn);
    int64_t cap = batch < nnz ? batch : (nnz > 0 ? nnz : 1);
    double *term = malloc(sizeof(double) * (size_t)cap * Jn);
    int64_t *row = malloc(sizeof(int64_t) * (size_t)cap);
    double *delta = malloc(sizeof(double) * (size_t)In * Jn);
    unsigned char *touched = calloc((size_t)In, 1);
    int64_t *order_touched = malloc(sizeof(int64_t) * (size_t)cap);
    if (!p || !v || !pa || !ca || !va || !term || !row || !delta || !touched || !order_touched) {
        free(p); free(v); free(pa); free(ca); free(va); free(term); free(row); free(delta);
        free(touched); free(order_touched);
        return ORC_ENOMEM;
    }
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        int64_t Mb = nnz - b0 < batch ? nnz - b0 : batch;
        /* (i) snapshot predictions and per-sample terms */
        for (int64_t t = 0; t < Mb; ++t) {
            int64_t s = sample_index(perm, b0 + t);
            int64_t i = idx[n][s];
            hadamard_others(N, R, n, C, idx, s, p);
            core_times(Jn, R, Bn, p, v);
            double xh = 0.0;
            for (int j = 0; j < Jn; ++j)
                xh += An[i * Jn + j] * v[j];
            double e = (double)val[s] - xh;
            for (int j = 0; j < Jn; ++j)
                term[t * Jn + j] = e * v[j] - lam * An[i * Jn + j];
            row[t] = i;
            if (scale) {
                for (int r = 0; r < R; ++r)
                    pa[r] = 1.0;
                for (int k = 0; k < N; ++k) {
                    if (k == n)
                        continue;
                    abs_cached_row(J[k], R, A[k], B[k], idx[k][s], ca);
                    for (int r = 0; r < R; ++r)
                        pa[r] *= ca[r];
                }
                double xa = 0.0;
                for (int j = 0; j < Jn; ++j) {
                    double acc = 0.0;
                    for (int r = 0; r < R; ++r)
                        acc += fabs(Bn[(int64_t)j * R + r]) * pa[r];
                    va[j] = acc;
                    xa += fabs(An[i * Jn + j]) * acc;
                }
                const double ea = fabs((double)val[s]) + xa;
                for (int j = 0; j < Jn; ++j) {
                    const double aj = fabs(An[i * Jn + j]);
                    scale[i * Jn + j] += lr * (ea * va[j] + lam * aj);
                    scale[In * Jn + i * Jn + j] += aj;
                }
            }
        }
        /* (ii) per-row sums in sample order, then one move per touched row */
        int64_t ntouched = 0;
        for (int64_t t = 0; t < Mb; ++t) {
            int64_t i = row[t];
            if (!touched[i]) {
                touched[i] = 1;
                order_touched[ntouched++] = i;
                for (int j = 0; j < Jn; ++j)
                    delta[i * Jn + j] = 0.0;
            }
            for (int j = 0; j < Jn; ++j)
                delta[i * Jn + j] += term[t * Jn + j];
        }
        for (int64_t q = 0; q < ntouched; ++q) {
            int64_t i = order_touched[q];
            for (int j = 0; j < Jn; ++j)
                An[i * Jn + j] += lr * delta[i * Jn + j];
            touched[i] = 0;
        }
    }
    free(p); free(v); free(pa); free(ca); free(va); free(term); free(row); free(delta);
    free(touched); free(order_touched);
    return ORC_OK;
}

int orc_factor_pass(int N, const int64_t *I, const int *J, int R, int n,
                    double *const *A, const double *const *B, const double *const *C,
                    const int32_t *const *idx, const float *val, const uint32_t *perm,
                    int64_t nnz, int64_t batch, double lr, double lam)
{
    return factor_pass_impl(N, I, J, R, n, A, B, C, idx, val, perm, nnz, batch, lr, lam, NULL);
}

/* orc_factor_pass plus the rounding scale described above (scale: 2 I_n J_n
 * doubles, zeroed by the caller). */
int orc_factor_pass_scaled(int N, const int64_t *I, const int *J, int R, int n,
                           double *const *A, const double *const *B, const double *const *C,
                           const int32_t *const *idx, const float *val, const uint32_t *perm,
                           int64_t nnz, int64_t batch, double lr, double lam, double *scale)
{
    if (!scale)
        return ORC_EINVAL;
    return factor_pass_impl(N, I, J, R, n, A, B, C, idx, val, perm, nnz, batch, lr, lam, scale);
}

/* One core pass over mode n (Algorithm 2, core module; Eq. (9), (11)).
 * For each minibatch, with B^(n) as it stood at the start of the batch:
 *   G = sum_s e_s a_{i_n(s)} p_s^T  (in sample order),
 *   B^(n) += lr (G / M_b - lambda B^(n)). */
int orc_core_pass(int N, const int64_t *I, const int *J, int R, int n,
                  const double *const *A, double *const *B, const double *const *C,
                  const int32_t *const *idx, const float *val, const uint32_t *perm,
                  int64_t nnz, int64_t batch, double lr, double lam)
{
    (void)I;
    if (N < 2 || N > ORC_MAX_ORDER || n < 0 || n >= N || batch < 1 || nnz < 0)
        return ORC_EINVAL;
    const int Jn = J[n];
    const double *An = A[n];
    double *Bn = B[n];
    double *p = malloc(sizeof(double) * R);
    double *v = malloc(sizeof(double) * Jn);
    double *G = malloc(sizeof(double) * (size_t)Jn * R);
    if (!p || !v || !G) {
        free(p); free(v); free(G);
        return ORC_ENOMEM;
    }
    for (int64_t b0 = 0; b0 < nnz; b0 += batch) {
        int64_t Mb = nnz - b0 < batch ? nnz - b0 : batch;
        memset(G, 0, sizeof(double) * (size_t)Jn * R);
        for (int64_t t = 0; t < Mb; ++t) {
            int64_t s = sample_index(perm, b0 + t);
            int64_t i = idx[n][s];
            hadamard_others(N, R, n, C, idx, s, p);
            core_times(Jn, R, Bn, p, v);
            double xh = 0.0;
            for (int j = 0; j < Jn; ++j)
                xh += An[i * Jn + j] * v[j];
            double e = (double)val[s] - xh;
            for (int j = 0; j < Jn; ++j)
                for (int r = 0; r < R; ++r)
                    G[(int64_t)j * R + r] += e * An[i * Jn + j] * p[r];
        }
        for (int j = 0; j < Jn; ++j)
            for (int r = 0; r < R; ++r) {
                int64_t q = (int64_t)j * R + r;
                Bn[q] += lr * (G[q] / (double)Mb - lam * Bn[q]);
            }
    }
    free(p); free(v); free(G);
    return ORC_OK;
}

/* Sum of squared and of absolute residuals over a set of nonzeros, with the
 * cached products (the quantities behind test RMSE and MAE). */
void orc_loss(int N, int R, const double *const *C, const int32_t *const *idx,
              const float *val, int64_t nnz, double *sse, double *sae)
{
    double s2 = 0.0, s1 = 0.0;
    for (int64_t s = 0; s < nnz; ++s) {
        double e = (double)val[s] - predict_cached(N, R, C, idx, s);
        s2 += e * e;
        s1 += fabs(e);
    }
    *sse = s2;
    *sae = s1;
}

/* Gradient of the sampled loss L = 1/2 sum_s (x_s - x^_s)^2 (the data term of
 * Eq. (6) with the factor 2 absorbed, as in Eq. (10)/(11)) with respect to
 * every factor and core matrix, summed over the nonzeros:
 *   dL/da^(n)_{i_n} = -sum_{s: i_n(s) = i_n} e_s v^(n)_s,   v^(n)_s = B^(n) p^(n)_s
 *   dL/dB^(n)       = -sum_s e_s a^(n)_{i_n(s)} p^(n)_s^T
 * (Eq. (10) and Eq. (11) without the regulariser).  gA[n] (I_n x J_n) and
 * gB[n] (J_n x R) are overwritten.  Also returns L. */
double orc_loss_grad(int N, const int64_t *I, const int *J, int R, const double *const *A,
                     const double *const *B, const double *const *C,
                     const int32_t *const *idx, const float *val, int64_t nnz,
                     double *const *gA, double *const *gB)
{
    for (int n = 0; n < N; ++n) {
        memset(gA[n], 0, sizeof(double) * (size_t)I[n] * J[n]);
        memset(gB[n], 0, sizeof(double) * (size_t)J[n] * R);
    }
    int Jmax = 1;
    for (int n = 0; n < N; ++n)
        if (J[n] > Jmax)
            Jmax = J[n];
    double *p = malloc(sizeof(double) * R);
    double *v = malloc(sizeof(double) * Jmax);
    if (!p || !v) {
        free(p);
        free(v);
        return NAN;
    }
    double loss = 0.0;
    for (int64_t s = 0; s < nnz; ++s) {
        const double e = (double)val[s] - predict_cached(N, R, C, idx, s);
        loss += 0.5 * e * e;
        for (int n = 0; n < N; ++n) {
            const int64_t i = idx[n][s];
            hadamard_others(N, R, n, C, idx, s, p);
            core_times(J[n], R, B[n], p, v);
            for (int j = 0; j < J[n]; ++j) {
                gA[n][i * J[n] + j] -= e * v[j];
                for (int r = 0; r < R; ++r)
                    gB[n][(int64_t)j * R + r] -= e * A[n][i * J[n] + j] * p[r];
            }
        }
    }
    free(p);
    free(v);
    return loss;
}

/* One epoch of Algorithm 2: the factor module over every mode (each followed
 * by a refresh of that mode's cached product), then the core module over every
 * mode (each followed by a refresh).  perm_factor[n] / perm_core[n] give the
 * sample order of each pass (NULL entries = identity).  The caller refreshes
 * every C^(n) once before the first epoch, as Algorithm 2 does before its loop. */
int orc_epoch(int N, const int64_t *I, const int *J, int R,
              double *const *A, double *const *B, double *const *C,
              const int32_t *const *idx, const float *val, int64_t nnz,
              const uint32_t *const *perm_factor, const uint32_t *const *perm_core,
              int64_t batch_factor, int64_t batch_core,
              double lr_A, double lam_A, double lr_B, double lam_B)
{
    for (int n = 0; n < N; ++n) {
        int rc = orc_factor_pass(N, I, J, R, n, A, (const double *const *)B,
                                 (const double *const *)C, idx, val,
                                 perm_factor ? perm_factor[n] : NULL, nnz, batch_factor,
                                 lr_A, lam_A);
        if (rc)
            return rc;
        orc_refresh(I[n], J[n], R, A[n], B[n], C[n]);
    }
    for (int n = 0; n < N; ++n) {
        int rc = orc_core_pass(N, I, J, R, n, (const double *const *)A, B,
                               (const double *const *)C, idx, val,
                               perm_core ? perm_core[n] : NULL, nnz, batch_core,
                               lr_B, lam_B);
        if (rc)
            return rc;
        orc_refresh(I[n], J[n], R, A[n], B[n], C[n]);
    }
    return ORC_OK;
}
