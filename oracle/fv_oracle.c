/*
 * Fisher-vector oracle: plain, slow, double-precision CPU encoder.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference that the GPU path is
 * checked against. Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product library never does, and it
 * shares no code, header or constant with the CUDA sources.
 *
 * Method (paper Sec. 3.1, Algorithm 1, "Fisher Vector Encoding Algorithm"),
 * followed step by step in the paper's order:
 *   1. precompute 1/sqrt(sigma^2) per component and dimension
 *      (the "compute sqrt(sigma^-1)" step; the paper's "covariances" are
 *      the diagonal variances sigma^2);
 *   2. per descriptor i and component k: distance
 *        d_ik = sum_d ((x_id - mu_kd) / sigma_kd)^2
 *      (centred form, no expansion), log-posterior with the prior
 *        l_ik = log w_k - 1/2 sum_d log sigma^2_kd - 1/2 d_ik
 *      (the -D/2 log 2pi term is common to all k and cancels), and the
 *      running maximum over k;
 *   3. gamma_ik = exp(l_ik - max_k l_ik) / sum_k exp(l_ik - max_k l_ik);
 *   4. for every (i, k) with gamma_ik > tau and every d, with
 *      t = (x_id - mu_kd) / sigma_kd:
 *        U_kd += gamma_ik * t,   V_kd += gamma_ik * (t^2 - 1);
 *      tau = 0 keeps every term (the exact encoding); the paper's
 *      early-termination threshold (Sec. 3.3, Algorithm 5) is 1e-6;
 *   5. the improved-FV scaling of the encoding scheme the paper adopts
 *      (Sec. 4, "the same encoding scheme as VLFeat"):
 *        u_kd = U_kd / (N sqrt(w_k)),   v_kd = V_kd / (N sqrt(2 w_k));
 *   6. z = [u_0 .. u_{K-1}, v_0 .. v_{K-1}] (each block D-contiguous),
 *      z_j <- sign(z_j) sqrt(|z_j|), z <- z / ||z||_2 (left as zeros when
 *      the norm is zero).
 *
 * All arithmetic is IEEE double with libm exp/log/sqrt. Parity pins for every
 * step live in the oracle tests (posteriors against a library mixture model,
 * U/V against autograd gradients of the log-likelihood, K=1 and
 * identical-component closed forms, invariances, hard assignment).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FVO_OK 0
#define FVO_EMPTY 1
#define FVO_BADARG 2
#define FVO_NOMEM 3

/* Step 1's per-component constant of the log posterior,
 *   c_k = log w_k - 1/2 sum_d log sigma^2_kd
 * (Algorithm 1: the prior and the Gaussian normaliser; the -D/2 log 2pi term
 * is common to every component and cancels in the posteriors). */
int fvo_log_constants(int D, int K, const double *w, const double *var, double *cst) {
    if (D <= 0 || K <= 0 || !w || !var || !cst) return FVO_BADARG;
    for (int k = 0; k < K; ++k) {
        double slog = 0.0;
        for (int d = 0; d < D; ++d) slog += log(var[(int64_t)k * D + d]);
        cst[k] = log(w[k]) - 0.5 * slog;
    }
    return FVO_OK;
}

int fvo_encode(int64_t N, int D, int K,
               const double *X,    /* N x D, row-major */
               const double *w,    /* K priors */
               const double *mu,   /* K x D means */
               const double *var,  /* K x D diagonal variances */
               double tau,         /* posterior threshold (0 = exact) */
               double *fv,         /* out 2KD: normalised Fisher vector */
               double *fv_raw,     /* out 2KD or NULL: [u; v] before sqrt/L2 */
               double *gamma_out,  /* out N x K or NULL: posteriors */
               double *U_out,      /* out K x D or NULL: unscaled first order */
               double *V_out,      /* out K x D or NULL: unscaled second order */
               double *S0_out)     /* out K or NULL: sum_i gamma_ik (terms > tau) */
{
    if (D <= 0 || K <= 0 || N < 0 || !X || !w || !mu || !var || !fv) return FVO_BADARG;
    const int64_t KD = (int64_t)K * D;
    memset(fv, 0, sizeof(double) * 2 * KD);
    if (fv_raw) memset(fv_raw, 0, sizeof(double) * 2 * KD);
    if (N == 0) return FVO_EMPTY;

    double *isd = (double *)malloc(sizeof(double) * KD);   /* 1/sigma */
    double *cst = (double *)malloc(sizeof(double) * K);    /* log w - 1/2 sum log var */
    double *U = (double *)calloc((size_t)KD, sizeof(double));
    double *V = (double *)calloc((size_t)KD, sizeof(double));
    double *S0 = (double *)calloc((size_t)K, sizeof(double));
    double *post = gamma_out ? gamma_out : (double *)malloc(sizeof(double) * (size_t)(N * K));
    if (!isd || !cst || !U || !V || !S0 || !post) {
        free(isd); free(cst); free(U); free(V); free(S0);
        if (post != gamma_out) free(post);
        return FVO_NOMEM;
    }

    /* Step 1: sqrt(sigma^-1), i.e. 1/sigma, and the per-component constant. */
    for (int64_t j = 0; j < KD; ++j) isd[j] = 1.0 / sqrt(var[j]);
    fvo_log_constants(D, K, w, var, cst);

    /* Steps 2-3: posteriors of every descriptor (first phase). */
    for (int64_t i = 0; i < N; ++i) {
        const double *x = X + i * D;
        double *p = post + i * K;
        double maxpost = -INFINITY;
        for (int k = 0; k < K; ++k) {
            double dist = 0.0;
            for (int d = 0; d < D; ++d) {
                double t = (x[d] - mu[(int64_t)k * D + d]) * isd[(int64_t)k * D + d];
                dist += t * t;
            }
            p[k] = cst[k] - 0.5 * dist;
            if (p[k] > maxpost) maxpost = p[k];
        }
        double sum = 0.0;
        for (int k = 0; k < K; ++k) {
            p[k] = exp(p[k] - maxpost);
            sum += p[k];
        }
        for (int k = 0; k < K; ++k) p[k] = p[k] / sum;
    }

    /* Step 4: first- and second-order statistics (second phase). */
    for (int64_t i = 0; i < N; ++i) {
        const double *x = X + i * D;
        const double *p = post + i * K;
        for (int k = 0; k < K; ++k) {
            double g = p[k];
            if (!(g > tau)) continue;
            S0[k] += g;
            for (int d = 0; d < D; ++d) {
                double t = (x[d] - mu[(int64_t)k * D + d]) * isd[(int64_t)k * D + d];
                U[(int64_t)k * D + d] += t * g;
                V[(int64_t)k * D + d] += (t * t - 1.0) * g;
            }
        }
    }

    /* Step 5: improved-FV scaling; step 6: signed square root, L2. */
    double nrm2 = 0.0;
    for (int k = 0; k < K; ++k) {
        double su = 1.0 / ((double)N * sqrt(w[k]));
        double sv = 1.0 / ((double)N * sqrt(2.0 * w[k]));
        for (int d = 0; d < D; ++d) {
            double u = U[(int64_t)k * D + d] * su;
            double v = V[(int64_t)k * D + d] * sv;
            if (fv_raw) {
                fv_raw[(int64_t)k * D + d] = u;
                fv_raw[KD + (int64_t)k * D + d] = v;
            }
            double zu = (u > 0) ? sqrt(u) : ((u < 0) ? -sqrt(-u) : 0.0);
            double zv = (v > 0) ? sqrt(v) : ((v < 0) ? -sqrt(-v) : 0.0);
            fv[(int64_t)k * D + d] = zu;
            fv[KD + (int64_t)k * D + d] = zv;
            nrm2 += zu * zu + zv * zv;
        }
    }
    if (nrm2 > 0.0) {
        double inv = 1.0 / sqrt(nrm2);
        for (int64_t j = 0; j < 2 * KD; ++j) fv[j] *= inv;
    }

    if (U_out) memcpy(U_out, U, sizeof(double) * KD);
    if (V_out) memcpy(V_out, V, sizeof(double) * KD);
    if (S0_out) memcpy(S0_out, S0, sizeof(double) * K);
    free(isd); free(cst); free(U); free(V); free(S0);
    if (post != gamma_out) free(post);
    return FVO_OK;
}
