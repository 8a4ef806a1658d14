/*
 * Fisher-vector oracle: plain, slow, double-precision CPU encoder.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference that the GPU path is
 * checked against. Only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it; the product library never does, and it
 * shares no code, header or constant with the CUDA sources.
 *
 * What it computes, stated from the definitions (paper Sec. 3.1 and the
 * encoding scheme adopted in Sec. 4, improved Fisher vectors of FV-ijcv13):
 *
 *   log-likelihood matrix (Sec. 3.1: a diagonal-covariance GMM with priors
 *   w_k, means mu_k and "covariances" sigma^2_k):
 *     L_ik = log w_k + log N(x_i; mu_k, diag sigma^2_k) + (D/2) log 2pi
 *          = log w_k - 1/2 sum_d log sigma^2_kd
 *                    - 1/2 sum_d (x_id - mu_kd)^2 / sigma^2_kd
 *     (the (D/2) log 2pi term is common to every component and cancels);
 *   posteriors (Bayes' rule, the "posteriors" of Algorithm 1):
 *     gamma_ik = exp(L_ik - lse_i),  lse_i = log sum_k exp(L_ik),
 *     with lse_i evaluated around the row maximum so nothing overflows;
 *   gradient statistics (Sec. 3.1, the U and V of Algorithm 1), with the
 *   standardised residual t_ikd = (x_id - mu_kd) / sigma_kd:
 *     U_kd = sum_i gamma_ik t_ikd,   V_kd = sum_i gamma_ik (t_ikd^2 - 1),
 *     S0_k = sum_i gamma_ik, each sum over the terms with gamma_ik > tau
 *     (tau = 0 keeps every term: the exact encoding; the paper's early
 *     termination threshold, Sec. 3.3, is 1e-6);
 *   encoding (Sec. 4, "the same encoding scheme as VLFeat"):
 *     u_kd = U_kd / (N sqrt(w_k)),  v_kd = V_kd / (N sqrt(2 w_k)),
 *     z = [u_0 .. u_{K-1}, v_0 .. v_{K-1}] (each block D-contiguous),
 *     z_j <- sign(z_j) sqrt|z_j|,  z <- z / ||z||_2 (zeros stay zeros).
 *
 * All arithmetic is IEEE double with libm exp/log/sqrt, one definition per
 * function. Parity pins for every function live in the oracle tests
 * (posteriors against a library mixture model, U/V against autograd
 * gradients of the log-likelihood, K=1 and identical-component closed forms,
 * invariances, hard assignment, brute force in 50-digit decimal).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define FVO_OK 0
#define FVO_EMPTY 1
#define FVO_BADARG 2
#define FVO_NOMEM 3

/* The component-only part of L_ik: log w_k - 1/2 sum_d log sigma^2_kd. */
int fvo_log_constants(int D, int K, const double *w, const double *var, double *cst) {
    if (D <= 0 || K <= 0 || !w || !var || !cst) return FVO_BADARG;
    for (int k = 0; k < K; ++k) {
        double slog = 0.0;
        for (int d = 0; d < D; ++d) slog += log(var[(int64_t)k * D + d]);
        cst[k] = log(w[k]) - 0.5 * slog;
    }
    return FVO_OK;
}

/* The N x K log-likelihood matrix L (definition above), row-major. */
int fvo_log_likelihoods(int64_t N, int D, int K, const double *X, const double *w, const double *mu,
                        const double *var, double *L) {
    if (N < 0 || D <= 0 || K <= 0 || !X || !w || !mu || !var || !L) return FVO_BADARG;
    double *cst = (double *)malloc(sizeof(double) * K);
    double *prec = (double *)malloc(sizeof(double) * (size_t)K * D);   /* 1 / sigma^2 */
    if (!cst || !prec) {
        free(cst);
        free(prec);
        return FVO_NOMEM;
    }
    fvo_log_constants(D, K, w, var, cst);
    for (int64_t j = 0; j < (int64_t)K * D; ++j) prec[j] = 1.0 / var[j];
    for (int64_t i = 0; i < N; ++i) {
        for (int k = 0; k < K; ++k) {
            double q = 0.0;   /* squared Mahalanobis distance of x_i from mu_k */
            for (int d = 0; d < D; ++d) {
                const double r = X[i * D + d] - mu[(int64_t)k * D + d];
                q += r * r * prec[(int64_t)k * D + d];
            }
            L[i * K + k] = cst[k] - 0.5 * q;
        }
    }
    free(cst);
    free(prec);
    return FVO_OK;
}

/* gamma = exp(L - lse) row by row; lse_out (N, nullable) receives lse_i. */
int fvo_posteriors(int64_t N, int K, const double *L, double *gamma, double *lse_out) {
    if (N < 0 || K <= 0 || !L || !gamma) return FVO_BADARG;
    for (int64_t i = 0; i < N; ++i) {
        const double *l = L + i * K;
        double m = -INFINITY;
        for (int k = 0; k < K; ++k) m = l[k] > m ? l[k] : m;
        double z = 0.0;
        for (int k = 0; k < K; ++k) z += exp(l[k] - m);
        const double lse = m + log(z);
        for (int k = 0; k < K; ++k) gamma[i * K + k] = exp(l[k] - lse);
        if (lse_out) lse_out[i] = lse;
    }
    return FVO_OK;
}

/* U, V (K x D) and S0 (K) from the posteriors, terms with gamma > tau. */
int fvo_moments(int64_t N, int D, int K, const double *X, const double *mu, const double *var, const double *gamma,
                double tau, double *U, double *V, double *S0) {
    if (N < 0 || D <= 0 || K <= 0 || !X || !mu || !var || !gamma || !U || !V || !S0) return FVO_BADARG;
    double *isd = (double *)malloc(sizeof(double) * D);   /* 1 / sigma of one component */
    if (!isd) return FVO_NOMEM;
    for (int k = 0; k < K; ++k) {
        const double *m = mu + (int64_t)k * D;
        double *u_k = U + (int64_t)k * D, *v_k = V + (int64_t)k * D;
        for (int d = 0; d < D; ++d) {
            isd[d] = 1.0 / sqrt(var[(int64_t)k * D + d]);
            u_k[d] = v_k[d] = 0.0;
        }
        S0[k] = 0.0;
        for (int64_t i = 0; i < N; ++i) {
            const double g = gamma[i * K + k];
            if (!(g > tau)) continue;
            S0[k] += g;
            for (int d = 0; d < D; ++d) {
                const double t = (X[i * D + d] - m[d]) * isd[d];
                u_k[d] += g * t;
                v_k[d] += g * (t * t - 1.0);
            }
        }
    }
    free(isd);
    return FVO_OK;
}

static double signed_sqrt(double a) { return a > 0 ? sqrt(a) : (a < 0 ? -sqrt(-a) : 0.0); }

/* The encoding of Sec. 4 from U, V: fv_raw = [u; v] (nullable), fv = the
 * signed square root of it, L2-normalised. */
int fvo_fisher_vector(int64_t N, int D, int K, const double *w, const double *U, const double *V, double *fv,
                      double *fv_raw) {
    if (N <= 0 || D <= 0 || K <= 0 || !w || !U || !V || !fv) return FVO_BADARG;
    const int64_t KD = (int64_t)K * D;
    for (int k = 0; k < K; ++k) {
        for (int d = 0; d < D; ++d) {
            const double u = U[(int64_t)k * D + d] / ((double)N * sqrt(w[k]));
            const double v = V[(int64_t)k * D + d] / ((double)N * sqrt(2.0 * w[k]));
            if (fv_raw) {
                fv_raw[(int64_t)k * D + d] = u;
                fv_raw[KD + (int64_t)k * D + d] = v;
            }
            fv[(int64_t)k * D + d] = signed_sqrt(u);
            fv[KD + (int64_t)k * D + d] = signed_sqrt(v);
        }
    }
    double nrm2 = 0.0;
    for (int64_t j = 0; j < 2 * KD; ++j) nrm2 += fv[j] * fv[j];
    if (nrm2 > 0.0) {
        const double nrm = sqrt(nrm2);
        for (int64_t j = 0; j < 2 * KD; ++j) fv[j] /= nrm;
    }
    return FVO_OK;
}

/* Whole encoder: descriptors and GMM in, normalised Fisher vector out.
 * Optional outputs (nullable): fv_raw (2KD), gamma (N x K), U, V (K x D),
 * S0 (K). N == 0 gives FVO_EMPTY and a zero vector. */
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

    double *L = (double *)malloc(sizeof(double) * (size_t)(N * K));
    double *gam = gamma_out ? gamma_out : (double *)malloc(sizeof(double) * (size_t)(N * K));
    double *U = (double *)malloc(sizeof(double) * KD);
    double *V = (double *)malloc(sizeof(double) * KD);
    double *S0 = (double *)malloc(sizeof(double) * K);
    int rc = FVO_NOMEM;
    if (L && gam && U && V && S0) {
        rc = fvo_log_likelihoods(N, D, K, X, w, mu, var, L);
        if (rc == FVO_OK) rc = fvo_posteriors(N, K, L, gam, NULL);
        if (rc == FVO_OK) rc = fvo_moments(N, D, K, X, mu, var, gam, tau, U, V, S0);
        if (rc == FVO_OK) rc = fvo_fisher_vector(N, D, K, w, U, V, fv, fv_raw);
        if (rc == FVO_OK) {
            if (U_out) memcpy(U_out, U, sizeof(double) * KD);
            if (V_out) memcpy(V_out, V, sizeof(double) * KD);
            if (S0_out) memcpy(S0_out, S0, sizeof(double) * K);
        }
    }
    free(L);
    if (gam != gamma_out) free(gam);
    free(U);
    free(V);
    free(S0);
    return rc;
}

/* One expectation-maximisation step for the diagonal GMM (the model the
 * paper's encoder assumes trained beforehand, Sec. 3.1), from the
 * definitions: with the posteriors gamma of the input model,
 *   N_k        = sum_i gamma_ik + 10 eps      (eps = 2^-52, keeps an empty
 *                                              component's divisions finite)
 *   w'_k       = N_k / N
 *   mu'_kd     = sum_i gamma_ik x_id / N_k
 *   sigma2'_kd = sum_i gamma_ik (x_id - mu'_kd)^2 / N_k + reg
 * and the mean log-likelihood of the descriptors under the INPUT model,
 *   mean_loglik = 1/N sum_i log sum_k w_k N(x_i; mu_k, sigma2_k).
 * Outputs: w_out (K), mu_out, var_out (K x D), mean_loglik (nullable). */
int fvo_em_step(int64_t N, int D, int K, const double *X, const double *w, const double *mu, const double *var,
                double reg, double *w_out, double *mu_out, double *var_out, double *mean_loglik) {
    if (N <= 0 || D <= 0 || K <= 0 || !X || !w || !mu || !var || !w_out || !mu_out || !var_out) return FVO_BADARG;
    double *L = (double *)malloc(sizeof(double) * (size_t)(N * K));
    double *gam = (double *)malloc(sizeof(double) * (size_t)(N * K));
    double *lse = (double *)malloc(sizeof(double) * (size_t)N);
    if (!L || !gam || !lse) {
        free(L);
        free(gam);
        free(lse);
        return FVO_NOMEM;
    }
    int rc = fvo_log_likelihoods(N, D, K, X, w, mu, var, L);
    if (rc == FVO_OK) rc = fvo_posteriors(N, K, L, gam, lse);
    if (rc == FVO_OK) {
        const double two_pi_term = 0.5 * D * log(2.0 * 3.14159265358979323846);
        if (mean_loglik) {
            double s = 0.0;
            for (int64_t i = 0; i < N; ++i) s += lse[i] - two_pi_term;
            *mean_loglik = s / (double)N;
        }
        for (int k = 0; k < K; ++k) {
            double nk = 10.0 * 2.220446049250313e-16;
            for (int64_t i = 0; i < N; ++i) nk += gam[i * K + k];
            w_out[k] = nk / (double)N;
            for (int d = 0; d < D; ++d) {
                double s1 = 0.0;
                for (int64_t i = 0; i < N; ++i) s1 += gam[i * K + k] * X[i * D + d];
                const double m = s1 / nk;
                double s2 = 0.0;
                for (int64_t i = 0; i < N; ++i) {
                    const double r = X[i * D + d] - m;
                    s2 += gam[i * K + k] * r * r;
                }
                mu_out[(int64_t)k * D + d] = m;
                var_out[(int64_t)k * D + d] = s2 / nk + reg;
            }
        }
    }
    free(L);
    free(gam);
    free(lse);
    return rc;
}

/* The descriptor step of Sec. 3.1 before the encoding: a 128-dimensional
 * descriptor x is reduced to m dimensions by PCA and the normalised X and Y
 * position of the descriptor is appended, D = m + 2:
 *   y_i = [ P (x_i - mean) ; xy_i ]
 * P is the m x Din matrix of principal directions (rows), mean the Din-vector
 * the PCA was centred on, xy_i the two normalised coordinates (omitted when
 * xy is NULL, D = m). Y is N x D row-major. */
int fvo_pca_project(int64_t N, int Din, int m, const double *X, const double *mean, const double *P, const double *xy,
                    double *Y) {
    if (N < 0 || Din <= 0 || m <= 0 || !X || !P || !Y) return FVO_BADARG;
    const int D = m + (xy ? 2 : 0);
    for (int64_t i = 0; i < N; ++i) {
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int k = 0; k < Din; ++k) s += P[(int64_t)j * Din + k] * (X[i * Din + k] - (mean ? mean[k] : 0.0));
            Y[i * D + j] = s;
        }
        if (xy) {
            Y[i * D + m] = xy[2 * i];
            Y[i * D + m + 1] = xy[2 * i + 1];
        }
    }
    return FVO_OK;
}
