// GMM training by expectation-maximisation on the GPU, built on the plain
// FP32 form's kernels. The paper encodes with a GMM "trained beforehand"
// (Sec. 3.1); EM's E-step is exactly the first part of the encoder
// (posteriors, Algorithm 1's first loop, and the centred statistics of its
// second loop), so one EM step is
//
//   E-step: f32 posteriors (with each row's log-sum-exp) -> f32 statistics
//           A_kd = sum_i g_ik (x_id - mu_kd), B_kd = sum_i g_ik (x_id - mu_kd)^2,
//           S0_k = sum_i g_ik per row range -> slot reduction (fixed order);
//   M-step: one block per component, in FP64 from the FP32 sums,
//           N_k = S0_k + 10 eps (eps = 2^-52: an empty component's divisions
//                                stay finite),
//           w'_k = N_k / N,   mu'_kd = (mu_kd S0_k + A_kd) / N_k,
//           with delta = mu' - mu the statistics re-centred on the new mean:
//           var'_kd = (B_kd - 2 delta A_kd + delta^2 S0_k) / N_k + reg;
//   log-likelihood of the descriptors under the input model:
//           1/N sum_i lse_i - (D/2) log(2 pi), summed in FP64 in a fixed order.
//
// The centred sums keep the new variance free of the cancellation of
// E[x^2] - E[x]^2. fv_gmm_fit repeats the step on the device, re-running the
// GMM preparation kernel on the new parameters between steps.
#include <cmath>
#include <string>
#include <vector>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr double kEmEps = 10.0 * 2.220446049250313e-16;

// grid (K), block 128: the M-step of component k from the reduced slot
// part[0][j][Kp] (j: A (D), B (D), S0).
__global__ void __launch_bounds__(128)
em_mstep_kernel(const float *__restrict__ part, int Kp, int Dp, int D, int64_t N, const float *__restrict__ mu_kd,
                double reg, float *__restrict__ w_out, float *__restrict__ mu_out, float *__restrict__ var_out) {
    const int k = blockIdx.x;
    const double S0 = (double)part[(size_t)(2 * D) * Kp + k];
    const double nk = S0 + kEmEps;
    if (threadIdx.x == 0) w_out[k] = (float)(nk / (double)N);
    for (int d = threadIdx.x; d < D; d += blockDim.x) {
        const double A = (double)part[(size_t)d * Kp + k];
        const double B = (double)part[(size_t)(D + d) * Kp + k];
        const double m = (double)mu_kd[(size_t)k * Dp + d];
        const double m2 = (m * S0 + A) / nk;
        const double dl = m2 - m;
        mu_out[(size_t)k * D + d] = (float)m2;
        var_out[(size_t)k * D + d] = (float)((B - 2.0 * dl * A + dl * dl * S0) / nk + reg);
    }
}

// One block of 1024 threads: fixed-order FP64 mean of the rows' log-sum-exp
// minus the common (D/2) log(2 pi).
__global__ void __launch_bounds__(1024)
em_loglik_kernel(const float *__restrict__ lse, int64_t N, int D, double *__restrict__ out) {
    __shared__ double red[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += 1024) s += (double)lse[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int h = 512; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0] / (double)N - 0.5 * D * log(2.0 * 3.14159265358979323846);
}

struct EmScratch {
    char *base = nullptr;
    float *gam = nullptr, *lse = nullptr, *part = nullptr;
    FrameInfo *frame = nullptr;
    StatUnit *units = nullptr;
    double *ll = nullptr;
    int nunits = 0, P = 0;
};

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Statistics ranges of about three blocks per SM (as the FP32 encoder), the
// work list uploaded, scratch taken stream-ordered from the pool.
int em_scratch(const fv_gmm *g, int64_t N, cudaStream_t st, EmScratch &s) {
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    const int Kp = g->Kp, D = g->D;
    s.P = 2 * D + 1;
    const int64_t per_range = (int64_t)(Kp / 64) * ((D + 63) / 64);
    int64_t rpr = (N * per_range + 3LL * sms - 1) / (3LL * sms);
    rpr = std::min<int64_t>(std::max<int64_t>(round_up64(rpr, 32), 64), 16384);
    s.nunits = (int)((N + rpr - 1) / rpr);
    std::vector<StatUnit> units(s.nunits);
    for (int u = 0; u < s.nunits; ++u) {
        units[u].row0 = (int64_t)u * rpr;
        units[u].nrows = (int32_t)std::min<int64_t>(rpr, N - (int64_t)u * rpr);
        units[u].slot = u;
    }
    FrameInfo fr{0, N, 0, s.nunits};
    const size_t b_gam = al256(f32_gamma_bytes(N, Kp)), b_lse = al256(sizeof(float) * N);
    const size_t b_part = al256(sizeof(float) * (size_t)s.nunits * Kp * s.P);
    const size_t b_fr = al256(sizeof(FrameInfo)), b_un = al256(sizeof(StatUnit) * s.nunits), b_ll = al256(8);
    cudaError_t e = cudaMallocAsync((void **)&s.base, b_gam + b_lse + b_part + b_fr + b_un + b_ll, st);
    if (e != cudaSuccess) return cuda_fail(e, "EM: cudaMallocAsync(scratch)");
    char *p = s.base;
    s.gam = (float *)p;
    p += b_gam;
    s.lse = (float *)p;
    p += b_lse;
    s.part = (float *)p;
    p += b_part;
    s.frame = (FrameInfo *)p;
    p += b_fr;
    s.units = (StatUnit *)p;
    p += b_un;
    s.ll = (double *)p;
    // pageable sources: the copies are staged before cudaMemcpyAsync returns
    if ((e = cudaMemcpyAsync(s.frame, &fr, sizeof(fr), cudaMemcpyHostToDevice, st)) != cudaSuccess ||
        (e = cudaMemcpyAsync(s.units, units.data(), sizeof(StatUnit) * s.nunits, cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_fail(e, "EM: work-list upload");
    return FV_OK;
}

// E-step + M-step into device arrays w, mu, var; log-likelihood into s.ll.
int em_step_device(const fv_gmm *g, const float *Xd, int64_t N, double reg, float *w, float *mu, float *var,
                   EmScratch &s, cudaStream_t st) {
    cudaError_t e;
    if ((e = launch_f32_posteriors(g, Xd, N, s.gam, st, s.lse)) != cudaSuccess)
        return cuda_fail(e, "EM: posteriors launch");
    if ((e = launch_f32_stats(g, Xd, s.gam, N, s.units, s.nunits, s.part, s.P, st)) != cudaSuccess)
        return cuda_fail(e, "EM: statistics launch");
    if ((e = launch_slot_reduce(g, s.part, s.P, s.frame, 1, s.nunits, st)) != cudaSuccess)
        return cuda_fail(e, "EM: slot reduction launch");
    {
        KernelTimer kt_("em_mstep", st);
        em_mstep_kernel<<<g->K, 128, 0, st>>>(s.part, g->Kp, g->Dp, g->D, N, g->dev.mu_kd, reg, w, mu, var);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "EM: M-step launch");
    {
        KernelTimer kt_("em_loglik", st);
        em_loglik_kernel<<<1, 1024, 0, st>>>(s.lse, N, g->D, s.ll);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "EM: log-likelihood launch");
    return FV_OK;
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Descriptors on the device: X itself, or a stream-ordered copy of host X.
int stage_x(const float *X, int64_t N, int D, int x_on_device, cudaStream_t st, const float **Xd, float **owned) {
    *owned = nullptr;
    if (x_on_device) {
        if (!dev_ptr(X)) return fail(FV_ERR_INVALID, "x_on_device=1 but X is not device memory");
        *Xd = X;
        return FV_OK;
    }
    cudaError_t e = cudaMallocAsync((void **)owned, sizeof(float) * N * D, st);
    if (e != cudaSuccess) return cuda_fail(e, "EM: cudaMallocAsync(X)");
    if ((e = cudaMemcpyAsync(*owned, X, sizeof(float) * N * D, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "EM: cudaMemcpyAsync(X)");
    *Xd = *owned;
    return FV_OK;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" int fv_gmm_em_step(const fv_gmm *gmm, const float *X, int64_t N, int x_on_device, double reg_covar,
                              float *w_out, float *mu_out, float *var_out, int out_on_device, double *mean_loglik,
                              void *cuda_stream) {
    if (!gmm || !X || !w_out || !mu_out || !var_out) return fail(FV_ERR_INVALID, "fv_gmm_em_step: NULL argument");
    if (gmm->prec != FV_PREC_FP32) return fail(FV_ERR_INVALID, "fv_gmm_em_step: needs an FV_PREC_FP32 GMM");
    if (N <= 0) return fail(FV_ERR_EMPTY, "fv_gmm_em_step: no descriptors");
    if (!(reg_covar >= 0.0) || !std::isfinite(reg_covar)) return fail(FV_ERR_INVALID, "fv_gmm_em_step: reg_covar < 0");
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != gmm->device) return fail(FV_ERR_INVALID, "fv_gmm_em_step: GMM handle belongs to another device");
    if (out_on_device && (!dev_ptr(w_out) || !dev_ptr(mu_out) || !dev_ptr(var_out)))
        return fail(FV_ERR_INVALID, "fv_gmm_em_step: out_on_device=1 but an output is not device memory");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int K = gmm->K, D = gmm->D;
    const size_t KD = (size_t)K * D;
    const float *Xd = nullptr;
    float *xown = nullptr, *pown = nullptr;
    EmScratch s;
    int rc = stage_x(X, N, D, x_on_device, st, &Xd, &xown);
    if (rc == FV_OK) rc = em_scratch(gmm, N, st, s);
    float *w = w_out, *mu = mu_out, *var = var_out;
    if (rc == FV_OK && !out_on_device) {
        cudaError_t e = cudaMallocAsync((void **)&pown, sizeof(float) * (K + 2 * KD), st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fv_gmm_em_step: cudaMallocAsync(outputs)");
        w = pown;
        mu = pown + K;
        var = pown + K + KD;
    }
    if (rc == FV_OK) rc = em_step_device(gmm, Xd, N, reg_covar, w, mu, var, s, st);
    if (rc == FV_OK && !out_on_device) {
        cudaError_t e = cudaMemcpyAsync(w_out, w, sizeof(float) * K, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(mu_out, mu, sizeof(float) * KD, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(var_out, var, sizeof(float) * KD, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fv_gmm_em_step: copy of the parameters");
    }
    if (rc == FV_OK && mean_loglik) {
        cudaError_t e = cudaMemcpyAsync(mean_loglik, s.ll, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fv_gmm_em_step: copy of the log-likelihood");
    }
    if (s.base) cudaFreeAsync(s.base, st);
    if (pown) cudaFreeAsync(pown, st);
    if (xown) cudaFreeAsync(xown, st);
    if (rc == FV_OK && (mean_loglik || !out_on_device)) {
        cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fv_gmm_em_step: cudaStreamSynchronize");
    }
    return rc;
}

extern "C" int fv_gmm_fit(const fv_gmm_desc *init, const float *X, int64_t N, int x_on_device, int max_iter,
                          double tol, double reg_covar, float *w_out, float *mu_out, float *var_out, int *n_iter,
                          double *mean_loglik, void *cuda_stream) {
    if (!init || !X || !w_out || !mu_out || !var_out) return fail(FV_ERR_INVALID, "fv_gmm_fit: NULL argument");
    if (max_iter < 1) return fail(FV_ERR_INVALID, "fv_gmm_fit: max_iter must be >= 1");
    if (N <= 0) return fail(FV_ERR_EMPTY, "fv_gmm_fit: no descriptors");
    if (!(reg_covar >= 0.0) || !std::isfinite(reg_covar) || !(tol >= 0.0))
        return fail(FV_ERR_INVALID, "fv_gmm_fit: reg_covar and tol must be >= 0");
    fv_gmm *g = nullptr;
    int rc = fv_gmm_load(init, FV_PREC_FP32, &g);
    if (rc != FV_OK) return rc;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const int K = g->K, D = g->D;
    const size_t KD = (size_t)K * D;
    const float *Xd = nullptr;
    float *xown = nullptr;
    EmScratch s;
    rc = stage_x(X, N, D, x_on_device, st, &Xd, &xown);
    if (rc == FV_OK) rc = em_scratch(g, N, st, s);
    double prev = -INFINITY, ll = 0.0;
    int it = 0;
    float *par = g->dev.params;   // [K] w, [K][D] mu, [K][D] var: rewritten in place each step
    while (rc == FV_OK && it < max_iter) {
        rc = em_step_device(g, Xd, N, reg_covar, par, par + K, par + K + KD, s, st);
        if (rc != FV_OK) break;
        cudaError_t e = launch_prep(g, par, par + K, par + K + KD, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&ll, s.ll, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "fv_gmm_fit: step");
            break;
        }
        ++it;
        if (!std::isfinite(ll)) {
            rc = fail(FV_ERR_INVALID, "fv_gmm_fit: the log-likelihood is not finite (a variance collapsed; "
                                      "raise reg_covar)");
            break;
        }
        if (std::fabs(ll - prev) < tol) break;
        prev = ll;
    }
    if (rc == FV_OK) {
        cudaError_t e = cudaMemcpyAsync(w_out, par, sizeof(float) * K, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(mu_out, par + K, sizeof(float) * KD, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(var_out, par + K + KD, sizeof(float) * KD, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = cuda_fail(e, "fv_gmm_fit: copy of the parameters");
    }
    if (s.base) cudaFreeAsync(s.base, st);
    if (xown) cudaFreeAsync(xown, st);
    cudaStreamSynchronize(st);
    fv_gmm_free(g);
    if (n_iter) *n_iter = it;
    if (mean_loglik) *mean_loglik = ll;
    return rc;
}
