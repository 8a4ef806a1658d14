// GMM preparation (Algorithm 1, "compute sqrt(sigma^-1)"; Sec. 3.2 runs it as
// "a simple GPU kernel" once per model) and the GMM handle's life cycle.
//
// Everything here is computed in FP64 on the device from the caller's FP32
// parameters, once per GMM:
//   w'_k      = w_k / sum_j w_j                    (renormalised priors)
//   1/sigma   = 1/sqrt(sigma^2),  -mu/sigma,  1/sigma^2
//   c'_k      = log w'_k - 1/2 sum_d log sigma^2_kd        (FP32 form)
//   c_k       = c'_k - 1/2 sum_d mu_kd^2 / sigma^2_kd     (BF16 form: the
//               constant term of the expanded log-likelihood)
//   alpha_k   = 1/sqrt(w'_k),  beta_k = 1/sqrt(2 w'_k)   (improved-FV scalings)
//   BF16 GEMM operands Q = mu/sigma^2 and R = -1/(2 sigma^2), each split into
//   a bfloat16 high part and a bfloat16 low part (hi + lo carries ~16 bits).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "fv_internal.h"

namespace fv {

namespace {

__device__ double block_sum(double v, double *red) {
    // fixed-order tree over the block (blockDim.x is a power of two <= 1024)
    red[threadIdx.x] = v;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ float bf16_value(uint16_t b) {
    return __uint_as_float(((uint32_t)b) << 16);
}

// One block per (padded) component; threads stride over dimensions.
__global__ void prep_kernel(int K, int D, int Kp, int Dp, int D16, const float *__restrict__ w,
                            const float *__restrict__ mu, const float *__restrict__ var, GmmDev g) {
    __shared__ double red[256];
    const int k = blockIdx.x;
    // renormalising sum of priors (every block recomputes it; K <= 512)
    double ws = 0.0;
    for (int j = threadIdx.x; j < K; j += blockDim.x) ws += (double)w[j];
    ws = block_sum(ws, red);

    if (k >= K) {  // padded component: never wins the softmax, contributes nothing
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            g.s_t[(size_t)d * Kp + k] = 0.f;
            g.nms_t[(size_t)d * Kp + k] = 0.f;
            g.mu_t[(size_t)d * Kp + k] = 0.f;
            g.prec_t[(size_t)d * Kp + k] = 0.f;
        }
        for (int d = threadIdx.x; d < Dp; d += blockDim.x) {
            g.s_kd[(size_t)k * Dp + d] = 0.f;
            g.mu_kd[(size_t)k * Dp + d] = 0.f;
        }
        if (g.bimg)
            for (int d = threadIdx.x; d < D16; d += blockDim.x)
                for (int t = 0; t < 4; ++t) g.bimg[((size_t)t * Kp + k) * D16 + d] = 0;
        if (threadIdx.x == 0) {
            g.cst[k] = -INFINITY;
            g.c64[k] = -INFINITY;
            g.c64[Kp + k] = -INFINITY;
            if (g.cfull) g.cfull[k] = -INFINITY;
            if (g.cl2) g.cl2[k] = -INFINITY;
            g.alpha[k] = 0.f;
            g.beta[k] = 0.f;
        }
        return;
    }

    double slog = 0.0, smq = 0.0;
    for (int d = threadIdx.x; d < Dp || d < D16; d += blockDim.x) {
        if (d < D) {
            const double v = (double)var[(size_t)k * D + d];
            const double m = (double)mu[(size_t)k * D + d];
            const double isd = 1.0 / sqrt(v);
            const double p = 1.0 / v;
            slog += log(v);
            smq += m * m * p;
            g.s_t[(size_t)d * Kp + k] = (float)isd;
            g.nms_t[(size_t)d * Kp + k] = (float)(-m * isd);
            g.s_kd[(size_t)k * Dp + d] = (float)isd;
            g.mu_kd[(size_t)k * Dp + d] = (float)m;
            g.mu_t[(size_t)d * Kp + k] = (float)m;
            g.prec_t[(size_t)d * Kp + k] = (float)p;
            if (g.bimg) {
                const double q = m * p, r = -0.5 * p;
                const uint16_t qh = bf16_bits((float)q), rh = bf16_bits((float)r);
                const uint16_t ql = bf16_bits((float)(q - (double)bf16_value(qh)));
                const uint16_t rl = bf16_bits((float)(r - (double)bf16_value(rh)));
                g.bimg[((size_t)0 * Kp + k) * D16 + d] = qh;
                g.bimg[((size_t)1 * Kp + k) * D16 + d] = ql;
                g.bimg[((size_t)2 * Kp + k) * D16 + d] = rh;
                g.bimg[((size_t)3 * Kp + k) * D16 + d] = rl;
            }
        } else {
            if (d < Dp) {
                g.s_kd[(size_t)k * Dp + d] = 0.f;
                g.mu_kd[(size_t)k * Dp + d] = 0.f;
            }
            if (g.bimg && d < D16)
                for (int t = 0; t < 4; ++t) g.bimg[((size_t)t * Kp + k) * D16 + d] = 0;
        }
    }
    slog = block_sum(slog, red);
    smq = block_sum(smq, red);
    if (threadIdx.x == 0) {
        const double wk = (double)w[k] / ws;
        const double c1 = log(wk) - 0.5 * slog;
        g.cst[k] = (float)c1;
        g.c64[k] = c1;
        g.c64[Kp + k] = c1 - 0.5 * smq;
        if (g.cfull) g.cfull[k] = (float)(c1 - 0.5 * smq);
        if (g.cl2) g.cl2[k] = (float)((c1 - 0.5 * smq) * 1.4426950408889634);
        g.alpha[k] = (float)(1.0 / sqrt(wk));
        g.beta[k] = (float)(1.0 / sqrt(2.0 * wk));
    }
}

}  // namespace

cudaError_t launch_prep(const fv_gmm *g, const float *w, const float *mu, const float *var, cudaStream_t st) {
    const int D16 = round_up(g->D, 16);
    {
        KernelTimer kt_("prep", st);
        prep_kernel<<<g->Kp, 256, 0, st>>>(g->K, g->D, g->Kp, g->Dp, D16, w, mu, var, g->dev);
    }
    return cudaGetLastError();
}

}  // namespace fv

using namespace fv;

extern "C" int fv_limits(fv_precision precision, int *max_K, int *max_D) {
    if (precision == FV_PREC_FP32) {
        if (max_K) *max_K = kMaxK_F32;
        if (max_D) *max_D = kMaxD_F32;
        return FV_OK;
    }
    if (is_bf16(precision)) {
        if (max_K) *max_K = kMaxK_BF16;
        if (max_D) *max_D = precision == FV_PREC_BF16X2 ? kMaxD_BF16X2 : kMaxD_BF16;
        return FV_OK;
    }
    return fail(FV_ERR_INVALID, "fv_limits: unknown precision");
}

extern "C" int fv_gmm_load(const fv_gmm_desc *desc, fv_precision precision, fv_gmm **out) {
    if (!out) return fail(FV_ERR_INVALID, "fv_gmm_load: out is NULL");
    *out = nullptr;
    if (!desc || !desc->weights || !desc->means || !desc->variances)
        return fail(FV_ERR_INVALID, "fv_gmm_load: NULL descriptor or parameter array");
    const int K = desc->K, D = desc->D;
    if (K <= 0 || D <= 0) return fail(FV_ERR_INVALID, "fv_gmm_load: K and D must be positive");
    if (precision != FV_PREC_FP32 && !is_bf16(precision))
        return fail(FV_ERR_INVALID, "fv_gmm_load: unknown precision");
    int mK = 0, mD = 0;
    fv_limits(precision, &mK, &mD);
    if (K > mK || D > mD)
        return fail(FV_ERR_UNSUPPORTED, "fv_gmm_load: K=" + std::to_string(K) + " D=" + std::to_string(D) +
                                            " beyond limits K<=" + std::to_string(mK) + " D<=" + std::to_string(mD));
    double ws = 0.0;
    for (int k = 0; k < K; ++k) {
        const float v = desc->weights[k];
        if (!std::isfinite(v) || !(v > 0.f)) return fail(FV_ERR_INVALID, "fv_gmm_load: weights must be finite and > 0");
        ws += v;
    }
    if (std::fabs(ws - 1.0) > 1e-5) return fail(FV_ERR_INVALID, "fv_gmm_load: weights must sum to 1 (|sum-1| <= 1e-5)");
    for (size_t i = 0; i < (size_t)K * D; ++i) {
        if (!std::isfinite(desc->means[i])) return fail(FV_ERR_INVALID, "fv_gmm_load: means must be finite");
        const float v = desc->variances[i];
        if (!std::isfinite(v) || !(v > 0.f)) return fail(FV_ERR_INVALID, "fv_gmm_load: variances must be finite and > 0");
    }

    fv_gmm *g = new fv_gmm();
    g->K = K;
    g->D = D;
    g->prec = precision;
    g->Kp = is_bf16(precision) ? round_up(K, 128) : round_up(K, 64);
    g->Dp = is_bf16(precision) ? round_up(D, 16) : round_up(D, 8);
    cudaGetDevice(&g->device);
    const int Kp = g->Kp, Dp = g->Dp, D16 = round_up(D, 16);

    // carve every array out of one allocation (256-byte aligned pieces)
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += (bytes + 255) / 256 * 256; return o; };
    const size_t o_s_t = take(sizeof(float) * D * Kp), o_nms_t = take(sizeof(float) * D * Kp);
    const size_t o_cst = take(sizeof(float) * Kp), o_c64 = take(sizeof(double) * 2 * Kp);
    const size_t o_s_kd = take(sizeof(float) * Kp * Dp), o_mu_kd = take(sizeof(float) * Kp * Dp);
    const size_t o_alpha = take(sizeof(float) * Kp), o_beta = take(sizeof(float) * Kp);
    const size_t o_mu = take(sizeof(float) * D * Kp), o_prec = take(sizeof(float) * D * Kp);
    size_t o_bimg = 0, o_cfull = 0, o_cl2 = 0;
    if (is_bf16(precision)) {
        o_bimg = take(sizeof(uint16_t) * 4 * Kp * D16);
        o_cfull = take(sizeof(float) * Kp);
        o_cl2 = take(sizeof(float) * Kp);
    }
    const size_t o_in = take(sizeof(float) * (K + 2 * (size_t)K * D));
    char *base = nullptr;
    cudaError_t e = cudaMalloc(&base, off);
    if (e != cudaSuccess) {
        delete g;
        return fail(FV_ERR_OOM, std::string("fv_gmm_load: cudaMalloc: ") + cudaGetErrorString(e));
    }
    g->block = base;
    g->block_bytes = off;
    GmmDev &d = g->dev;
    d.s_t = (float *)(base + o_s_t);
    d.nms_t = (float *)(base + o_nms_t);
    d.cst = (float *)(base + o_cst);
    d.c64 = (double *)(base + o_c64);
    d.s_kd = (float *)(base + o_s_kd);
    d.mu_kd = (float *)(base + o_mu_kd);
    d.alpha = (float *)(base + o_alpha);
    d.beta = (float *)(base + o_beta);
    d.mu_t = (float *)(base + o_mu);
    d.prec_t = (float *)(base + o_prec);
    d.bimg = is_bf16(precision) ? (uint16_t *)(base + o_bimg) : nullptr;
    d.cfull = is_bf16(precision) ? (float *)(base + o_cfull) : nullptr;
    d.cl2 = is_bf16(precision) ? (float *)(base + o_cl2) : nullptr;
    float *in = (float *)(base + o_in);
    d.params = in;

    cudaStream_t st;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
        cudaFree(base);
        delete g;
        return cuda_fail(e, "fv_gmm_load: cudaStreamCreate");
    }
    std::vector<float> host(K + 2 * (size_t)K * D);
    std::memcpy(host.data(), desc->weights, sizeof(float) * K);
    std::memcpy(host.data() + K, desc->means, sizeof(float) * K * D);
    std::memcpy(host.data() + K + (size_t)K * D, desc->variances, sizeof(float) * K * D);
    e = cudaMemcpyAsync(in, host.data(), sizeof(float) * host.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_prep(g, in, in + K, in + K + (size_t)K * D, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess) {
        cudaFree(base);
        delete g;
        return cuda_fail(e, "fv_gmm_load: preparation kernel");
    }
    *out = g;
    return FV_OK;
}

extern "C" void fv_gmm_free(fv_gmm *g) {
    if (!g) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) cudaSetDevice(g->device);
    cudaFree(g->block);
    if (cur != g->device) cudaSetDevice(cur);
    delete g;
}

extern "C" int fv_gmm_constants(const fv_gmm *g, double *c_direct, double *c_expanded) {
    if (!g) return fail(FV_ERR_INVALID, "fv_gmm_constants: NULL handle");
    if (c_direct) {
        const cudaError_t e = cudaMemcpy(c_direct, g->dev.c64, sizeof(double) * g->K, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "fv_gmm_constants: copy");
    }
    if (c_expanded) {
        const cudaError_t e =
            cudaMemcpy(c_expanded, g->dev.c64 + g->Kp, sizeof(double) * g->K, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "fv_gmm_constants: copy");
    }
    return FV_OK;
}

extern "C" int fv_gmm_info(const fv_gmm *g, int *K, int *D, int *precision) {
    if (!g) return fail(FV_ERR_INVALID, "fv_gmm_info: NULL handle");
    if (K) *K = g->K;
    if (D) *D = g->D;
    if (precision) *precision = g->prec;
    return FV_OK;
}
