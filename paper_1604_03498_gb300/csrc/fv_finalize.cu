// Finalise: reduction of the per-range statistics copies (the paper's second
// Phase-2 kernel, Algorithm 3: "each block processes U and V for one GMM
// component" and adds the per-block copies) followed by the encoding scheme of
// Sec. 4: u = U/(N sqrt(w)), v = V/(N sqrt(2w)), signed square root, L2.
//
// Kernel A: one block per (component, frame). Sums that frame's slots in slot
// order (fixed, so a frame's vector does not depend on what else ran with it),
// forms u and v in FP64, writes sign(z) sqrt|z| and the component's sum of
// squares. Kernel B: one block per frame, sums the K squares in a fixed tree
// order and scales the frame's vector by 1/||z||.
//
// FP32 form slots hold centred sums [A = sum g (x-mu) (D), B = sum g (x-mu)^2
// (D), S0]: u = A/sigma alpha/N, v = (B/sigma^2 - S0) beta/N.
// BF16 form slots hold raw moments [S1 (D), S2hi (D), S2lo (D), S0] and the
// centring happens here in FP64:
//   u = (S1 - mu S0) / sigma * alpha / N
//   v = ((S2 - 2 mu S1 + mu^2 S0) / sigma^2 - S0) * beta / N.
#include "fv_internal.h"

namespace fv {

namespace {

constexpr int FA_THREADS = 128;
constexpr int FB_THREADS = 256;

__device__ __forceinline__ double ssqrt(double v) { return v > 0.0 ? sqrt(v) : (v < 0.0 ? -sqrt(-v) : 0.0); }

template <bool RAW>
__global__ void __launch_bounds__(FA_THREADS)
finalize_a_kernel(const float *__restrict__ part, int P, int Kp, int K, int D, const FrameInfo *__restrict__ frames,
                  GmmDev g, double *__restrict__ sq, float *__restrict__ out) {
    extern __shared__ double sacc[];   // [P]
    __shared__ double red[FA_THREADS];
    const int k = blockIdx.x, f = blockIdx.y;
    const FrameInfo fr = frames[f];
    const size_t KD = (size_t)K * D;
    float *o = out + (size_t)f * 2 * KD;
    if (fr.n == 0) {
        for (int d = threadIdx.x; d < D; d += FA_THREADS) {
            o[(size_t)k * D + d] = 0.f;
            o[KD + (size_t)k * D + d] = 0.f;
        }
        if (threadIdx.x == 0) sq[(size_t)f * K + k] = 0.0;
        return;
    }
    const size_t sstride = (size_t)Kp * P;
    for (int j = threadIdx.x; j < P; j += FA_THREADS) {
        // four interleaved partial sums keep four loads in flight; the
        // combination order is fixed
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        const float *p = part + ((size_t)fr.slot0 * Kp + k) * P + j;
        int s = 0;
        for (; s + 4 <= fr.nslots; s += 4) {
            a0 += (double)p[(size_t)s * sstride];
            a1 += (double)p[(size_t)(s + 1) * sstride];
            a2 += (double)p[(size_t)(s + 2) * sstride];
            a3 += (double)p[(size_t)(s + 3) * sstride];
        }
        for (; s < fr.nslots; ++s) a0 += (double)p[(size_t)s * sstride];
        sacc[j] = (a0 + a1) + (a2 + a3);
    }
    __syncthreads();
    const double S0 = sacc[P - 1];
    const double inv_n = 1.0 / (double)fr.n;
    const double al = g.alpha[k] * inv_n, be = g.beta[k] * inv_n;
    double acc = 0.0;
    for (int d = threadIdx.x; d < D; d += FA_THREADS) {
        double u, v;
        if (RAW) {
            const double m = g.mu64[(size_t)k * D + d];
            const double S1 = sacc[d];
            const double S2 = sacc[D + d] + sacc[2 * D + d];
            u = (S1 - m * S0) * g.isd64[(size_t)k * D + d] * al;
            v = ((S2 - 2.0 * m * S1 + m * m * S0) * g.prec64[(size_t)k * D + d] - S0) * be;
        } else {
            u = sacc[d] * g.isd64[(size_t)k * D + d] * al;
            v = (sacc[D + d] * g.prec64[(size_t)k * D + d] - S0) * be;
        }
        const double zu = ssqrt(u), zv = ssqrt(v);
        o[(size_t)k * D + d] = (float)zu;
        o[KD + (size_t)k * D + d] = (float)zv;
        acc += zu * zu + zv * zv;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = FA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) sq[(size_t)f * K + k] = red[0];
}

__global__ void __launch_bounds__(FB_THREADS)
finalize_b_kernel(int K, int D, const double *__restrict__ sq, float *__restrict__ out,
                  const uint32_t *__restrict__ err) {
    __shared__ double red[FB_THREADS];
    const int f = blockIdx.x;
    double a = 0.0;
    for (int k = threadIdx.x; k < K; k += FB_THREADS) a += sq[(size_t)f * K + k];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = FB_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const double tot = red[0];
    const size_t n = (size_t)2 * K * D;
    float *o = out + (size_t)f * n;
    if (err && *err) {   // an earlier kernel of this call gave up: poison the output
        for (size_t j = threadIdx.x; j < n; j += FB_THREADS) o[j] = __int_as_float(0x7fc00000);
        return;
    }
    if (!(tot > 0.0)) return;   // all-zero vector stays zero
    const float inv = (float)(1.0 / sqrt(tot));
    for (size_t j = threadIdx.x; j < n; j += FB_THREADS) o[j] *= inv;
}

}  // namespace

cudaError_t launch_finalize(const fv_gmm *g, const float *part, int P, bool raw_moments, const FrameInfo *frames,
                            int B, double *sq, float *out, cudaStream_t st, const uint32_t *err) {
    if (B <= 0) return cudaSuccess;
    dim3 grid_a((unsigned)g->K, (unsigned)B);
    const size_t smem = sizeof(double) * P;
    if (raw_moments) {
        cudaError_t e = cudaFuncSetAttribute(finalize_a_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("finalize_a", st);
        finalize_a_kernel<true><<<grid_a, FA_THREADS, smem, st>>>(part, P, g->Kp, g->K, g->D, frames, g->dev, sq, out);
    }
    } else {
        cudaError_t e = cudaFuncSetAttribute(finalize_a_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("finalize_a", st);
        finalize_a_kernel<false><<<grid_a, FA_THREADS, smem, st>>>(part, P, g->Kp, g->K, g->D, frames, g->dev, sq, out);
    }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    {
        KernelTimer kt_("finalize_b", st);
        finalize_b_kernel<<<(unsigned)B, FB_THREADS, 0, st>>>(g->K, g->D, sq, out, err);
    }
    return cudaGetLastError();
}

}  // namespace fv
