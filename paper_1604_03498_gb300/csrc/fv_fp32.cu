// Plain FP32 form of the encoder: SIMT kernels in the centred (direct) form.
//
// Posteriors (Algorithm 1 first loop; the paper's Phase 1, Algorithm 2):
//   l_ik = c'_k - 1/2 sum_d t_ikd^2,  t_ikd = x_id/sigma_kd - mu_kd/sigma_kd
//   gamma_ik = exp(l_ik - max_k l_ik) / sum_k exp(l_ik - max_k l_ik)
// computed for a 64-row block against every component with register tiles of
// 8 rows x CPL components per thread (t is one FMA, t^2 accumulation another),
// the row block's log-likelihoods kept in shared memory for the softmax.
//
// Statistics (Algorithm 1 second loop; the paper's Phase 2, Algorithm 3 with
// one private copy of U, V per block): each block owns one row range and one
// 64-component chunk and accumulates, per (k, d) held in registers,
//   A_kd += gamma_ik (x_id - mu_kd),  B_kd += gamma_ik (x_id - mu_kd)^2,
//   S0_k += gamma_ik
// and the finalise kernel forms U = A/sigma and V = B/sigma^2 - S0 in FP64.
// The residual x - mu carries a rounding error relative to itself; the
// posteriors' single-FMA form x/sigma - mu/sigma errs by ~eps |mu/sigma|, which
// is harmless inside a softmax but would be amplified near zero by the signed
// square root when a component's variance is tiny. Every block writes its own
// statistics slot; the finalise kernel reduces the slots in a fixed order, so
// no atomics touch the result.
#include "fv_internal.h"

namespace fv {

namespace {

constexpr int P_BM = 64;   // rows per posterior block
constexpr int P_DS = 32;   // dimension slice staged in shared memory
constexpr int P_THREADS = 256;

// Dynamic shared memory layout of the posteriors kernel:
//   sS[P_DS][KC], sN[P_DS][KC]   1/sigma and -mu/sigma of the current chunk
//   sX[P_DS][P_BM + 4]           descriptor slice, dimension-major
//   sL[P_BM][Kp]                 log-likelihoods of the row block
template <int CPL>
__global__ void __launch_bounds__(P_THREADS)
f32_posteriors_kernel(const float *__restrict__ X, int64_t rows, int D, int Kp,
                      const float *__restrict__ s_t, const float *__restrict__ nms_t,
                      const float *__restrict__ cst, float *__restrict__ gamma) {
    constexpr int KC = 32 * CPL;
    constexpr int XS = P_BM + 4;
    extern __shared__ __align__(16) float smem[];
    float *sS = smem;
    float *sN = sS + P_DS * KC;
    float *sX = sN + P_DS * KC;
    float *sL = sX + P_DS * XS;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * P_BM;

    for (int kc0 = 0; kc0 < Kp; kc0 += KC) {
        float acc[8][CPL];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < CPL; ++c) acc[r][c] = 0.f;

        for (int d0 = 0; d0 < D; d0 += P_DS) {
            __syncthreads();
            for (int i = tid; i < P_DS * KC; i += P_THREADS) {
                const int dd = i / KC, kk = i % KC, d = d0 + dd;
                const bool ok = d < D;
                sS[i] = ok ? s_t[(size_t)d * Kp + kc0 + kk] : 0.f;
                sN[i] = ok ? nms_t[(size_t)d * Kp + kc0 + kk] : 0.f;
            }
            for (int i = tid; i < P_DS * P_BM; i += P_THREADS) {
                const int r = i / P_DS, dd = i % P_DS, d = d0 + dd;
                const int64_t row = row0 + r;
                sX[dd * XS + r] = (row < rows && d < D) ? X[row * D + d] : 0.f;
            }
            __syncthreads();
#pragma unroll 4
            for (int dd = 0; dd < P_DS; ++dd) {
                const float4 xa = *reinterpret_cast<const float4 *>(&sX[dd * XS + warp * 8]);
                const float4 xb = *reinterpret_cast<const float4 *>(&sX[dd * XS + warp * 8 + 4]);
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                float sv[CPL], nv[CPL];
                if constexpr (CPL == 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(&sS[dd * KC + lane * 4]);
                    const float4 b = *reinterpret_cast<const float4 *>(&sN[dd * KC + lane * 4]);
                    sv[0] = a.x; sv[1] = a.y; sv[2] = a.z; sv[3] = a.w;
                    nv[0] = b.x; nv[1] = b.y; nv[2] = b.z; nv[3] = b.w;
                } else {
                    const float2 a = *reinterpret_cast<const float2 *>(&sS[dd * KC + lane * 2]);
                    const float2 b = *reinterpret_cast<const float2 *>(&sN[dd * KC + lane * 2]);
                    sv[0] = a.x; sv[1] = a.y;
                    nv[0] = b.x; nv[1] = b.y;
                }
#pragma unroll
                for (int r = 0; r < 8; ++r)
#pragma unroll
                    for (int c = 0; c < CPL; ++c) {
                        const float t = fmaf(xv[r], sv[c], nv[c]);
                        acc[r][c] = fmaf(t, t, acc[r][c]);
                    }
            }
        }
        // l = c' - dist/2 for this chunk
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const float ck = cst[kc0 + lane * CPL + c];
#pragma unroll
            for (int r = 0; r < 8; ++r) sL[(warp * 8 + r) * Kp + kc0 + lane * CPL + c] = fmaf(-0.5f, acc[r][c], ck);
        }
    }
    __syncthreads();

    // row softmax: each warp owns its 8 rows
    for (int r = 0; r < 8; ++r) {
        const int lr = warp * 8 + r;
        const int64_t row = row0 + lr;
        if (row >= rows) break;
        float *L = sL + (size_t)lr * Kp;
        float m = -INFINITY;
        for (int k = lane; k < Kp; k += 32) m = fmaxf(m, L[k]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float z = 0.f;
        for (int k = lane; k < Kp; k += 32) {
            const float e = expf(L[k] - m);
            L[k] = e;
            z += e;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        const float iz = 1.0f / z;
        float *G = gamma + row * Kp;
        for (int k = lane; k < Kp; k += 32) G[k] = L[k] * iz;
    }
}

constexpr int S_RS = 32;   // rows staged per step
constexpr int S_KC = 64;   // components per block
constexpr int S_DC = 64;   // dimensions per block
constexpr int S_CPT = 4;   // components per thread
constexpr int S_DPT = 8;   // dimensions per thread
constexpr int S_THREADS = (S_KC / S_CPT) * (S_DC / S_DPT);  // 128

constexpr int S_PER_THREAD = S_RS * S_KC / S_THREADS;  // 16 staged values of each kind per thread

// grid.x = statistics units (row ranges), grid.y = 64-component chunks,
// grid.z = 64-dimension chunks. Stages of 32 rows are double-buffered: the
// next stage's posteriors and descriptors are loaded into registers while the
// current one is consumed from shared memory.
__global__ void __launch_bounds__(S_THREADS, 3)
f32_stats_kernel(const float *__restrict__ X, int D, const float *__restrict__ gamma, int Kp, int Dp,
                 const float *__restrict__ mu_kd, const StatUnit *__restrict__ units, float *__restrict__ part,
                 int P) {
    __shared__ __align__(16) float sG[2][S_RS * S_KC];
    __shared__ __align__(16) float sXs[2][S_RS * S_DC];

    const StatUnit u = units[blockIdx.x];
    const int kc0 = blockIdx.y * S_KC, dc0 = blockIdx.z * S_DC;
    const int tid = threadIdx.x;
    const int cg = tid & 15, dg = tid >> 4;
    const int kb = kc0 + cg * S_CPT, dl = dg * S_DPT, db = dc0 + dl;
    const bool active = db < D;

    float m[S_CPT][S_DPT], U[S_CPT][S_DPT], W[S_CPT][S_DPT], S0[S_CPT];
#pragma unroll
    for (int c = 0; c < S_CPT; ++c) {
        S0[c] = 0.f;
#pragma unroll
        for (int j = 0; j < S_DPT; ++j) {
            m[c][j] = active ? mu_kd[(size_t)(kb + c) * Dp + db + j] : 0.f;
            U[c][j] = 0.f;
            W[c][j] = 0.f;
        }
    }

    float rg[S_PER_THREAD], rx[S_PER_THREAD];
    auto load = [&](int r0) {
#pragma unroll
        for (int q = 0; q < S_PER_THREAD; ++q) {
            const int i = tid + q * S_THREADS;
            const int r = i / S_KC, kk = i % S_KC, d = dc0 + kk;
            const bool rok = r0 + r < u.nrows;
            const int64_t row = u.row0 + r0 + r;
            rg[q] = rok ? gamma[row * Kp + kc0 + kk] : 0.f;
            rx[q] = (rok && d < D) ? X[row * D + d] : 0.f;
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int q = 0; q < S_PER_THREAD; ++q) {
            sG[b][tid + q * S_THREADS] = rg[q];
            sXs[b][tid + q * S_THREADS] = rx[q];
        }
    };

    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int r0 = 0; r0 < u.nrows; r0 += S_RS) {
        const bool more = r0 + S_RS < u.nrows;
        if (more) load(r0 + S_RS);
        if (active) {
            const float *G = sG[buf];
            const float *Xs = sXs[buf];
#pragma unroll 4
            for (int r = 0; r < S_RS; ++r) {
                const float4 g4 = *reinterpret_cast<const float4 *>(&G[r * S_KC + cg * S_CPT]);
                const float4 xa = *reinterpret_cast<const float4 *>(&Xs[r * S_DC + dl]);
                const float4 xb = *reinterpret_cast<const float4 *>(&Xs[r * S_DC + dl + 4]);
                const float gv[4] = {g4.x, g4.y, g4.z, g4.w};
                const float xv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
                for (int c = 0; c < S_CPT; ++c) {
                    S0[c] += gv[c];
#pragma unroll
                    for (int j = 0; j < S_DPT; ++j) {
                        const float dx = xv[j] - m[c][j];
                        const float gd = gv[c] * dx;
                        U[c][j] += gd;
                        W[c][j] = fmaf(gd, dx, W[c][j]);
                    }
                }
            }
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }
    if (!active) return;
    // slot layout part[slot][j][Kp]: this thread's 4 components are contiguous
    float *dst = part + (size_t)u.slot * Kp * P + kb;
#pragma unroll
    for (int j = 0; j < S_DPT; ++j) {
        if (db + j < D) {
            *reinterpret_cast<float4 *>(dst + (size_t)(db + j) * Kp) = make_float4(U[0][j], U[1][j], U[2][j], U[3][j]);
            *reinterpret_cast<float4 *>(dst + (size_t)(D + db + j) * Kp) =
                make_float4(W[0][j], W[1][j], W[2][j], W[3][j]);
        }
    }
    if (db == 0) *reinterpret_cast<float4 *>(dst + (size_t)(2 * D) * Kp) = make_float4(S0[0], S0[1], S0[2], S0[3]);
}

}  // namespace

cudaError_t launch_f32_posteriors(const fv_gmm *g, const float *X, int64_t rows, float *gamma, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int Kp = g->Kp;
    const int cpl = (Kp % 128 == 0) ? 4 : 2;
    const int KC = 32 * cpl;
    const size_t smem = sizeof(float) * (2 * P_DS * KC + P_DS * (P_BM + 4) + (size_t)P_BM * Kp);
    const unsigned grid = (unsigned)((rows + P_BM - 1) / P_BM);
    cudaError_t e;
    if (cpl == 4) {
        e = cudaFuncSetAttribute(f32_posteriors_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("f32_posteriors", st);
        f32_posteriors_kernel<4><<<grid, P_THREADS, smem, st>>>(X, rows, g->D, Kp, g->dev.s_t, g->dev.nms_t,
                                                                g->dev.cst, gamma);
    }
    } else {
        e = cudaFuncSetAttribute(f32_posteriors_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("f32_posteriors", st);
        f32_posteriors_kernel<2><<<grid, P_THREADS, smem, st>>>(X, rows, g->D, Kp, g->dev.s_t, g->dev.nms_t,
                                                                g->dev.cst, gamma);
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_f32_stats(const fv_gmm *g, const float *X, const float *gamma, const StatUnit *units,
                             int n_units, float *part, int P, cudaStream_t st) {
    if (n_units <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_units, (unsigned)(g->Kp / S_KC), (unsigned)((g->D + S_DC - 1) / S_DC));
    {
        KernelTimer kt_("f32_stats", st);
        f32_stats_kernel<<<grid, S_THREADS, 0, st>>>(X, g->D, gamma, g->Kp, g->Dp, g->dev.mu_kd, units, part, P);
    }
    return cudaGetLastError();
}

}  // namespace fv
