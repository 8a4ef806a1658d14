// Plain FP32 form of the encoder: SIMT kernels in the centred (direct) form.
//
// Posteriors (Algorithm 1 first loop; the paper's Phase 1, Algorithm 2):
//   l_ik = c'_k - 1/2 sum_d t_ikd^2,  t_ikd = x_id/sigma_kd - mu_kd/sigma_kd
//   gamma_ik = exp(l_ik - max_k l_ik) / sum_k exp(l_ik - max_k l_ik)
// (evaluated in base 2 on y = l log2(e))
// computed for a 64-row block against every component with register tiles of
// 8 rows x CPL components per thread (t is one FMA, t^2 accumulation another,
// both on component pairs with packed f32x2 instructions),
// the row block's log-likelihoods kept in shared memory for the softmax.
//
// Statistics (Algorithm 1 second loop; the paper's Phase 2, Algorithm 3 with
// one private copy of U, V per block): each block owns one row range and one
// 64-component chunk and accumulates, per (k, d) held in registers,
//   A_kd += gamma_ik (x_id - mu_kd),  B_kd += gamma_ik (x_id - mu_kd)^2,
//   S0_k += gamma_ik
// and the finalise kernel forms U = A/sigma and V = B/sigma^2 - S0.
// The residual x - mu carries a rounding error relative to itself; the
// posteriors' single-FMA form x/sigma - mu/sigma errs by ~eps |mu/sigma|, which
// is harmless inside a softmax but would be amplified near zero by the signed
// square root when a component's variance is tiny. Terms whose posterior is
// exactly zero (the FP32 exponential underflows for every component far from
// the descriptor, most of them in 64 dimensions) add exact zeros, so a warp
// skips a row when all its components' posteriors are zero: the sums are
// bitwise those of the dense loop. Every block writes its own statistics slot;
// the finalise kernel reduces the slots in a fixed order, so no atomics touch
// the result.
//
// Early termination (Sec. 3.3, Algorithm 5): with a posterior threshold
// tau > 0 a term whose posterior is not above tau is dropped (the threshold
// test of Algorithm 1's second loop), and a warp skips a row when all 16 of
// its components' posteriors are at or below tau (the paper skips an
// iteration when all 8 posteriors of its 2 x 4 tile are below 1e-6). The
// result is the thresholded encoding, not the exact one; tau = 0 runs the
// exact kernel unchanged.
#include "fv_internal.h"

namespace fv {

namespace {

// Packed FP32 pairs (f32x2: two lanes per instruction, same rounding as the
// scalar operations; halves the instruction count of the inner loops).
__device__ __forceinline__ uint64_t pk2(float a, float b) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void up2(uint64_t r, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r)); }
__device__ __forceinline__ uint64_t add2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t mul2(uint64_t a, uint64_t b) {
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c) {
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Asynchronous global -> shared copies (cp.async): `bytes` of 4 or 16, zero
// fill when !valid (the source is then not read; a valid address is passed).
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem, bool valid) {
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(s), "l"(gmem), "r"(valid ? 4 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

constexpr float kLog2eF = 1.4426950408889634f;
// 2^x (ex2.approx: relative error about 2^-22, far inside the FP32 form's tolerance)
__device__ __forceinline__ float ex2f_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int P_BM = 64;   // rows per posterior block
constexpr int P_DS = 16;   // dimension slice staged in shared memory
constexpr int P_THREADS = 256;

// Dynamic shared memory layout of the posteriors kernel:
//   two stages of
//     sS[P_DS][KC], sN[P_DS][KC]   1/sigma and -mu/sigma of a (component chunk, dimension slice)
//     sX[P_DS][P_BM + 4]           descriptor slice, dimension-major
//   sL[P_BM][Kp]                   log-likelihoods of the row block
// The (chunk, slice) phases run in order; phase p + 1 is copied in by
// cp.async while phase p is computed.
template <int CPL>
__global__ void __launch_bounds__(P_THREADS)
f32_posteriors_kernel(const float *__restrict__ X, int64_t rows, int D, int Kp,
                      const float *__restrict__ s_t, const float *__restrict__ nms_t,
                      const float *__restrict__ cst, float *__restrict__ gamma, float *__restrict__ lse) {
    constexpr int KC = 32 * CPL;
    constexpr int XS = P_BM + 4;
    constexpr int STAGE = 2 * P_DS * KC + P_DS * XS;
    extern __shared__ __align__(16) float smem[];
    float *sL = smem + 2 * STAGE;

    pdl_trigger();   // the statistics kernel may start launching (it waits for this grid)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * P_BM;
    const int nslice = (D + P_DS - 1) / P_DS, nphase = (Kp / KC) * nslice;

    auto issue = [&](int ph, int b) {
        const int kc0 = (ph / nslice) * KC, d0 = (ph % nslice) * P_DS;
        float *bS = smem + b * STAGE, *bN = bS + P_DS * KC, *bX = bN + P_DS * KC;
#pragma unroll
        for (int q = 0; q < P_DS * KC / 4 / P_THREADS; ++q) {   // 16-byte chunks of the GMM slices
            const int i = tid + q * P_THREADS;
            const int dd = i / (KC / 4), c4 = (i % (KC / 4)) * 4, d = d0 + dd;
            const bool ok = d < D;
            cp_async<16>(bS + dd * KC + c4, ok ? s_t + (size_t)d * Kp + kc0 + c4 : s_t, ok);
            cp_async<16>(bN + dd * KC + c4, ok ? nms_t + (size_t)d * Kp + kc0 + c4 : nms_t, ok);
        }
#pragma unroll
        for (int q = 0; q < P_DS * P_BM / P_THREADS; ++q) {     // descriptors, transposed
            const int i = tid + q * P_THREADS;
            const int r = i / P_DS, dd = i % P_DS, d = d0 + dd;
            const int64_t row = row0 + r;
            const bool ok = row < rows && d < D;
            cp_async<4>(bX + dd * XS + r, ok ? X + row * D + d : X, ok);
        }
        cp_async_commit();
    };
    issue(0, 0);

    uint64_t acc[8][CPL / 2];   // component pairs
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int c = 0; c < CPL / 2; ++c) acc[r][c] = 0ull;
    for (int ph = 0; ph < nphase; ++ph) {
        const int b = ph & 1;
        if (ph + 1 < nphase) issue(ph + 1, b ^ 1);
        else cp_async_commit();   // an empty group keeps the wait count uniform
        cp_async_wait1();         // this phase's copies (of this thread) have landed
        __syncthreads();          // ... and every thread's
        const float *sS = smem + b * STAGE, *sN = sS + P_DS * KC, *sX = sN + P_DS * KC;
        // the shared-memory operands of slice dd + 1 are loaded into
        // registers while slice dd is computed (the loads' latency is hidden)
        float4 pxa, pxb;
        float pv[2 * CPL];   // CPL scale values, then CPL offsets
        auto load = [&](int dd) {
            pxa = *reinterpret_cast<const float4 *>(&sX[dd * XS + warp * 8]);
            pxb = *reinterpret_cast<const float4 *>(&sX[dd * XS + warp * 8 + 4]);
            if constexpr (CPL == 4) {
                const float4 a = *reinterpret_cast<const float4 *>(&sS[dd * KC + lane * 4]);
                const float4 c = *reinterpret_cast<const float4 *>(&sN[dd * KC + lane * 4]);
                pv[0] = a.x; pv[1] = a.y; pv[2] = a.z; pv[3] = a.w;
                pv[4] = c.x; pv[5] = c.y; pv[6] = c.z; pv[7] = c.w;
            } else {
                const float2 a = *reinterpret_cast<const float2 *>(&sS[dd * KC + lane * 2]);
                const float2 c = *reinterpret_cast<const float2 *>(&sN[dd * KC + lane * 2]);
                pv[0] = a.x; pv[1] = a.y;
                pv[2] = c.x; pv[3] = c.y;
            }
        };
        load(0);
#pragma unroll
        for (int dd = 0; dd < P_DS; ++dd) {
            const float xv[8] = {pxa.x, pxa.y, pxa.z, pxa.w, pxb.x, pxb.y, pxb.z, pxb.w};
            uint64_t s2[CPL / 2], n2[CPL / 2];
#pragma unroll
            for (int c = 0; c < CPL / 2; ++c) {
                s2[c] = pk2(pv[2 * c], pv[2 * c + 1]);
                n2[c] = pk2(pv[CPL + 2 * c], pv[CPL + 2 * c + 1]);
            }
            if (dd + 1 < P_DS) load(dd + 1);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const uint64_t x2 = pk2(xv[r], xv[r]);
#pragma unroll
                for (int c = 0; c < CPL / 2; ++c) {
                    const uint64_t t = fma2(x2, s2[c], n2[c]);
                    acc[r][c] = fma2(t, t, acc[r][c]);
                }
            }
        }
        if (ph % nslice == nslice - 1) {   // chunk done: y = (c' - dist/2) log2(e)
            const int kc0 = (ph / nslice) * KC;
#pragma unroll
            for (int c = 0; c < CPL / 2; ++c) {
                const float ck0 = cst[kc0 + lane * CPL + 2 * c] * kLog2eF, ck1 = cst[kc0 + lane * CPL + 2 * c + 1] * kLog2eF;
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    float a0, a1;
                    up2(acc[r][c], a0, a1);
                    sL[(warp * 8 + r) * Kp + kc0 + lane * CPL + 2 * c] = fmaf(-0.5f * kLog2eF, a0, ck0);
                    sL[(warp * 8 + r) * Kp + kc0 + lane * CPL + 2 * c + 1] = fmaf(-0.5f * kLog2eF, a1, ck1);
                    acc[r][c] = 0ull;
                }
            }
        }
        __syncthreads();   // the stage is consumed before it is refilled (and sL is complete at the end)
    }

    // row softmax in base 2: each warp owns its 8 rows, a lane holds up to 16
    // of a row's values in registers (Kp <= 512)
    for (int r = 0; r < 8; ++r) {
        const int lr = warp * 8 + r;
        const int64_t row = row0 + lr;
        if (row >= rows) break;
        const float *L = sL + (size_t)lr * Kp;
        const int nk = Kp >> 5;
        float v[16];
        float m = -INFINITY;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = j < nk ? L[lane + 32 * j] : -INFINITY;
            m = fmaxf(m, v[j]);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float z = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            v[j] = j < nk ? ex2f_approx(v[j] - m) : 0.f;
            z += v[j];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        // the row's log-sum-exp, log sum_k exp(l_ik) = ln 2 (m + log2 z) (natural log; EM's log-likelihood)
        if (lse && lane == 0) lse[row] = (m + log2f(z)) * 0.69314718055994531f;
        const float iz = 1.0f / z;
        float *G = gamma + row * Kp;
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (j < nk) G[lane + 32 * j] = v[j] * iz;
    }
}

constexpr int S_RS = 32;   // rows staged per step
constexpr int S_KC = 64;   // components per block
constexpr int S_DC = 64;   // dimensions per block
constexpr int S_CPT = 4;   // components per thread
constexpr int S_DPT = 8;   // dimensions per thread
constexpr int S_THREADS = (S_KC / S_CPT) * (S_DC / S_DPT);  // 128

constexpr int S_BLOCKS_PER_SM = 3;

// grid.x = statistics units (row ranges), grid.y = 64-component chunks,
// grid.z = 64-dimension chunks. Stages of 32 rows are double-buffered in
// shared memory and filled by cp.async (16-byte copies when the rows allow,
// VEC) while the previous stage is consumed.
// THRESH: posteriors <= tau are dropped and rows whose 16 posteriors are all
// <= tau skipped (early termination); skip_count (nullable) receives, per
// block, the number of (row, 16-component group) pairs skipped and visited.
template <bool VEC, bool THRESH>
__global__ void __launch_bounds__(S_THREADS, S_BLOCKS_PER_SM)
f32_stats_kernel(const float *__restrict__ X, int D, const float *__restrict__ gamma, int Kp, int Dp,
                 const float *__restrict__ mu_kd, const StatUnit *__restrict__ units, float *__restrict__ part,
                 int P, float tau, unsigned long long *__restrict__ skip_count) {
    __shared__ __align__(16) float sG[2][S_RS * S_KC];
    __shared__ __align__(16) float sXs[2][S_RS * S_DC];

    pdl_wait();      // the posteriors are complete
    pdl_trigger();
    const StatUnit u = units[blockIdx.x];
    const int kc0 = blockIdx.y * S_KC, dc0 = blockIdx.z * S_DC;
    const int tid = threadIdx.x;
    // warp w takes components 16w..16w+15 over all 64 dimensions (lanes:
    // 4 component groups x 8 dimension groups), so a row whose posteriors
    // are exactly zero for those 16 components can be skipped by the whole
    // warp: it would add exact zeros (the FP32 exponential underflows for
    // every component far from the descriptor)
    const int cg = (tid >> 5) * 4 + (tid & 3), dg = (tid & 31) >> 2;
    const int kb = kc0 + cg * S_CPT, dl = dg * S_DPT, db = dc0 + dl;
    const bool active = db < D;

    // stage r0 -> buffer b: gamma[row][kc0..kc0+63] and X[row][dc0..dc0+63]
    auto issue = [&](int r0, int b) {
        if constexpr (VEC) {
#pragma unroll
            for (int q = 0; q < S_RS * S_KC / 4 / S_THREADS; ++q) {   // 16-byte chunks
                const int i = tid + q * S_THREADS;
                const int r = i >> 4, c4 = (i & 15) * 4;
                const bool rok = r0 + r < u.nrows;
                const int64_t row = u.row0 + r0 + r;
                cp_async<16>(&sG[b][r * S_KC + c4], rok ? gamma + row * Kp + kc0 + c4 : gamma, rok);
                const bool xok = rok && dc0 + c4 < D;
                cp_async<16>(&sXs[b][r * S_DC + c4], xok ? X + row * D + dc0 + c4 : X, xok);
            }
        } else {
#pragma unroll
            for (int q = 0; q < S_RS * S_KC / S_THREADS; ++q) {
                const int i = tid + q * S_THREADS;
                const int r = i / S_KC, kk = i % S_KC;
                const bool rok = r0 + r < u.nrows;
                const int64_t row = u.row0 + r0 + r;
                cp_async<4>(&sG[b][i], rok ? gamma + row * Kp + kc0 + kk : gamma, rok);
                const bool xok = rok && dc0 + kk < D;
                cp_async<4>(&sXs[b][i], xok ? X + row * D + dc0 + kk : X, xok);
            }
        }
        cp_async_commit();
    };
    issue(0, 0);

    uint64_t nm[S_CPT][S_DPT / 2], U[S_CPT][S_DPT / 2], W[S_CPT][S_DPT / 2];
    float S0[S_CPT];
#pragma unroll
    for (int c = 0; c < S_CPT; ++c) {
        S0[c] = 0.f;
#pragma unroll
        for (int j = 0; j < S_DPT / 2; ++j) {
            const float m0 = active ? mu_kd[(size_t)(kb + c) * Dp + db + 2 * j] : 0.f;
            const float m1 = active ? mu_kd[(size_t)(kb + c) * Dp + db + 2 * j + 1] : 0.f;
            nm[c][j] = pk2(-m0, -m1);
            U[c][j] = 0ull;
            W[c][j] = 0ull;
        }
    }

    int buf = 0;
    unsigned skipped = 0, visited = 0;   // (row, 16-component group) pairs of this warp
    for (int r0 = 0; r0 < u.nrows; r0 += S_RS) {
        if (r0 + S_RS < u.nrows) issue(r0 + S_RS, buf ^ 1);
        else cp_async_commit();   // an empty group keeps the wait count uniform
        cp_async_wait1();         // this stage's copies (of this thread) have landed
        __syncthreads();          // ... and every thread's
        {
            const float *G = sG[buf];
            const float *Xs = sXs[buf];
            // the operands of row r + 1 are loaded while row r is accumulated
            float4 g4 = *reinterpret_cast<const float4 *>(&G[cg * S_CPT]);
            float4 xa = *reinterpret_cast<const float4 *>(&Xs[dl]);
            float4 xb = *reinterpret_cast<const float4 *>(&Xs[dl + 4]);
#pragma unroll 4
            for (int r = 0; r < S_RS; ++r) {
                float gv[4] = {g4.x, g4.y, g4.z, g4.w};
                const uint64_t xv[4] = {pk2(xa.x, xa.y), pk2(xa.z, xa.w), pk2(xb.x, xb.y), pk2(xb.z, xb.w)};
                if (r + 1 < S_RS) {
                    g4 = *reinterpret_cast<const float4 *>(&G[(r + 1) * S_KC + cg * S_CPT]);
                    xa = *reinterpret_cast<const float4 *>(&Xs[(r + 1) * S_DC + dl]);
                    xb = *reinterpret_cast<const float4 *>(&Xs[(r + 1) * S_DC + dl + 4]);
                }
                if constexpr (THRESH) {
#pragma unroll
                    for (int c = 0; c < S_CPT; ++c) gv[c] = gv[c] > tau ? gv[c] : 0.f;   // dropped terms
                    if (r0 + r < u.nrows) ++visited;
                }
                const bool nz = (gv[0] != 0.f) | (gv[1] != 0.f) | (gv[2] != 0.f) | (gv[3] != 0.f);
                if (!__any_sync(0xffffffffu, nz)) {   // exact zeros (or dropped terms) for all 16 components
                    if constexpr (THRESH) {
                        if (r0 + r < u.nrows) ++skipped;
                    }
                    continue;
                }
#pragma unroll
                for (int c = 0; c < S_CPT; ++c) {
                    S0[c] += gv[c];
                    const uint64_t g2 = pk2(gv[c], gv[c]);
#pragma unroll
                    for (int j = 0; j < S_DPT / 2; ++j) {
                        const uint64_t dx = add2(xv[j], nm[c][j]);
                        const uint64_t gd = mul2(g2, dx);
                        U[c][j] = add2(U[c][j], gd);
                        W[c][j] = fma2(gd, dx, W[c][j]);
                    }
                }
            }
        }
        __syncthreads();   // the buffer is consumed before it is refilled
        buf ^= 1;
    }
    if constexpr (THRESH) {
        if (skip_count && (threadIdx.x & 31) == 0 && dc0 == 0) {   // one count per warp and component group
            atomicAdd(&skip_count[0], (unsigned long long)skipped);
            atomicAdd(&skip_count[1], (unsigned long long)visited);
        }
    }
    if (!active) return;
    // slot layout part[slot][j][Kp]: this thread's 4 components are contiguous
    float *dst = part + (size_t)u.slot * Kp * P + kb;
#pragma unroll
    for (int jp = 0; jp < S_DPT / 2; ++jp) {
        float u0[S_CPT], u1[S_CPT], w0[S_CPT], w1[S_CPT];
#pragma unroll
        for (int c = 0; c < S_CPT; ++c) {
            up2(U[c][jp], u0[c], u1[c]);
            up2(W[c][jp], w0[c], w1[c]);
        }
        const int j = db + 2 * jp;
        if (j < D) {
            *reinterpret_cast<float4 *>(dst + (size_t)j * Kp) = make_float4(u0[0], u0[1], u0[2], u0[3]);
            *reinterpret_cast<float4 *>(dst + (size_t)(D + j) * Kp) = make_float4(w0[0], w0[1], w0[2], w0[3]);
        }
        if (j + 1 < D) {
            *reinterpret_cast<float4 *>(dst + (size_t)(j + 1) * Kp) = make_float4(u1[0], u1[1], u1[2], u1[3]);
            *reinterpret_cast<float4 *>(dst + (size_t)(D + j + 1) * Kp) = make_float4(w1[0], w1[1], w1[2], w1[3]);
        }
    }
    if (db == 0) *reinterpret_cast<float4 *>(dst + (size_t)(2 * D) * Kp) = make_float4(S0[0], S0[1], S0[2], S0[3]);
}

}  // namespace

cudaError_t launch_f32_posteriors(const fv_gmm *g, const float *X, int64_t rows, float *gamma, cudaStream_t st,
                                  float *lse) {
    if (rows <= 0) return cudaSuccess;
    const int Kp = g->Kp;
    const int cpl = (Kp % 128 == 0) ? 4 : 2;
    const int KC = 32 * cpl;
    const size_t smem = sizeof(float) * (2 * (2 * P_DS * KC + P_DS * (P_BM + 4)) + (size_t)P_BM * Kp);
    const unsigned grid = (unsigned)((rows + P_BM - 1) / P_BM);
    cudaError_t e;
    if (cpl == 4) {
        e = cudaFuncSetAttribute(f32_posteriors_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("f32_posteriors", st);
        f32_posteriors_kernel<4><<<grid, P_THREADS, smem, st>>>(X, rows, g->D, Kp, g->dev.s_t, g->dev.nms_t,
                                                                g->dev.cst, gamma, lse);
    }
    } else {
        e = cudaFuncSetAttribute(f32_posteriors_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        {
        KernelTimer kt_("f32_posteriors", st);
        f32_posteriors_kernel<2><<<grid, P_THREADS, smem, st>>>(X, rows, g->D, Kp, g->dev.s_t, g->dev.nms_t,
                                                                g->dev.cst, gamma, lse);
    }
    }
    return cudaGetLastError();
}

cudaError_t launch_f32_stats(const fv_gmm *g, const float *X, const float *gamma, const StatUnit *units,
                             int n_units, float *part, int P, cudaStream_t st, bool pdl, float tau,
                             unsigned long long *skip_count) {
    if (n_units <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_units, (unsigned)(g->Kp / S_KC), (unsigned)((g->D + S_DC - 1) / S_DC));
    // 16-byte copies need 16-byte aligned rows of X (gamma rows always are)
    const bool vec = (g->D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const bool thr = tau > 0.f;
    auto kern = vec ? (thr ? f32_stats_kernel<true, true> : f32_stats_kernel<true, false>)
                    : (thr ? f32_stats_kernel<false, true> : f32_stats_kernel<false, false>);
    {
        KernelTimer kt_("f32_stats", st);
        return launch_pdl(pdl, kern, grid, dim3(S_THREADS), 0, st, X, g->D, gamma, g->Kp, g->Dp, g->dev.mu_kd, units,
                          part, P, tau, skip_count);
    }
    return cudaGetLastError();
}

}  // namespace fv
