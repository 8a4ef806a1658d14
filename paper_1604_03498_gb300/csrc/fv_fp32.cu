// Plain FP32 form of the encoder: SIMT kernels in the centred (direct) form.
//
// Posteriors (Algorithm 1 first loop; the paper's Phase 1, Algorithm 2):
//   l_ik = c'_k - 1/2 sum_d t_ikd^2,  t_ikd = x_id/sigma_kd - mu_kd/sigma_kd
//   gamma_ik = exp(l_ik - max_k l_ik) / sum_k exp(l_ik - max_k l_ik)
// (evaluated in base 2 on y = l log2(e))
// computed for 4 rows per warp against every component, a lane holding
// CPL components of each 32 CPL-component chunk (t is one FMA, t^2
// accumulation another, both on component pairs with packed f32x2
// instructions); the log-likelihoods stay in registers for the softmax.
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
// bitwise those of the dense loop. The posteriors kernel writes only the
// 16-component groups of a row that hold a non-zero posterior, with a 32-bit
// group mask per row; the statistics kernel zero-fills the other groups
// instead of reading them, so the posteriors' round trip through memory
// carries the non-zero groups only, and each statistics block first lists
// the rows with a non-zero group in its 64 components and stages only those. Every block writes its own statistics slot;
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

constexpr int P_THREADS = 256;

// Posteriors kernel: a warp owns RR rows and every component (lane l holds
// components c KCH + l CPL .. + CPL - 1 of each chunk c of KCH = 32 CPL), so a
// row's log-likelihoods never leave registers and the row softmax is a pair
// of warp shuffle reductions. The block (8 warps, 8 RR rows) stages only the
// GMM slices and the descriptor slice, 8 dimensions at a time (double-buffered
// by cp.async). Each GMM value read from shared memory serves RR rows: at
// RR = 4 a warp's shared-memory wavefronts per dimension (17) match its FMA
// cycles per SM (16), so K <= 256 takes RR = 8 (two blocks per SM, twice the
// FMAs per load); larger K keeps RR = 4 (three blocks per SM at K <= 256
// would need it, and 8 rows x 16 components of accumulators do not fit).
// dimension slice: 16 dimensions (half as many slice hand-overs) where two
// stages of it leave room for two blocks per SM, else 8
__host__ __device__ constexpr int r_ds(int kt) { return kt <= 256 ? 16 : 8; }

template <int CPL, int NC, int RR>
__global__ void __launch_bounds__(P_THREADS, (CPL * NC <= 8 && RR == 4) ? 3 : 2)
f32_post_reg_kernel(const float *__restrict__ X, int64_t rows, int D, int Kp, const float *__restrict__ s_t,
                    const float *__restrict__ nms_t, const float *__restrict__ cst, float *__restrict__ gamma,
                    uint32_t *__restrict__ gmask, float *__restrict__ lse) {
    constexpr int KCH = 32 * CPL;          // components per chunk
    constexpr int KT = KCH * NC;           // all (padded) components
    constexpr int BM = 8 * RR;             // rows per block
    constexpr int XS = BM + 4;
    constexpr int R_DS = r_ds(KT);
    constexpr int STAGE = 2 * R_DS * KT + R_DS * XS;
    extern __shared__ __align__(16) float smem[];

    pdl_trigger();   // the statistics kernel may start launching (it waits for this grid)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t row0 = (int64_t)blockIdx.x * BM;
    const int nslice = (D + R_DS - 1) / R_DS;

    auto issue = [&](int sl, int b) {
        const int d0 = sl * R_DS;
        float *bS = smem + b * STAGE, *bN = bS + R_DS * KT, *bX = bN + R_DS * KT;
#pragma unroll
        for (int i = tid; i < R_DS * KT / 4; i += P_THREADS) {   // 16-byte chunks of the GMM slices
            const int dd = i / (KT / 4), c4 = (i % (KT / 4)) * 4, d = d0 + dd;
            const bool ok = d < D;
            cp_async<16>(bS + dd * KT + c4, ok ? s_t + (size_t)d * Kp + c4 : s_t, ok);
            cp_async<16>(bN + dd * KT + c4, ok ? nms_t + (size_t)d * Kp + c4 : nms_t, ok);
        }
#pragma unroll
        for (int i = tid; i < BM * R_DS; i += P_THREADS) {   // the block's descriptor slice, dimension-major
            const int r = i / R_DS, dd = i % R_DS, d = d0 + dd;
            const int64_t row = row0 + r;
            const bool ok = row < rows && d < D;
            cp_async<4>(bX + dd * XS + r, ok ? X + row * D + d : X, ok);
        }
        cp_async_commit();
    };
    issue(0, 0);

    uint64_t acc[RR][NC][CPL / 2];
#pragma unroll
    for (int r = 0; r < RR; ++r)
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int p = 0; p < CPL / 2; ++p) acc[r][c][p] = 0ull;

    for (int sl = 0; sl < nslice; ++sl) {
        const int b = sl & 1;
        if (sl + 1 < nslice) issue(sl + 1, b ^ 1);
        else cp_async_commit();   // an empty group keeps the wait count uniform
        cp_async_wait1();
        __syncthreads();
        const float *sS = smem + b * STAGE, *sN = sS + R_DS * KT, *sX = sN + R_DS * KT;
#pragma unroll
        for (int dd = 0; dd < R_DS; ++dd) {
            uint64_t x2[RR];
#pragma unroll
            for (int q = 0; q < RR / 4; ++q) {
                const float4 xv = *reinterpret_cast<const float4 *>(&sX[dd * XS + warp * RR + 4 * q]);
                x2[4 * q] = pk2(xv.x, xv.x);
                x2[4 * q + 1] = pk2(xv.y, xv.y);
                x2[4 * q + 2] = pk2(xv.z, xv.z);
                x2[4 * q + 3] = pk2(xv.w, xv.w);
            }
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                uint64_t s2[CPL / 2], n2[CPL / 2];
                const int k = c * KCH + lane * CPL;
                if constexpr (CPL == 4) {
                    const float4 a = *reinterpret_cast<const float4 *>(&sS[dd * KT + k]);
                    const float4 o = *reinterpret_cast<const float4 *>(&sN[dd * KT + k]);
                    s2[0] = pk2(a.x, a.y);
                    s2[1] = pk2(a.z, a.w);
                    n2[0] = pk2(o.x, o.y);
                    n2[1] = pk2(o.z, o.w);
                } else {
                    const float2 a = *reinterpret_cast<const float2 *>(&sS[dd * KT + k]);
                    const float2 o = *reinterpret_cast<const float2 *>(&sN[dd * KT + k]);
                    s2[0] = pk2(a.x, a.y);
                    n2[0] = pk2(o.x, o.y);
                }
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int p = 0; p < CPL / 2; ++p) {
                        const uint64_t t = fma2(x2[r], s2[p], n2[p]);
                        acc[r][c][p] = fma2(t, t, acc[r][c][p]);
                    }
            }
        }
        __syncthreads();   // the stage is consumed before it is refilled
    }

    // y = (c' - dist/2) log2(e), row softmax in base 2 across the warp
    float cl[NC][CPL];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int j = 0; j < CPL; ++j) cl[c][j] = cst[c * KCH + lane * CPL + j] * kLog2eF;
#pragma unroll
    for (int r = 0; r < RR; ++r) {
        const int64_t row = row0 + warp * RR + r;
        float y[NC][CPL];
        float m = -INFINITY;
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int p = 0; p < CPL / 2; ++p) {
                float a0, a1;
                up2(acc[r][c][p], a0, a1);
                y[c][2 * p] = fmaf(-0.5f * kLog2eF, a0, cl[c][2 * p]);
                y[c][2 * p + 1] = fmaf(-0.5f * kLog2eF, a1, cl[c][2 * p + 1]);
                m = fmaxf(m, fmaxf(y[c][2 * p], y[c][2 * p + 1]));
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        float z = 0.f;
#pragma unroll
        for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                y[c][j] = ex2f_approx(y[c][j] - m);
                z += y[c][j];
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        if (row >= rows) continue;
        // the row's log-sum-exp, log sum_k exp(l_ik) = ln 2 (m + log2 z) (natural log; EM's log-likelihood)
        if (lse && lane == 0) lse[row] = (m + log2f(z)) * 0.69314718055994531f;
        const float iz = 1.0f / z;
        float *G = gamma + row * Kp;
        // only the 16-component groups holding a non-zero posterior are
        // written; the row's group mask tells the statistics kernel which
        constexpr int L = 16 / CPL;   // lanes per group
        uint32_t rmask = 0;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            float gv[CPL];
            bool nz = false;
#pragma unroll
            for (int j = 0; j < CPL; ++j) {
                gv[j] = y[c][j] * iz;
                nz |= gv[j] != 0.f;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, nz);
#pragma unroll
            for (int q = 0; q < 32 / L; ++q)
                if ((bal >> (q * L)) & ((1u << L) - 1u)) rmask |= 1u << (c * (KCH / 16) + q);
            if (!((bal >> ((lane / L) * L)) & ((1u << L) - 1u))) continue;
            if constexpr (CPL == 4)
                *reinterpret_cast<float4 *>(G + c * KCH + lane * 4) = make_float4(gv[0], gv[1], gv[2], gv[3]);
            else
                *reinterpret_cast<float2 *>(G + c * KCH + lane * 2) = make_float2(gv[0], gv[1]);
        }
        if (lane == 0) gmask[row] = rmask;
    }
}

constexpr int S_RS = 32;   // rows staged per step
constexpr int S_KC = 64;   // components per block
constexpr int S_DC = 64;   // dimensions per block
constexpr int S_CPT = 4;   // components per thread
constexpr int S_DPT = 8;   // dimensions per thread
constexpr int S_THREADS = (S_KC / S_CPT) * (S_DC / S_DPT);  // 128

constexpr int S_BLOCKS_PER_SM = 3;
constexpr int S_WIN = 512;  // rows per compaction window (row offsets fit 16 bits)

// grid.x = statistics units (row ranges), grid.y = 64-component chunks,
// grid.z = 64-dimension chunks. Stages of 32 rows are double-buffered in
// shared memory and filled by cp.async (16-byte copies when the rows allow,
// VEC) while the previous stage is consumed.
// THRESH: posteriors <= tau are dropped and rows whose 16 posteriors are all
// <= tau skipped (early termination); skip_count (nullable) receives, per
// block, the number of (row, 16-component group) pairs skipped and visited.
template <bool VEC, bool THRESH>
__global__ void __launch_bounds__(S_THREADS, S_BLOCKS_PER_SM)
f32_stats_kernel(const float *__restrict__ X, int D, const float *__restrict__ gamma,
                 const uint32_t *__restrict__ gmask, int Kp, int Dp,
                 const float *__restrict__ mu_kd, const StatUnit *__restrict__ units, float *__restrict__ part,
                 int P, float tau, unsigned long long *__restrict__ skip_count) {
    __shared__ __align__(16) float sG[2][S_RS * S_KC];
    __shared__ __align__(16) float sXs[2][S_RS * S_DC];
    __shared__ uint32_t sList[S_WIN];
    __shared__ int sWarpCnt[S_THREADS / 32];

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

    // The unit's rows in windows of S_WIN. First the window's live rows (some
    // posterior of the block's 64 components non-zero, from the group masks)
    // are listed in increasing order as (row - w0) | (group bits << 16); a row
    // whose four groups are all zero would add exact zeros, so it is neither
    // staged nor visited (the early-termination counts take it as visited and
    // skipped by every warp). Then the listed rows are staged 32 at a time,
    // double-buffered: entries l0..l0+31 -> buffer b, gamma[row][kc0..kc0+63]
    // (a group whose bit is clear zero-filled, not read) and X[row][dc0..dc0+63].
    auto issue = [&](int w0, int l0, int nlive, int b) {
        if constexpr (VEC) {
#pragma unroll
            for (int q = 0; q < S_RS * S_KC / 4 / S_THREADS; ++q) {   // 16-byte chunks
                const int i = tid + q * S_THREADS;
                const int r = i >> 4, c4 = (i & 15) * 4;
                const bool rok = l0 + r < nlive;
                const uint32_t e = rok ? sList[l0 + r] : 0u;
                const int64_t row = u.row0 + w0 + (int)(e & 0xFFFFu);
                const bool gok = rok && ((e >> (16 + (c4 >> 4))) & 1u);
                cp_async<16>(&sG[b][r * S_KC + c4], gok ? gamma + row * Kp + kc0 + c4 : gamma, gok);
                const bool xok = rok && dc0 + c4 < D;
                cp_async<16>(&sXs[b][r * S_DC + c4], xok ? X + row * D + dc0 + c4 : X, xok);
            }
        } else {
#pragma unroll
            for (int q = 0; q < S_RS * S_KC / S_THREADS; ++q) {
                const int i = tid + q * S_THREADS;
                const int r = i / S_KC, kk = i % S_KC;
                const bool rok = l0 + r < nlive;
                const uint32_t e = rok ? sList[l0 + r] : 0u;
                const int64_t row = u.row0 + w0 + (int)(e & 0xFFFFu);
                const bool gok = rok && ((e >> (16 + (kk >> 4))) & 1u);
                cp_async<4>(&sG[b][i], gok ? gamma + row * Kp + kc0 + kk : gamma, gok);
                const bool xok = rok && dc0 + kk < D;
                cp_async<4>(&sXs[b][i], xok ? X + row * D + dc0 + kk : X, xok);
            }
        }
        cp_async_commit();
    };

    int buf = 0;
    unsigned skipped = 0, visited = 0;   // (row, 16-component group) pairs of this warp
    for (int w0 = 0; w0 < u.nrows; w0 += S_WIN) {
        const int wn = min(S_WIN, u.nrows - w0);
        int nlive = 0;
#pragma unroll
        for (int q = 0; q < S_WIN / S_THREADS; ++q) {   // the window's live rows, in order
            const int r = q * S_THREADS + tid;
            const uint32_t gb = r < wn ? (gmask[u.row0 + w0 + r] >> (kc0 >> 4)) & 0xFu : 0u;
            const uint32_t bal = __ballot_sync(0xffffffffu, gb != 0u);
            if ((tid & 31) == 0) sWarpCnt[tid >> 5] = __popc(bal);
            __syncthreads();
            int base = nlive, tot = 0;
#pragma unroll
            for (int w = 0; w < S_THREADS / 32; ++w) {
                base += w < (tid >> 5) ? sWarpCnt[w] : 0;
                tot += sWarpCnt[w];
            }
            if (gb) sList[base + __popc(bal & ((1u << (tid & 31)) - 1u))] = (uint32_t)r | (gb << 16);
            nlive += tot;
            __syncthreads();   // the counts are read before the next pass writes them; the list is complete
        }
        if constexpr (THRESH) {
            visited += (unsigned)(wn - nlive);
            skipped += (unsigned)(wn - nlive);
        }
        if (nlive == 0) continue;
        issue(w0, 0, nlive, buf);
        for (int l0 = 0; l0 < nlive; l0 += S_RS) {
            if (l0 + S_RS < nlive) issue(w0, l0 + S_RS, nlive, buf ^ 1);
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
                        if (l0 + r < nlive) ++visited;
                    }
                    const bool nz = (gv[0] != 0.f) | (gv[1] != 0.f) | (gv[2] != 0.f) | (gv[3] != 0.f);
                    if (!__any_sync(0xffffffffu, nz)) {   // exact zeros (or dropped terms) for all 16 components
                        if constexpr (THRESH) {
                            if (l0 + r < nlive) ++skipped;
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

namespace {
template <int CPL, int NC, int RR = (CPL * NC <= 8 ? 8 : 4)>
cudaError_t launch_post_reg(const fv_gmm *g, const float *X, int64_t rows, float *gamma, cudaStream_t st, float *lse) {
    constexpr int KT = 32 * CPL * NC, BM = 8 * RR;
    constexpr int R_DS = r_ds(KT);
    const size_t smem = sizeof(float) * 2 * (2 * R_DS * KT + R_DS * (BM + 4));
    cudaError_t e = cudaFuncSetAttribute(f32_post_reg_kernel<CPL, NC, RR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    {
        KernelTimer kt_("f32_posteriors", st);
        f32_post_reg_kernel<CPL, NC, RR><<<(unsigned)((rows + BM - 1) / BM), P_THREADS, smem, st>>>(
            X, rows, g->D, g->Kp, g->dev.s_t, g->dev.nms_t, g->dev.cst, gamma, f32_gamma_mask(gamma, rows, g->Kp), lse);
    }
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_f32_posteriors(const fv_gmm *g, const float *X, int64_t rows, float *gamma, cudaStream_t st,
                                  float *lse) {
    if (rows <= 0) return cudaSuccess;
    switch (g->Kp) {   // Kp is K rounded up to 64, at most 512
        case 64: return launch_post_reg<2, 1>(g, X, rows, gamma, st, lse);
        case 128: return launch_post_reg<4, 1>(g, X, rows, gamma, st, lse);
        case 192: return launch_post_reg<2, 3>(g, X, rows, gamma, st, lse);
        case 256: return launch_post_reg<4, 2>(g, X, rows, gamma, st, lse);
        case 320: return launch_post_reg<2, 5>(g, X, rows, gamma, st, lse);
        case 384: return launch_post_reg<4, 3>(g, X, rows, gamma, st, lse);
        case 448: return launch_post_reg<2, 7>(g, X, rows, gamma, st, lse);
        case 512: return launch_post_reg<4, 4>(g, X, rows, gamma, st, lse);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_f32_stats(const fv_gmm *g, const float *X, const float *gamma, int64_t rows,
                             const StatUnit *units, int n_units, float *part, int P, cudaStream_t st, bool pdl,
                             float tau, unsigned long long *skip_count) {
    if (n_units <= 0) return cudaSuccess;
    dim3 grid((unsigned)n_units, (unsigned)(g->Kp / S_KC), (unsigned)((g->D + S_DC - 1) / S_DC));
    // 16-byte copies need 16-byte aligned rows of X (gamma rows always are)
    const bool vec = (g->D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    const bool thr = tau > 0.f;
    auto kern = vec ? (thr ? f32_stats_kernel<true, true> : f32_stats_kernel<true, false>)
                    : (thr ? f32_stats_kernel<false, true> : f32_stats_kernel<false, false>);
    {
        KernelTimer kt_("f32_stats", st);
        return launch_pdl(pdl, kern, grid, dim3(S_THREADS), 0, st, X, g->D, gamma,
                          (const uint32_t *)f32_gamma_mask(const_cast<float *>(gamma), rows, g->Kp), g->Kp, g->Dp, g->dev.mu_kd, units,
                          part, P, tau, skip_count);
    }
    return cudaGetLastError();
}

}  // namespace fv
