// BF16 precision form of the encoder on the 5th-generation tensor cores
// (tcgen05 MMA with TMEM accumulators, TMA-fed shared-memory operands).
//
// Log-likelihood GEMM (the distance/posterior step of Algorithm 1; the
// paper's Phase 1, Algorithm 2, "the most time consuming computation"):
//   l_ik = c_k + sum_d x_id Q_kd + sum_d x_id^2 R_kd,
//   Q = mu/sigma^2, R = -1/(2 sigma^2), c_k = log w_k - 1/2 sum log sigma^2
//   - 1/2 sum mu^2/sigma^2 (FP64 on the device, once per GMM).
// x is bfloat16 (exact), Q and R are split into bf16 hi + lo parts, and x^2
// (16 significant bits for a bf16 x) into hi + lo, so five products
//   x Q_hi + x Q_lo + x2_hi R_hi + x2_hi R_lo + x2_lo R_hi
// accumulate in FP32 in TMEM and undo the cancellation between x^2/sigma^2
// and 2 x mu/sigma^2. A 128-row tile x all components of the CTA lives in one
// TMEM buffer (two buffers alternate so the next tile's MMAs overlap this
// tile's epilogue). The epilogue (one thread per row) makes three passes over
// the row in TMEM: row max, exponentials (stored back into TMEM) with their
// sum, then normalised posteriors written to global memory as bfloat16.
// With more than 256 components the components are split over a 2-CTA
// cluster; the two CTAs exchange each row's (max, sum) through distributed
// shared memory.
//
// Statistics GEMM (Algorithm 1 second loop; Phase 2, Algorithm 3):
//   [S1 | S2hi | S2lo | S0] = gamma^T [X | X2hi | X2lo | 1]
// with gamma^T (components x rows) and the row-major Y both read as MN-major
// operands; 128-component accumulators live in TMEM for a whole row range and
// are written to that range's statistics slot (the paper's per-block copies).
// The finalise kernel centres the raw moments in FP64.
//
// Shared-memory operand layout everywhere: blocks of 16 bf16 columns, each a
// [rows][16] array of 32-byte rows with the 32-byte swizzle (TMA writes it,
// the MMA descriptors read it: SBO = 256 B per 8-row group, LBO = block stride).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "fv_bf16.h"
#include "fv_sm100.cuh"

namespace fv {

using namespace sm100;

namespace {

constexpr int kThreads = 256;          // statistics kernel: 8 warps
constexpr int kPostThreads = 384;      // posteriors kernel: 12 warps
constexpr int kTileRows = 128;         // posteriors tile (MMA M)
constexpr int kStatRows = 64;          // statistics stage rows
constexpr int kStatStages = 3;
constexpr uint32_t kGBlk = 64u * kStatRows * 2u;   // one 64-component x 64-row gamma box (8 KB)
constexpr float kLog2e = 1.4426950408889634f;

// ---- small device helpers ---------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float bf16lo_to_f32(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16hi_to_f32(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// x (8 bf16 in a uint4) -> x^2 split into bf16 hi and lo parts (exact: hi + lo == x^2)
__device__ __forceinline__ void square_split(const uint4 &x, uint4 &hi, uint4 &lo) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = bf16lo_to_f32(w[i]), b = bf16hi_to_f32(w[i]);
        const float a2 = a * a, b2 = b * b;
        const uint32_t hp = pack_bf16x2(a2, b2);
        h[i] = hp;
        l[i] = pack_bf16x2(a2 - bf16lo_to_f32(hp), b2 - bf16hi_to_f32(hp));
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---- posteriors ------------------------------------------------------------------------
struct PostArgs {
    int64_t rows;
    int ntiles;
    const int64_t *rows_dev;   // if set, the row count is read here at kernel start (graph replays)
    int nkb;        // D16 / 16
    int Kp;
    int ncta;       // components per CTA (multiple of 16, <= 256)
    int split;      // CTAs per cluster sharing a row tile (1 or 2)
    int nstage;     // A-operand stages (1 or 2)
    uint32_t tmem_cols;
    const float *cl2;     // [Kp] log-constant times log2(e) (-inf on padding)
    uint16_t *gamma;      // [rows][Kp] bf16 posteriors
    uint32_t *err;
};

struct PostSmem {
    // byte offsets from the (1024-aligned) dynamic shared-memory base
    uint32_t b, a, hx, xchg, bars, misc, total;
    uint32_t a_stage;   // bytes per A stage
};

__host__ __device__ inline PostSmem post_smem(int nkb, int ncta, int nstage, int split) {
    PostSmem s;
    uint32_t off = 0;
    s.b = off;
    off += 4u * nkb * ncta * 32u;
    s.a_stage = 3u * nkb * kTileRows * 32u;
    s.a = off;
    off += nstage * s.a_stage;
    s.hx = off;                       // (max, sum) of each row's two column halves
    off += 2u * kTileRows * 8u;
    s.xchg = off;
    off += split > 1 ? 2u * kTileRows * 8u : 0u;
    off = (off + 15u) & ~15u;
    s.bars = off;
    off += 24u * 8u;
    s.misc = off;
    off += 16u;
    s.total = off;
    return s;
}

// Barrier indices in the barrier array.
enum { PB_BFULL = 0, PB_XFULL = 1, PB_AFULL = 3, PB_AEMPTY = 5, PB_LFULL = 7, PB_LEMPTY = 9, PB_XCHG = 11,
       PB_DRAIN = 13, PB_HXFULL = 16, PB_HXFREE = 20 };

__global__ void __launch_bounds__(kPostThreads, 1)
bf16_posteriors_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB,
                       PostArgs p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const PostSmem L = post_smem(p.nkb, p.ncta, p.nstage, p.split);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);   // [0] tmem base, [1] abort
    volatile uint32_t *abort_flag = misc + 1;

    if ((smem_u32(smem) & 1023u) != 0u) {   // layout assumption broken: refuse to run
        if (threadIdx.x == 0) atomicOr(p.err, kErrAlign);
        return;
    }
    const uint32_t rank = p.split > 1 ? cluster_ctarank() : 0u;
    const int cluster_id = blockIdx.x / p.split, nclusters = gridDim.x / p.split;
    const int64_t nrows = p.rows_dev ? *p.rows_dev : p.rows;
    const int ntiles = p.rows_dev ? (int)((nrows + kTileRows - 1) / kTileRows) : p.ntiles;

    if (threadIdx.x == 0) {
        mbar_init(&bars[PB_BFULL], 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bars[PB_XFULL + s], 1);
            mbar_init(&bars[PB_AFULL + s], 2);
            mbar_init(&bars[PB_AEMPTY + s], 1);
            mbar_init(&bars[PB_LFULL + s], 1);
            mbar_init(&bars[PB_LEMPTY + s], 8);
            mbar_init(&bars[PB_XCHG + s], kTileRows);
        }
        mbar_init(&bars[PB_DRAIN], 1);
        for (int q = 0; q < 4; ++q) {
            mbar_init(&bars[PB_HXFULL + q], 64);
            mbar_init(&bars[PB_HXFREE + q], 64);
        }
        misc[1] = 0u;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&misc[0], p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    if (p.split > 1) cluster_sync();   // peers' barriers initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = misc[0];

    const uint32_t bw_bytes = (uint32_t)p.ncta * 32u;   // one 16-column block of a B term
    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        prefetch_tmap(&tmX);
        prefetch_tmap(&tmB);
        mbar_arrive_expect_tx(&bars[PB_BFULL], 4u * p.nkb * bw_bytes);
        for (int t = 0; t < 4; ++t)
            for (int j = 0; j < p.nkb; ++j)
                tma_load_2d(smem + L.b + (t * p.nkb + j) * bw_bytes, &tmB, &bars[PB_BFULL], j * 16,
                            t * p.Kp + (int)rank * p.ncta);
        int last_use[2] = {-1, -1};
        int i = 0;
        for (int tile = cluster_id; tile < ntiles; tile += nclusters, ++i) {
            const int s = i % p.nstage, u = i / p.nstage;
            if (u > 0 && !mbar_wait(&bars[PB_AEMPTY + s], (u - 1) & 1, abort_flag, p.err)) break;
            uint8_t *ax = smem + L.a + s * L.a_stage;
            mbar_arrive_expect_tx(&bars[PB_XFULL + s], (uint32_t)p.nkb * kTileRows * 32u);
            for (int j = 0; j < p.nkb; ++j)
                tma_load_2d(ax + j * kTileRows * 32, &tmX, &bars[PB_XFULL + s], j * 16, tile * kTileRows);
            last_use[s] = u;
        }
        // wait (bounded, even when aborting) for this thread's copies still in flight
        for (int s = 0; s < 2; ++s) {
            if (last_use[s] < 0) continue;
            mbar_drain(&bars[PB_XFULL + s], last_use[s] & 1, 200000000ll);
        }
        mbar_drain(&bars[PB_BFULL], 0, 200000000ll);
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_bf16(kTileRows, p.ncta, false, false);
        const uint32_t sB = smem_u32(smem + L.b);
        bool ok = mbar_wait(&bars[PB_BFULL], 0, abort_flag, p.err);
        int i = 0;
        bool issued = false;
        for (int tile = cluster_id; ok && tile < ntiles; tile += nclusters, ++i) {
            const int s = i % p.nstage, b = i & 1;
            if (!mbar_wait(&bars[PB_AFULL + s], (i / p.nstage) & 1, abort_flag, p.err)) break;
            if (i >= 2 && !mbar_wait(&bars[PB_LEMPTY + b], ((i >> 1) - 1) & 1, abort_flag, p.err)) break;
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + L.a + s * L.a_stage);
            const uint32_t d = tmem + (uint32_t)(b * p.ncta);
            const uint32_t ablk = kTileRows * 32u;   // one 16-column block of an A operand
            uint32_t acc = 0;
            for (int j = 0; j < p.nkb; ++j) {
                const uint32_t ax = sA + (0 * p.nkb + j) * ablk;
                const uint32_t ah = sA + (1 * p.nkb + j) * ablk;
                const uint32_t al = sA + (2 * p.nkb + j) * ablk;
                const uint32_t bqh = sB + (0 * p.nkb + j) * bw_bytes;
                const uint32_t bql = sB + (1 * p.nkb + j) * bw_bytes;
                const uint32_t brh = sB + (2 * p.nkb + j) * bw_bytes;
                const uint32_t brl = sB + (3 * p.nkb + j) * bw_bytes;
                mma_bf16(d, sdesc_sw32(ax, 16, 256), sdesc_sw32(bqh, 16, 256), idesc, acc);
                acc = 1;
                mma_bf16(d, sdesc_sw32(ax, 16, 256), sdesc_sw32(bql, 16, 256), idesc, 1);
                mma_bf16(d, sdesc_sw32(ah, 16, 256), sdesc_sw32(brh, 16, 256), idesc, 1);
                mma_bf16(d, sdesc_sw32(ah, 16, 256), sdesc_sw32(brl, 16, 256), idesc, 1);
                mma_bf16(d, sdesc_sw32(al, 16, 256), sdesc_sw32(brh, 16, 256), idesc, 1);
            }
            mma_commit(&bars[PB_AEMPTY + s]);
            mma_commit(&bars[PB_LFULL + b]);
            issued = true;
        }
        if (issued) {   // every issued MMA has finished before TMEM is released
            mma_commit(&bars[PB_DRAIN]);
            mbar_drain(&bars[PB_DRAIN], 0, 2000000000ll);
        }
    } else if (warp == 2 || warp == 3) {
        // ---------------- x^2 hi/lo builders ----------------
        const int t = threadIdx.x - 64;
        const int chunks = p.nkb * kTileRows * 2;   // 16-byte chunks of the x blocks
        int i = 0;
        for (int tile = cluster_id; tile < ntiles; tile += nclusters, ++i) {
            const int s = i % p.nstage;
            if (!mbar_wait(&bars[PB_XFULL + s], (i / p.nstage) & 1, abort_flag, p.err)) break;
            uint8_t *sa = smem + L.a + s * L.a_stage;
            const uint32_t plane = (uint32_t)p.nkb * kTileRows * 32u;
            for (int c = t; c < chunks; c += 64) {
                const uint4 x = *reinterpret_cast<const uint4 *>(sa + c * 16);
                uint4 hi, lo;
                square_split(x, hi, lo);
                *reinterpret_cast<uint4 *>(sa + plane + c * 16) = hi;
                *reinterpret_cast<uint4 *>(sa + 2 * plane + c * 16) = lo;
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[PB_AFULL + s]);
        }
    } else if (warp >= 4) {
        // ---------------- softmax epilogue ----------------
        // Two warps per TMEM lane quadrant: warp 4+q and 8+q own rows
        // 32q..32q+31, each over half of the CTA's columns. Pass A reads L,
        // forms y = l log2(e) + c log2(e), keeps an online row max/sum with a
        // reference max per 32-column chunk and stores 2^(y - ref) back into
        // TMEM; the halves (and, with a component split, the peer CTA) combine
        // their (max, sum); pass B rescales each chunk and writes bf16.
        const int q = warp & 3, h = (warp - 4) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const int nh = p.ncta / 64;          // 32-column chunks per half (2, 3 or 4)
        const int c0 = h * nh;
        float2 *hx = reinterpret_cast<float2 *>(smem + L.hx);
        float2 *xbuf = reinterpret_cast<float2 *>(smem + L.xchg);
        const float *cl = p.cl2 + rank * p.ncta;
        int i = 0;
        for (int tile = cluster_id; tile < ntiles; tile += nclusters, ++i) {
            const int b = i & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[PB_LFULL + b], (i >> 1) & 1, abort_flag, p.err))) break;
            tc_fence_after();
            const uint32_t ta = lane_base + (uint32_t)(b * p.ncta);
            float m = -INFINITY, z = 0.f;
            float mc[4] = {0.f, 0.f, 0.f, 0.f};
            uint32_t ra[32], rb[32];
            // software pipeline: the next chunk's TMEM load is in flight while
            // this chunk is processed; this chunk's constants are requested
            // before waiting on its TMEM load
            tmem_ld32_issue(ta + c0 * 32, ra);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                if (cc >= nh) break;
                const int c = c0 + cc;
                uint32_t(&cur)[32] = (cc & 1) ? rb : ra;
                uint32_t(&nxt)[32] = (cc & 1) ? ra : rb;
                float4 ccur[8];
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) ccur[k4] = __ldg(reinterpret_cast<const float4 *>(cl + c * 32) + k4);
                tmem_ld_wait(cur);
                if (cc + 1 < nh) tmem_ld32_issue(ta + (c + 1) * 32, nxt);
                float y[32];
                float cm0 = -INFINITY, cm1 = -INFINITY;
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) {
                    y[4 * k4 + 0] = fmaf(__uint_as_float(cur[4 * k4 + 0]), kLog2e, ccur[k4].x);
                    y[4 * k4 + 1] = fmaf(__uint_as_float(cur[4 * k4 + 1]), kLog2e, ccur[k4].y);
                    y[4 * k4 + 2] = fmaf(__uint_as_float(cur[4 * k4 + 2]), kLog2e, ccur[k4].z);
                    y[4 * k4 + 3] = fmaf(__uint_as_float(cur[4 * k4 + 3]), kLog2e, ccur[k4].w);
                    cm0 = fmaxf(cm0, fmaxf(y[4 * k4 + 0], y[4 * k4 + 1]));
                    cm1 = fmaxf(cm1, fmaxf(y[4 * k4 + 2], y[4 * k4 + 3]));
                }
                const float mn = fmaxf(m, fmaxf(cm0, cm1));
                const float mref = (mn == -INFINITY) ? 0.f : mn;
                float z0 = z * ex2_approx(m - mref), z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
                for (int k = 0; k < 32; k += 4) {
                    const float e0 = ex2_approx(y[k + 0] - mref), e1 = ex2_approx(y[k + 1] - mref);
                    const float e2 = ex2_approx(y[k + 2] - mref), e3 = ex2_approx(y[k + 3] - mref);
                    z0 += e0;
                    z1 += e1;
                    z2 += e2;
                    z3 += e3;
                    cur[k + 0] = __float_as_uint(e0);
                    cur[k + 1] = __float_as_uint(e1);
                    cur[k + 2] = __float_as_uint(e2);
                    cur[k + 3] = __float_as_uint(e3);
                }
                z = (z0 + z1) + (z2 + z3);
                tmem_st32_u(ta + c * 32, cur);
                mc[cc] = mref;
                m = mn;
            }
            // combine the two column halves of the row (bounded handshakes:
            // the partner warp has read the previous tile's value before this
            // one is written, and has written this tile's before it is read)
            if (i > 0 && !__all_sync(0xffffffffu, mbar_wait(&bars[PB_HXFREE + q], (i - 1) & 1, abort_flag, p.err)))
                break;
            hx[h * kTileRows + r] = make_float2(m, z);
            mbar_arrive(&bars[PB_HXFULL + q]);
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[PB_HXFULL + q], i & 1, abort_flag, p.err))) break;
            const float2 o = hx[(h ^ 1) * kTileRows + r];
            mbar_arrive(&bars[PB_HXFREE + q]);
            float M = fmaxf(m, o.x);
            float Mref = (M == -INFINITY) ? 0.f : M;
            float Z = z * ex2_approx(m - Mref) + o.y * ex2_approx(o.x - Mref);
            if (p.split > 1) {
                const uint32_t peer = rank ^ 1u;
                if (h == 0) {
                    st_cluster_f32x2(mapa(smem_u32(&xbuf[b * kTileRows + r]), peer), M, Z);
                    mbar_arrive_remote(mapa(smem_u32(&bars[PB_XCHG + b]), peer));
                }
                if (!__all_sync(0xffffffffu, mbar_wait(&bars[PB_XCHG + b], (i >> 1) & 1, abort_flag, p.err, true)))
                    break;
                const float2 po = xbuf[b * kTileRows + r];
                const float M2 = fmaxf(M, po.x);
                const float M2ref = (M2 == -INFINITY) ? 0.f : M2;
                Z = Z * ex2_approx(M - M2ref) + po.y * ex2_approx(po.x - M2ref);
                M = M2;
                Mref = M2ref;
            }
            const float inv = 1.0f / Z;
            // pass B: normalised posteriors -> bf16 global (next chunk's load in flight)
            const int64_t row = (int64_t)tile * kTileRows + r;
            uint16_t *g = p.gamma + row * p.Kp + rank * p.ncta;
            tmem_ld32_issue(ta + c0 * 32, ra);
            tmem_ld_wait(ra);
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                if (cc >= nh) break;
                const int c = c0 + cc;
                uint32_t(&cur)[32] = (cc & 1) ? rb : ra;
                uint32_t(&nxt)[32] = (cc & 1) ? ra : rb;
                if (cc + 1 < nh) tmem_ld32_issue(ta + (c + 1) * 32, nxt);
                const float sc = ex2_approx(mc[cc] - Mref) * inv;
                if (row < nrows) {   // 64 bytes of the row: two full 32-byte sectors
                    uint32_t pk[16];
#pragma unroll
                    for (int k = 0; k < 16; ++k)
                        pk[k] = pack_bf16x2(__uint_as_float(cur[2 * k]) * sc, __uint_as_float(cur[2 * k + 1]) * sc);
                    st_global_v8(g + c * 32, pk);
                    st_global_v8(g + c * 32 + 16, pk + 8);
                }
                if (cc + 1 < nh) tmem_ld_wait(nxt);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[PB_LEMPTY + b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (p.split > 1) cluster_sync();   // no remote access into a CTA that has exited
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}

// ---- statistics -----------------------------------------------------------------------
struct StatArgs {
    int nkb;       // D16 / 16
    int D;
    int Kp;
    int sc;        // components per CTA (128 or 256)
    int ny;        // 3*D16 + 16 columns of Y
    int P;         // 3*D16 + 1 floats per component in a slot
    uint32_t tmem_cols;
    const StatUnit *units;
    const int2 *cta_units;   // per CTA: (first unit, number of units)
    float *part;
    uint32_t *err;
};

struct StatSmem {
    uint32_t g_stage, y_stage, stage, bars, misc, total;
};
__host__ __device__ inline StatSmem stat_smem(int nkb, int sc) {
    StatSmem s;
    s.g_stage = (uint32_t)(sc / 16) * kStatRows * 32u;
    s.y_stage = (uint32_t)(3 * nkb + 1) * kStatRows * 32u;
    s.stage = s.g_stage + s.y_stage;
    s.bars = kStatStages * s.stage;
    s.misc = s.bars + 16u * 8u;
    s.total = s.misc + 16u;
    return s;
}
enum { SB_FULL = 0, SB_READY = 3, SB_EMPTY = 6, SB_DONE = 9, SB_TEMPTY = 10, SB_DRAIN = 11 };

// Persistent: CTA (blockIdx.x, blockIdx.y) walks its units (row segments of
// one frame, contiguous in the packed rows) through one continuous ring of
// 64-row stages for the component group blockIdx.y; after each unit the
// accumulator is flushed from TMEM to the unit's slot.
__global__ void __launch_bounds__(kThreads, 1)
bf16_stats_kernel(const __grid_constant__ CUtensorMap tmG, const __grid_constant__ CUtensorMap tmX, StatArgs p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const StatSmem L = stat_smem(p.nkb, p.sc);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);
    volatile uint32_t *abort_flag = misc + 1;
    if ((smem_u32(smem) & 1023u) != 0u) {
        if (threadIdx.x == 0) atomicOr(p.err, kErrAlign);
        return;
    }
    const int2 cu = p.cta_units[blockIdx.x];
    const int kc0 = blockIdx.y * p.sc;
    const int nchunk = p.sc / 128;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStatStages; ++s) {
            mbar_init(&bars[SB_FULL + s], 1);
            mbar_init(&bars[SB_READY + s], 6);
            mbar_init(&bars[SB_EMPTY + s], 1);
        }
        mbar_init(&bars[SB_DONE], 1);
        mbar_init(&bars[SB_TEMPTY], 4);
        mbar_init(&bars[SB_DRAIN], 1);
        misc[1] = 0u;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&misc[0], p.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = misc[0];
    const uint32_t blk = kStatRows * 32u;   // bytes of one 16-column block

    if (warp == 0 && lane == 0) {
        // ---------------- TMA producer ----------------
        prefetch_tmap(&tmG);
        prefetch_tmap(&tmX);
        int last_use[kStatStages] = {-1, -1, -1};
        int gs = 0;
        bool ok = true;
        for (int ui = 0; ok && ui < cu.y; ++ui) {
            const StatUnit u = p.units[cu.x + ui];
            const int nit = (u.nrows + kStatRows - 1) / kStatRows;
            for (int it = 0; it < nit; ++it, ++gs) {
                const int s = gs % kStatStages, use = gs / kStatStages;
                if (use > 0 && !mbar_wait(&bars[SB_EMPTY + s], (use - 1) & 1, abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                uint8_t *sg = smem + s * L.stage;
                uint8_t *sy = sg + L.g_stage;
                const int y = (int)(u.row0 + (int64_t)it * kStatRows);
                mbar_arrive_expect_tx(&bars[SB_FULL + s], (uint32_t)(p.sc / 16 + p.nkb) * blk);
                for (int cb = 0; cb < p.sc / 64; ++cb)   // 64 components x 64 rows, 128-byte rows
                    tma_load_2d(sg + cb * kGBlk, &tmG, &bars[SB_FULL + s], kc0 + cb * 64, y);
                for (int j = 0; j < p.nkb; ++j) tma_load_2d(sy + j * blk, &tmX, &bars[SB_FULL + s], j * 16, y);
                last_use[s] = use;
            }
        }
        for (int s = 0; s < kStatStages; ++s) {
            if (last_use[s] < 0) continue;
            mbar_drain(&bars[SB_FULL + s], last_use[s] & 1, 200000000ll);
        }
    } else if (warp == 1 && lane == 0) {
        // ---------------- MMA issuer ----------------
        const uint32_t idesc = idesc_bf16(128, p.ny, true, true);
        bool issued = false, ok = true;
        int gs = 0;
        for (int ui = 0; ok && ui < cu.y; ++ui) {
            const StatUnit u = p.units[cu.x + ui];
            const int nit = (u.nrows + kStatRows - 1) / kStatRows;
            if (ui > 0) {   // the epilogue has read the previous unit's accumulator
                if (!mbar_wait(&bars[SB_TEMPTY], (ui - 1) & 1, abort_flag, p.err)) break;
                tc_fence_after();
            }
            for (int it = 0; it < nit; ++it, ++gs) {
                const int s = gs % kStatStages;
                if (!mbar_wait(&bars[SB_READY + s], (gs / kStatStages) & 1, abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t sg = smem_u32(smem + s * L.stage);
                const uint32_t sy = sg + L.g_stage;
                for (int q = 0; q < kStatRows / 16; ++q) {
                    for (int c = 0; c < nchunk; ++c) {
                        // gamma^T, MN-major, 128-byte swizzle: 64-component blocks kGBlk
                        // apart, 8-row groups 1024 B apart, 16 rows per K step
                        const uint64_t a = sdesc_sw128(sg + c * 2 * kGBlk + q * 2048, kGBlk, 1024);
                        const uint64_t b = sdesc_sw32(sy + q * 512, blk, 256);
                        mma_bf16(tmem + (uint32_t)(c * p.ny), a, b, idesc, (it > 0 || q > 0) ? 1u : 0u);
                    }
                }
                mma_commit(&bars[SB_EMPTY + s]);
                issued = true;
            }
            if (ok) mma_commit(&bars[SB_DONE]);
        }
        if (issued) {   // every issued MMA has finished before TMEM is released
            mma_commit(&bars[SB_DRAIN]);
            mbar_drain(&bars[SB_DRAIN], 0, 2000000000ll);
        }
    } else if (warp >= 2) {
        // ---------------- Y builders (warps 2-7); warps 4-7 also flush TMEM ----------------
        const int t = threadIdx.x - 64;          // 0..191
        const int xchunks = p.nkb * kStatRows * 2;
        const uint32_t plane = (uint32_t)p.nkb * blk;
        int gs = 0;
        bool ok = true;
        for (int ui = 0; ok && ui < cu.y; ++ui) {
            const StatUnit u = p.units[cu.x + ui];
            const int nit = (u.nrows + kStatRows - 1) / kStatRows;
            for (int it = 0; it < nit; ++it, ++gs) {
                const int s = gs % kStatStages;
                if (!mbar_wait(&bars[SB_FULL + s], (gs / kStatStages) & 1, abort_flag, p.err)) {
                    ok = false;
                    break;
                }
                uint8_t *sy = smem + s * L.stage + L.g_stage;
                const int valid = min(kStatRows, u.nrows - it * kStatRows);
                for (int c = t; c < xchunks; c += 192) {
                    const int row = (c >> 1) % kStatRows;   // 32-byte rows; the swizzle stays inside a row
                    uint4 x = *reinterpret_cast<const uint4 *>(sy + c * 16);
                    uint4 hi, lo;
                    if (row < valid) {
                        square_split(x, hi, lo);
                    } else {
                        x = make_uint4(0, 0, 0, 0);
                        hi = x;
                        lo = x;
                        *reinterpret_cast<uint4 *>(sy + c * 16) = x;
                    }
                    *reinterpret_cast<uint4 *>(sy + plane + c * 16) = hi;
                    *reinterpret_cast<uint4 *>(sy + 2 * plane + c * 16) = lo;
                }
                for (int c = t; c < kStatRows * 2; c += 192) {
                    const int row = c >> 1;
                    const uint32_t one = row < valid ? 0x3F803F80u : 0u;   // bf16 1.0 pairs
                    *reinterpret_cast<uint4 *>(sy + 3 * plane + c * 16) = make_uint4(one, one, one, one);
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[SB_READY + s]);
            }
            if (!ok || warp < 4) continue;
            // flush this unit's accumulator: TMEM -> slot part[slot][j][Kp]
            const int q = warp & 3;
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[SB_DONE], ui & 1, abort_flag, p.err))) {
                ok = false;
                break;
            }
            tc_fence_after();
            // slot columns follow the TMEM columns: [S1 | S2hi | S2lo] blocks of
            // D16, then S0 (the first ones column), so the flush is a copy; two
            // 32-column TMEM loads are in flight at a time
            for (int c = 0; c < nchunk; ++c) {
                const int k = kc0 + c * 128 + q * 32 + lane;
                float *dst = p.part + (size_t)u.slot * p.Kp * p.P + k;
                const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(c * p.ny);
                for (int n0 = 0; n0 < p.P; n0 += 64) {
                    uint32_t va[32], vb[32];
                    tmem_ld32_issue(ta + n0, va);
                    tmem_ld32_issue(ta + n0 + 32, vb);
                    tmem_ld_wait(va);
                    tmem_ld_wait(vb);
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        if (n0 + e < p.P) dst[(size_t)(n0 + e) * p.Kp] = __uint_as_float(va[e]);
                        if (n0 + 32 + e < p.P) dst[(size_t)(n0 + 32 + e) * p.Kp] = __uint_as_float(vb[e]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[SB_TEMPTY]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, p.tmem_cols);
    }
}

// FP32 rows -> bf16 rows of pitch ldx, zero padded past D.
__global__ void convert_kernel(const float *__restrict__ X, int64_t rows, int D, int ldx, uint16_t *__restrict__ Xb) {
    const int64_t n = rows * ldx;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / ldx;
        const int d = (int)(i - r * ldx);
        const float v = d < D ? X[r * D + d] : 0.f;
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        Xb[i] = *reinterpret_cast<uint16_t *>(&h);
    }
}

// ---- host side ----------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

cudaError_t get_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    return g_encode ? cudaSuccess : cudaErrorNotSupported;
}

// 2D bf16 tensor map: `cols` x `rows` with row pitch `pitch_elems`, box
// 16 x box_rows with the 32-byte swizzle, or 64 x box_rows with the 128-byte
// swizzle when wide; zero fill out of bounds.
bool make_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t pitch_elems, uint32_t box_rows,
              bool wide = false) {
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {pitch_elems * 2};
    cuuint32_t box[2] = {wide ? 64u : 16u, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, wide ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_32B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

uint32_t pow2_cols(int n) {
    uint32_t c = 32;
    while ((int)c < n) c <<= 1;
    return c;
}

struct BfCfg {
    int split, ncta, nstage, sc, ny;
    size_t post_smem, stat_smem;
};

bool bf16_config(const fv_gmm *g, BfCfg &c) {
    const int nkb = round_up(g->D, 16) / 16;
    c.split = g->Kp > 256 ? 2 : 1;
    c.ncta = g->Kp / c.split;
    c.nstage = 2;
    int maxsmem = 232448;
    if (post_smem(nkb, c.ncta, 2, c.split).total > (uint32_t)maxsmem) c.nstage = 1;
    c.post_smem = post_smem(nkb, c.ncta, c.nstage, c.split).total;
    c.sc = (g->Kp % 256 == 0) ? 256 : 128;
    c.ny = 3 * nkb * 16 + 16;
    c.stat_smem = stat_smem(nkb, c.sc).total;
    return c.post_smem <= (size_t)maxsmem && c.stat_smem <= (size_t)maxsmem && c.ncta % 64 == 0 && c.ncta <= 256 &&
           c.ny <= 256;
}

}  // namespace

int bf16_stat_ctas(const fv_gmm *g, int64_t rows, int sms) {
    // one persistent CTA per SM per component group, each with at least 512
    // rows (a slot is K x (3D+1) floats; shorter shares would move more slot
    // bytes than posterior bytes)
    const int sc = (g->Kp % 256 == 0) ? 256 : 128;
    const int groups = g->Kp / sc;
    const int per_group = std::max(1, sms / groups);
    const int64_t by_rows = std::max<int64_t>(1, rows / 512);
    return (int)std::max<int64_t>(1, std::min<int64_t>(per_group, by_rows));
}

cudaError_t launch_bf16_convert(const fv_gmm *g, const float *X, int64_t rows, uint16_t *Xb, cudaStream_t st) {
    if (rows <= 0) return cudaSuccess;
    const int64_t n = rows * g->Dp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    {
        KernelTimer kt_("bf16_convert", st);
        convert_kernel<<<blocks, 256, 0, st>>>(X, rows, g->D, g->Dp, Xb);
    }
    return cudaGetLastError();
}

int run_bf16_encoder(const fv_gmm *g, const uint16_t *Xb, int64_t ldx, int64_t rows, uint16_t *gamma,
                     const StatUnit *units, const int2 *cta_units, int n_ctas, float *part, int P, int sms,
                     uint32_t *err, cudaStream_t st, const int64_t *rows_dev) {
    if (rows <= 0 || n_ctas <= 0) return FV_OK;
    if (get_encoder() != cudaSuccess) return fail(FV_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    BfCfg c;
    if (!bf16_config(g, c)) return fail(FV_ERR_UNSUPPORTED, "BF16 form: shape does not fit the kernels' shared memory");
    const int nkb = round_up(g->D, 16) / 16;
    if (rows > (int64_t)INT32_MAX - 256) return fail(FV_ERR_UNSUPPORTED, "BF16 form: too many rows for one call");

    CUtensorMap tmX128, tmX64, tmB, tmG;
    if (!make_map(&tmX128, Xb, (uint64_t)g->D, (uint64_t)rows, (uint64_t)ldx, kTileRows) ||
        !make_map(&tmX64, Xb, (uint64_t)g->D, (uint64_t)rows, (uint64_t)ldx, kStatRows) ||
        !make_map(&tmB, g->dev.bimg, (uint64_t)nkb * 16, (uint64_t)4 * g->Kp, (uint64_t)nkb * 16, (uint32_t)c.ncta) ||
        !make_map(&tmG, gamma, (uint64_t)g->Kp, (uint64_t)rows, (uint64_t)g->Kp, kStatRows, true))
        return fail(FV_ERR_CUDA, "cuTensorMapEncodeTiled failed");

    // posteriors: persistent clusters over 128-row tiles
    PostArgs pa;
    pa.rows = rows;
    pa.ntiles = (int)((rows + kTileRows - 1) / kTileRows);
    pa.rows_dev = rows_dev;   // rows is then the buffers' capacity
    pa.nkb = nkb;
    pa.Kp = g->Kp;
    pa.ncta = c.ncta;
    pa.split = c.split;
    pa.nstage = c.nstage;
    pa.tmem_cols = pow2_cols(2 * c.ncta);
    pa.cl2 = g->dev.cl2;
    pa.gamma = gamma;
    pa.err = err;
    cudaError_t e = cudaFuncSetAttribute(bf16_posteriors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)c.post_smem);
    if (e != cudaSuccess) return cuda_fail(e, "bf16 posteriors: smem attribute");
    const int nclusters = rows_dev ? std::max(1, sms / c.split) : std::max(1, std::min(pa.ntiles, sms / c.split));
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3((unsigned)(nclusters * c.split));
    cfg.blockDim = dim3(kPostThreads);
    cfg.dynamicSmemBytes = c.post_smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.split;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    {
        KernelTimer kt_("bf16_posteriors", st);
        e = cudaLaunchKernelEx(&cfg, bf16_posteriors_kernel, tmX128, tmB, pa);
    }
    if (e != cudaSuccess) return cuda_fail(e, "bf16 posteriors launch");

    // statistics: persistent CTAs over balanced row shares x component groups
    StatArgs sa;
    sa.nkb = nkb;
    sa.D = g->D;
    sa.Kp = g->Kp;
    sa.sc = c.sc;
    sa.ny = c.ny;
    sa.P = P;
    sa.tmem_cols = pow2_cols((c.sc / 128) * c.ny);
    sa.units = units;
    sa.cta_units = cta_units;
    sa.part = part;
    sa.err = err;
    e = cudaFuncSetAttribute(bf16_stats_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.stat_smem);
    if (e != cudaSuccess) return cuda_fail(e, "bf16 statistics: smem attribute");
    dim3 grid((unsigned)n_ctas, (unsigned)(g->Kp / c.sc));
    {
        KernelTimer kt_("bf16_stats", st);
        bf16_stats_kernel<<<grid, kThreads, c.stat_smem, st>>>(tmG, tmX64, sa);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bf16 statistics launch");
    return FV_OK;
}

}  // namespace fv
