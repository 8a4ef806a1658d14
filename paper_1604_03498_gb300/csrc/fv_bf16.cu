// BF16 precision form of the encoder on the 5th-generation tensor cores
// (tcgen05 MMA with TMEM accumulators, TMA-fed shared-memory operands), as
// one fused kernel: the posteriors never leave the SM.
//
// Per 128-row tile, each CTA of a cluster owns 128 components and runs
//
// 1. the log-likelihood GEMM (the distance/posterior step of Algorithm 1;
//    the paper's Phase 1, Algorithm 2, its most expensive part):
//      l_ik = c_k + sum_d x_id Q_kd + sum_d x_id^2 R_kd,
//      Q = mu/sigma^2, R = -1/(2 sigma^2), c_k = log w_k - 1/2 sum log sigma^2
//      - 1/2 sum mu^2/sigma^2 (FP64 on the device, once per GMM).
//    x is bfloat16 (exact), Q and R are split into bf16 hi + lo parts, and
//    x^2 (16 significant bits for a bf16 x) into hi + lo, so five products
//      x Q_hi + x Q_lo + x2_hi R_hi + x2_hi R_lo + x2_lo R_hi
//    accumulate in FP32 in TMEM and undo the cancellation between
//    x^2/sigma^2 and 2 x mu/sigma^2;
// 2. the posteriors (Eq. 2): per row a log-sum-exp over the CTA's 128
//    components in TMEM, combined over the cluster's CTAs through
//    distributed shared memory, then gamma written to shared memory as
//    bfloat16, laid out as the next GEMM's A operand;
// 3. the statistics GEMM (Algorithm 1 second loop; Phase 2, Algorithm 3):
//      [S1 | S2hi | S2lo | S0] += gamma^T [X | X2hi | X2lo | 1]
//    with the tile's own shared-memory X planes as the B operand; the
//    accumulator stays in TMEM for a whole row share of one frame (a unit)
//    and is then centred (A = S1 - mu S0, B = S2 - 2 mu S1 + mu^2 S0) as
//    it is written to the unit's statistics slot (the paper's per-block
//    copies of the statistics).
// The finalise kernels add the slots, scale and normalise.
//
// FV_PREC_BF16X2: the posteriors enter the statistics GEMM as a bf16 hi + lo
// pair (gamma = hi + lo to about 2^-16, two MMAs per K step into the same
// accumulator), so the statistics carry the posteriors' FP32 values instead
// of their bfloat16 rounding (2^-9 relative). That rounding is the largest
// error of the precision form, and the improved-FV scaling 1/(N sqrt(w))
// magnifies it for components of very small prior w. The hi + lo pair of a
// tile goes through the plain form's 32 KB gamma^T buffer in two 64-row
// halves: lane quadrants 0-1 write rows 0-63, the statistics GEMM reads them,
// then quadrants 2-3 write rows 64-127 (each half with its own full / free
// barriers), so the form keeps the plain form's Y stages (two at D = 64).
//
// Early termination (Sec. 3.3, Algorithm 5), as block sparsity of the
// statistics GEMM: with a posterior threshold tau > 0 the softmax writes
// posteriors not above tau as zeros and marks each 16-row K step of the
// gamma^T tile that still holds a non-zero posterior; the statistics issuer
// skips the MMAs of unmarked K steps (a 16-row x 128-component block of
// posteriors all at or below tau), which add nothing. tau = 0 is the exact
// encoding and issues every MMA.
//
// TMEM (512 columns): two log-likelihood buffers of 128 columns (the next
// tile's GEMM overlaps this tile's softmax) and the statistics accumulator.
// Shared memory: the GMM operand [Q_hi | Q_lo | R_hi | R_lo] for the CTA's
// components, resident; a TMA landing buffer for the next tile's x (its
// load is not held up by the stage still in use); one or two stages of the
// tile's Y planes; the gamma^T tile; the cluster exchange buffers. Operand layout: blocks of 16
// bf16 columns, each a [rows][16] array of 32-byte rows with the 32-byte
// swizzle (TMA writes it; read K-major by the first GEMM and MN-major by the
// second); gamma^T in 64-component blocks with the 128-byte swizzle.
//
// Warp roles (16 warps): 0 TMA loads and the log-likelihood MMAs, 1 the
// statistics MMAs, 2-3 and 12-15 build each tile's Y planes (x taken from the
// TMA landing buffer into registers, x^2 split, ones) while the softmax of
// the previous tile runs, 4-11 softmax (two warps per TMEM lane quadrant, one
// per 64-component half, on every tile).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <tuple>

#include "fv_bf16.h"
#include "fv_sm100.cuh"

namespace fv {

using namespace sm100;

namespace {

constexpr int kThreads = 512;          // 16 warps
constexpr int kRows = 128;             // row tile: M of the first GEMM, K of the second
constexpr int kComps = 128;            // components per CTA: N of the first GEMM, M of the second
constexpr uint32_t kBlk = kRows * 32u;           // one [128][16] bf16 block with 32-byte rows (4 KB)
constexpr uint32_t kGHalf = 64u * kRows * 2u;    // 64 components x 128 rows of gamma^T (16 KB)
constexpr uint32_t kSub = kGHalf / 2u;           // 64 components x 64 rows (BF16X2 halves, 8 KB)
constexpr uint32_t kStatCol = 2u * kComps;       // first TMEM column of the statistics accumulator
constexpr uint32_t kTmemCols = 512;
constexpr int kMaxSmem = 232448;
constexpr float kLog2e = 1.4426950408889634f;

// ---- small device helpers ---------------------------------------------------------
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// x (8 bf16 in a uint4) -> x^2 split into bf16 hi and lo parts, exactly:
// hi = RN(x*x) by a bf16x2 multiply, lo = RN(x*x - hi) by a bf16x2 fused
// multiply-add (x*x has 16 significant bits, so x*x - hi fits a bf16 and
// hi + lo == x^2).
__device__ __forceinline__ void square_split(const uint4 &x, uint4 &hi, uint4 &lo) {
    const uint32_t w[4] = {x.x, x.y, x.z, x.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 v = *reinterpret_cast<const __nv_bfloat162 *>(&w[i]);
        const __nv_bfloat162 vh = __hmul2(v, v);
        const __nv_bfloat162 vl = __hfma2(v, v, __hneg2(vh));
        h[i] = *reinterpret_cast<const uint32_t *>(&vh);
        l[i] = *reinterpret_cast<const uint32_t *>(&vl);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---- fused encoder kernel -------------------------------------------------------------
struct EncArgs {
    int nkb;        // D16 / 16
    int Kp;
    int S;          // CTAs per cluster (Kp / 128), each owning 128 components
    int nstage;     // Y-plane stages (1 or 2)
    int ny;         // 3*D16 + 16 columns of Y
    int P;          // 2D + 1 floats per component in a slot: [A | B | S0], centred
    int D;
    const float *mu_t;        // [D][Kp] means (FP32), for the centring of the slot write-out
    const float *cl2;         // [Kp] log-constant times log2(e) (-inf on padding)
    const StatUnit *units;    // row ranges of one frame each
    const int2 *cl_units;     // per cluster: (first unit, number of units)
    float *part;              // [slot][P][Kp] statistics slots
    uint32_t *err;
    int glo;                  // 1: posteriors as bf16 hi + lo (FV_PREC_BF16X2)
    float tau;                // posterior threshold (0: exact, every MMA issued)
    unsigned long long *skip_count;   // [skipped, issued + skipped] statistics K steps (nullable)
};

struct EncSmem {
    // byte offsets from the (1024-aligned) dynamic shared-memory base
    uint32_t b, xr, y, y_stage, g, hx, xchg, cl, bars, misc, flags, total;
};

__host__ __device__ inline EncSmem enc_smem(int nkb, int S, int nstage, bool glo = false) {
    EncSmem s;
    uint32_t off = 0;
    s.b = off;                                   // [Qh | Ql | Rh | Rl] x nkb blocks of 128 components
    off += 4u * nkb * kBlk;
    s.xr = off;                                  // TMA landing buffer of the next tile's x
    off += nkb * kBlk;
    s.y_stage = (3u * nkb + 1u) * kBlk;          // [X | X2hi | X2lo | 1] blocks of 128 rows
    s.y = off;
    off += nstage * s.y_stage;
    s.g = off;                                   // gamma^T: two 64-component halves (BF16X2: hi | lo of 64 rows)
    off += 2u * kGHalf;
    s.hx = off;                                  // (max, sum) per row of each column half
    off += 2u * kRows * 8u;
    s.xchg = off;                                // (max, sum) per row: 2 slots x S ranks
    off += S > 1 ? 2u * S * kRows * 8u : 0u;
    s.cl = off;                                  // the CTA's 128 log-constants
    off += kComps * 4u;
    s.bars = off;
    off += 32u * 8u;
    s.misc = off;
    off += 16u;
    s.flags = off;                               // [2 halves][8 K steps] non-zero posterior marks
    off += 16u;
    s.total = off;
    return s;
}

// Barrier indices. A parity wait cannot tell phase n from phase n + 2, so no
// thread may skip a phase of a barrier it waits on; every waiter below waits
// on every phase (barriers that complete per tile come in pairs indexed by
// the tile's parity where that keeps two tiles' waits apart).
enum {
    EB_BFULL = 0,     // GMM operand loaded
    EB_XRFULL = 1,    // [2] x landing buffer loaded (by tile parity)
    EB_DRAIN2 = 3,    // the statistics issuer's MMAs done
    EB_AFULL = 4,     // [2] Y planes of a stage built
    EB_STFREE = 6,    // [2] both GEMMs done with a tile's stage (by tile parity)
    EB_LFULL = 8,     // [2] log-likelihoods of a TMEM buffer ready
    EB_LEMPTY = 10,   // [2] softmax done with a TMEM buffer
    EB_GFULL = 12,    // gamma^T tile written
    EB_GFREE = 13,    // statistics GEMM done with gamma^T
    EB_SDONE = 14,    // a unit's statistics complete in TMEM
    EB_TEMPTY = 15,   // statistics accumulator written out
    EB_DRAIN = 16,
    EB_XCHG = 17,     // [2] peers' (max, sum) of a tile arrived, by bytes (slot = tile parity)
    EB_HXFULL = 19,   // [4] both column halves of a quadrant's rows have written (max, sum)
    EB_HXFREE = 23,   // [4] both halves have read them
    EB_XRFREE = 27,   // the builders hold a tile's x in registers: the landing buffer may refill
    EB_GFULL2 = 28,   // BF16X2: gamma^T hi + lo of rows 64-127 written (EB_GFULL: rows 0-63)
    EB_GFREE2 = 29,   // BF16X2: statistics GEMM done with rows 64-127 (EB_GFREE: rows 0-63)
    EB_NBARS = 30
};

// Y planes of one tile, built in two steps so that only the stores wait for
// the stage to come free. x_load reads thread t's 16-byte chunks of the x
// block from the landing buffer into registers (every supported D fits:
// 3*D16 + 16 <= 256 columns gives at most 5 column blocks, 1280 chunks, i.e.
// kHold chunks per builder thread); y_store writes x, the hi and lo halves of
// x^2 and the ones block. Rows past the unit's end (the next frame, or zero
// fill) are zeroed in every plane, so they add nothing to the statistics
// whatever their posteriors.
constexpr int kBuilders = 192;
constexpr int kHold = (5 * kRows * 2 + kBuilders - 1) / kBuilders;

__device__ __forceinline__ void x_load(uint4 (&x)[kHold], const uint8_t *xr, int nkb, int t) {
    const int chunks = nkb * kRows * 2;
#pragma unroll
    for (int u = 0; u < kHold; ++u) {
        const int c = t + u * kBuilders;
        if (c < chunks) x[u] = *reinterpret_cast<const uint4 *>(xr + c * 16);
    }
}

__device__ __forceinline__ void y_store(uint8_t *sy, uint4 (&x)[kHold], uint32_t plane, int nkb, int valid, int t) {
    const int chunks = nkb * kRows * 2;
#pragma unroll
    for (int u = 0; u < kHold; ++u) {
        const int c = t + u * kBuilders;
        if (c >= chunks) break;
        const int row = (c >> 1) & (kRows - 1);   // 32-byte rows; the swizzle stays inside a row
        uint4 hi, lo;
        if (row < valid) {
            square_split(x[u], hi, lo);
        } else {
            x[u] = make_uint4(0u, 0u, 0u, 0u);
            hi = x[u];
            lo = x[u];
        }
        *reinterpret_cast<uint4 *>(sy + c * 16) = x[u];
        *reinterpret_cast<uint4 *>(sy + plane + c * 16) = hi;
        *reinterpret_cast<uint4 *>(sy + 2 * plane + c * 16) = lo;
    }
    for (int c = t; c < kRows * 2; c += kBuilders) {
        const uint32_t one = (c >> 1) < valid ? 0x3F803F80u : 0u;   // bf16 1.0 pairs
        *reinterpret_cast<uint4 *>(sy + 3 * plane + c * 16) = make_uint4(one, one, one, one);
    }
}

// A softmax warp's share of a unit's statistics, TMEM -> slot, centred on the
// way. For the lane's component (mean mu_d in dimension d) and each dimension
// of the warp's 32-dimension chunks (h, h + 2, ...):
//   A = S1 - mu S0,   B = S2 - 2 mu S1 + mu^2 S0 = fma(-mu, A, fma(-mu, S1, S2hi) + S2lo)
// (the FMA order keeps each rounding relative to the centred quantities, and
// centring is linear, so the shares' A and B add up to the frame's). A slot
// then holds [A (D) | B (D) | S0] like the FP32 form's: 2D + 1 floats per
// component instead of the raw moments' 3 D16 + 1. The first chunk's 32 means
// are requested before the wait for the unit's last statistics MMA (SDONE,
// parity `par`), so their latency hides behind it; each 16-dimension block of A and B goes through the
// warp's own 4 KB of the gamma^T buffer (its pass-B rows in the plain form;
// the buffer is free of posteriors once the unit's last statistics MMA is
// done, and BF16X2's next pass B waits for this write-out) as
// [16 A rows + 16 B rows][32 c], and each lane then stores 16 bytes
// (4 components) of one row, so one warp store covers four 128-byte row
// pieces. Not inlined: it runs once per unit, and keeping it out of the
// kernel body leaves the tile loop's code as it is.
// Returns false when the wait gave up (the kernel is aborting).
__device__ __noinline__ bool write_stats(uint64_t *sdone, uint32_t par, volatile uint32_t *abort, uint32_t *err,
                                         uint32_t ts, float *stg, float *dst0, const float *__restrict__ mu_t, int h,
                                         int D, int D16, int Kp, int k, int lane) {
    float mu[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) mu[e] = h * 32 + e < D ? mu_t[(size_t)(h * 32 + e) * Kp + k] : 0.f;
    if (!__all_sync(0xffffffffu, mbar_wait(sdone, par, abort, err))) return false;
    tc_fence_after();
    const float S0 = tmem_ld1(ts + 3 * D16);
    if (h == 0) dst0[(size_t)(2 * D) * Kp + lane] = S0;
    for (int d0 = h * 32; d0 < D; d0 += 64) {
        if (d0 != h * 32) {
#pragma unroll
            for (int e = 0; e < 32; ++e) mu[e] = d0 + e < D ? mu_t[(size_t)(d0 + e) * Kp + k] : 0.f;
        }
#pragma unroll
        for (int b16 = 0; b16 < 32; b16 += 16) {
            if (d0 + b16 >= D) break;   // d0 + b16 + 16 <= D16
            const uint32_t c = ts + (uint32_t)(d0 + b16);
            uint32_t s1a[8], s2ha[8], s2la[8], s1b[8], s2hb[8], s2lb[8];
            tmem_ld8_issue(c, s1a);
            tmem_ld8_issue(c + D16, s2ha);
            tmem_ld8_issue(c + 2 * D16, s2la);
            tmem_ld8_issue(c + 8, s1b);
            tmem_ld8_issue(c + D16 + 8, s2hb);
            tmem_ld8_issue(c + 2 * D16 + 8, s2lb);
            tmem_ld8_wait3(s1a, s2ha, s2la);
            tmem_ld8_wait3(s1b, s2hb, s2lb);
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float m = mu[b16 + e];
                const float x1 = __uint_as_float(e < 8 ? s1a[e] : s1b[e - 8]);
                const float x2h = __uint_as_float(e < 8 ? s2ha[e] : s2hb[e - 8]);
                const float x2l = __uint_as_float(e < 8 ? s2la[e] : s2lb[e - 8]);
                const float a = fmaf(-m, S0, x1);
                stg[e * 32 + lane] = a;
                stg[(16 + e) * 32 + lane] = fmaf(-m, a, fmaf(-m, x1, x2h) + x2l);
            }
            __syncwarp();
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int row = it * 4 + (lane >> 3), c4 = (lane & 7) * 4;
                const int d = d0 + b16 + (row & 15);
                if (d < D)
                    *reinterpret_cast<float4 *>(dst0 + (size_t)(row < 16 ? d : D + d) * Kp + c4) =
                        *reinterpret_cast<const float4 *>(stg + row * 32 + c4);
            }
            __syncwarp();   // the block is read before the next one overwrites it
        }
    }
    return true;
}

// Walks a cluster's units tile by tile (the current unit is held in registers).
struct TileWalk {
    const StatUnit *u;
    int n, ui, t, nt;
    int64_t row0_;
    int nrows_, slot_;
    __device__ TileWalk(const StatUnit *units, int2 cu) : u(units + cu.x), n(cu.y), ui(0), t(0) { load(); }
    __device__ void load() {
        if (ui < n) {
            const StatUnit v = u[ui];
            row0_ = v.row0;
            nrows_ = v.nrows;
            slot_ = v.slot;
            nt = (nrows_ + kRows - 1) / kRows;
        } else {
            nt = 0;
        }
    }
    __device__ bool more() const { return ui < n; }
    __device__ void next() {
        if (++t == nt) {
            t = 0;
            ++ui;
            load();
        }
    }
    __device__ int row0() const { return (int)(row0_ + (int64_t)t * kRows); }
    __device__ int valid() const { return min(kRows, nrows_ - t * kRows); }
    __device__ bool first() const { return t == 0; }
    __device__ bool last() const { return t == nt - 1; }
    __device__ int slot() const { return slot_; }
};

// SPARSE: early termination with p.tau > 0 (a separate instantiation, so the
// exact encoder's code is the same as without it).
template <bool SPARSE, bool GLO>
__global__ void __launch_bounds__(kThreads, 1)
bf16_encode_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmB, EncArgs p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const EncSmem L = enc_smem(p.nkb, p.S, p.nstage, GLO);
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + L.bars);
    uint32_t *misc = reinterpret_cast<uint32_t *>(smem + L.misc);   // [0] tmem base, [1] abort
    volatile uint32_t *abort_flag = misc + 1;

    if ((smem_u32(smem) & 1023u) != 0u) {   // layout assumption broken (same in every CTA): refuse to run
        if (threadIdx.x == 0) atomicOr(p.err, kErrAlign);
        return;
    }
    const uint32_t rank = p.S > 1 ? cluster_ctarank() : 0u;
    const int2 cu = p.cl_units[blockIdx.x / p.S];

    if (threadIdx.x == 0) {
        mbar_init(&bars[EB_BFULL], 1);
        mbar_init(&bars[EB_DRAIN2], 1);
        for (int s = 0; s < 2; ++s) {
            mbar_init(&bars[EB_XRFULL + s], 1);
            mbar_init(&bars[EB_AFULL + s], 6);
            mbar_init(&bars[EB_STFREE + s], 1);
            mbar_init(&bars[EB_LFULL + s], 1);
            mbar_init(&bars[EB_LEMPTY + s], 8);
            mbar_init(&bars[EB_XCHG + s], 1);
        }
        mbar_init(&bars[EB_GFULL], GLO ? 4 : 8);   // BF16X2: the four warps of lane quadrants 0-1
        if (GLO) {
            mbar_init(&bars[EB_GFULL2], 4);
            mbar_init(&bars[EB_GFREE2], 1);
        }
        mbar_init(&bars[EB_GFREE], 1);
        mbar_init(&bars[EB_SDONE], 1);
        mbar_init(&bars[EB_TEMPTY], 8);
        mbar_init(&bars[EB_DRAIN], 1);
        for (int q = 0; q < 4; ++q) {
            mbar_init(&bars[EB_HXFULL + q], 2);   // one arrive per warp, after __syncwarp
            mbar_init(&bars[EB_HXFREE + q], 2);
        }
        mbar_init(&bars[EB_XRFREE], 6);
        misc[1] = 0u;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&misc[0], kTmemCols);
        tmem_relinquish();
    }
    if (threadIdx.x >= 64 && threadIdx.x < 64 + kComps)
        reinterpret_cast<float *>(smem + L.cl)[threadIdx.x - 64] = p.cl2[rank * kComps + threadIdx.x - 64];
    tc_fence_before();
    __syncthreads();
    if (p.S > 1) cluster_sync();   // peers' barriers initialised before any remote arrive
    tc_fence_after();
    const uint32_t tmem = misc[0];
    const uint32_t plane = (uint32_t)p.nkb * kBlk;   // one of the X, X2hi, X2lo planes

    if (warp == 0 && lane == 0) {
        // ---------------- TMA loads and log-likelihood GEMMs ----------------
        // The builders taking tile i's x into registers (XRFREE) frees the
        // landing buffer, so x of tile i + 1 is requested then; L(i) follows
        // once tile i's Y planes are built (AFULL) and its TMEM buffer is free. (Issuing L blocks this thread for most of its
        // duration, so the statistics GEMMs have their own thread.)
        prefetch_tmap(&tmX);
        prefetch_tmap(&tmB);
        mbar_arrive_expect_tx(&bars[EB_BFULL], 4u * plane);
        for (int t = 0; t < 4; ++t)
            for (int j = 0; j < p.nkb; ++j)
                tma_load_2d(smem + L.b + (t * p.nkb + j) * kBlk, &tmB, &bars[EB_BFULL], j * 16,
                            t * p.Kp + (int)rank * kComps);
        const uint32_t idesc_l = idesc_bf16(kRows, kComps, false, false);
        const uint32_t sB = smem_u32(smem + L.b);
        TileWalk w(p.units, cu), wn(p.units, cu);
        int last_load = -1;
        auto load_x = [&](int i, int row0) {
            mbar_arrive_expect_tx(&bars[EB_XRFULL + (i & 1)], plane);
            for (int j = 0; j < p.nkb; ++j)
                tma_load_2d(smem + L.xr + j * kBlk, &tmX, &bars[EB_XRFULL + (i & 1)], j * 16, row0);
            last_load = i;
        };
        if (wn.more()) {
            load_x(0, wn.row0());
            wn.next();
        }
        bool ok = mbar_wait(&bars[EB_BFULL], 0, abort_flag, p.err);
        bool issued = false;
        for (int i = 0; ok && w.more(); w.next(), ++i) {
            const int s = i % p.nstage, b = i & 1;
            if (!mbar_wait(&bars[EB_XRFREE], i & 1, abort_flag, p.err)) break;
            if (wn.more()) {
                load_x(i + 1, wn.row0());
                wn.next();
            }
            if (!mbar_wait(&bars[EB_AFULL + s], (i / p.nstage) & 1, abort_flag, p.err)) break;
            if (i >= 2 && !mbar_wait(&bars[EB_LEMPTY + b], ((i >> 1) - 1) & 1, abort_flag, p.err)) break;
            tc_fence_after();
            const uint32_t sA = smem_u32(smem + L.y + s * L.y_stage);
            const uint32_t d = tmem + (uint32_t)(b * kComps);
            for (int j = 0; j < p.nkb; ++j) {
                const uint64_t ax = sdesc_sw32(sA + j * kBlk, 16, 256);
                const uint64_t ah = sdesc_sw32(sA + plane + j * kBlk, 16, 256);
                const uint64_t al = sdesc_sw32(sA + 2 * plane + j * kBlk, 16, 256);
                const uint64_t bqh = sdesc_sw32(sB + (0 * p.nkb + j) * kBlk, 16, 256);
                const uint64_t bql = sdesc_sw32(sB + (1 * p.nkb + j) * kBlk, 16, 256);
                const uint64_t brh = sdesc_sw32(sB + (2 * p.nkb + j) * kBlk, 16, 256);
                const uint64_t brl = sdesc_sw32(sB + (3 * p.nkb + j) * kBlk, 16, 256);
                mma_bf16(d, ax, bqh, idesc_l, j > 0 ? 1u : 0u);
                mma_bf16(d, ax, bql, idesc_l, 1u);
                mma_bf16(d, ah, brh, idesc_l, 1u);
                mma_bf16(d, ah, brl, idesc_l, 1u);
                mma_bf16(d, al, brh, idesc_l, 1u);
            }
            mma_commit(&bars[EB_LFULL + b]);
            issued = true;
        }
        if (issued) {   // every issued MMA has finished before TMEM is released
            mma_commit(&bars[EB_DRAIN]);
            mbar_drain(&bars[EB_DRAIN], 0, 2000000000ll);
        }
        // wait (bounded, even when aborting) for this thread's copies still in flight
        if (last_load >= 0) mbar_drain(&bars[EB_XRFULL + (last_load & 1)], (last_load >> 1) & 1, 200000000ll);
        mbar_drain(&bars[EB_BFULL], 0, 200000000ll);
    } else if (warp == 1 && lane == 0) {
        // ---------------- statistics GEMMs ----------------
        const uint32_t idesc_s = idesc_bf16(kComps, p.ny, true, true);
        const uint32_t sG = smem_u32(smem + L.g);
        const volatile uint8_t *flags = smem + L.flags;
        bool issued = false, started = false;
        unsigned long long nskip = 0, nsteps = 0;
        int i = 0;
        for (TileWalk w(p.units, cu); w.more(); w.next(), ++i) {
            if (w.first() && w.ui > 0) {   // the previous unit's accumulator has been written out
                if (!mbar_wait(&bars[EB_TEMPTY], (w.ui - 1) & 1, abort_flag, p.err)) break;
            }
            const uint32_t sy = smem_u32(smem + L.y + (i % p.nstage) * L.y_stage);
            if constexpr (GLO) {
                // BF16X2: gamma^T hi + lo of rows 0-63, then of rows 64-127, through
                // the same buffer (hi at sG, lo at sG + kGHalf, 64-component blocks
                // kSub apart); each half has its own full / free barrier pair
                if (SPARSE && w.first()) started = false;
                bool ok = true;
                for (int hf = 0; hf < 2; ++hf) {
                    if (!mbar_wait(&bars[hf ? EB_GFULL2 : EB_GFULL], i & 1, abort_flag, p.err)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int ql = 0; ql < 4; ++ql) {
                        const int q = hf * 4 + ql;   // K step: rows 16q .. 16q + 15 of the tile
                        if constexpr (SPARSE) {
                            ++nsteps;
                            if (!(flags[q] | flags[8 + q]) && (started || !w.last() || q > 0)) {
                                ++nskip;
                                continue;
                            }
                        }
                        const uint64_t b = sdesc_sw32(sy + q * 512, kBlk, 256);
                        const uint32_t accum = SPARSE ? (started ? 1u : 0u) : ((w.first() && q == 0) ? 0u : 1u);
                        mma_bf16(tmem + kStatCol, sdesc_sw128(sG + ql * 2048, kSub, 1024), b, idesc_s, accum);
                        mma_bf16(tmem + kStatCol, sdesc_sw128(sG + kGHalf + ql * 2048, kSub, 1024), b, idesc_s, 1u);
                        started = true;
                    }
                    mma_commit(&bars[hf ? EB_GFREE2 : EB_GFREE]);
                    issued = true;   // drained before TMEM is freed, even if the next wait gives up
                }
                if (!ok) break;
            } else {
                if (!mbar_wait(&bars[EB_GFULL], i & 1, abort_flag, p.err)) break;
                tc_fence_after();
                if constexpr (SPARSE) {
                    if (w.first()) started = false;   // the next MMA initialises the unit's accumulator
                    for (int q = 0; q < kRows / 16; ++q) {
                        // a K step whose 16 x 128 posteriors are all zero adds nothing;
                        // a unit's last tile issues its first step regardless when
                        // nothing was issued yet (zero posteriors then zero the accumulator)
                        ++nsteps;
                        if (!(flags[q] | flags[8 + q]) && (started || !w.last() || q > 0)) {
                            ++nskip;
                            continue;
                        }
                        const uint64_t a = sdesc_sw128(sG + q * 2048, kGHalf, 1024);
                        const uint64_t b = sdesc_sw32(sy + q * 512, kBlk, 256);
                        mma_bf16(tmem + kStatCol, a, b, idesc_s, started ? 1u : 0u);
                        started = true;
                    }
                } else {
                    for (int q = 0; q < kRows / 16; ++q) {
                        // gamma^T: MN-major, 128-byte swizzle, 64-component halves kGHalf
                        // apart, 8-row groups 1 KB apart; Y: MN-major, 16-column blocks
                        // kBlk apart, 8-row groups 256 B apart; 16 rows per K step
                        const uint64_t a = sdesc_sw128(sG + q * 2048, kGHalf, 1024);
                        const uint64_t b = sdesc_sw32(sy + q * 512, kBlk, 256);
                        mma_bf16(tmem + kStatCol, a, b, idesc_s, (w.first() && q == 0) ? 0u : 1u);
                    }
                }
                mma_commit(&bars[EB_GFREE]);
            }
            mma_commit(&bars[EB_STFREE + (i & 1)]);
            if (w.last()) mma_commit(&bars[EB_SDONE]);
            issued = true;
        }
        if (issued) {
            mma_commit(&bars[EB_DRAIN2]);
            mbar_drain(&bars[EB_DRAIN2], 0, 2000000000ll);
        }
        if (SPARSE && p.skip_count) {
            atomicAdd(&p.skip_count[0], nskip);
            atomicAdd(&p.skip_count[1], nsteps);
        }
    } else if (warp == 2 || warp == 3 || warp >= 12) {
        // ---------------- Y builders: the tile's Y planes from the landing buffer ----------------
        const int bt = (warp < 12 ? warp - 2 : warp - 10) * 32 + lane;   // 0..kBuilders-1
        int i = 0;
        for (TileWalk w(p.units, cu); w.more(); w.next(), ++i) {
            const int s = i % p.nstage, j = i - p.nstage;   // tile j used this stage before
            if (!mbar_wait(&bars[EB_XRFULL + (i & 1)], (i >> 1) & 1, abort_flag, p.err)) break;
            uint4 x[kHold];
            x_load(x, smem + L.xr, p.nkb, bt);
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[EB_XRFREE]);   // release: the reads precede the next TMA write
            if (j >= 0 && !mbar_wait(&bars[EB_STFREE + (j & 1)], (j >> 1) & 1, abort_flag, p.err)) break;
            y_store(smem + L.y + s * L.y_stage, x, plane, p.nkb, w.valid(), bt);
            fence_proxy_async_smem();   // generic-proxy stores visible to the MMAs
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[EB_AFULL + s]);
        }
    } else if (warp >= 4) {
        // ---------------- softmax warps ----------------
        // Eight warps take every tile: warp 4+q and 8+q own rows 32q..32q+31
        // (their TMEM lane quadrant), one row per thread, over components
        // 64h..64h+63 (h = 0 for warps 4-7, 1 for 8-11) in two 32-column
        // chunks. Pass A forms y = l log2(e) + c log2(e), keeps an online row
        // max/sum with a reference max per chunk and holds 2^(y - ref) in
        // registers (the TMEM buffer is released at once); the two halves of a
        // row combine their (max, sum) through shared memory, then the
        // cluster's CTAs combine theirs; pass B rescales each chunk and writes
        // bf16 gamma^T to shared memory. After
        // a unit's last tile the eight warps write the unit's centred
        // statistics from TMEM to its slot (half the dimensions each).
        const int h = (warp - 4) >> 2, q = warp & 3;
        const int r = q * 32 + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
        const float *cl = reinterpret_cast<const float *>(smem + L.cl) + h * 64;
        float2 *xbuf = reinterpret_cast<float2 *>(smem + L.xchg);
        float2 *hx = reinterpret_cast<float2 *>(smem + L.hx);
        // this row of this warp's 64-component half (BF16X2: of the 64-row half
        // that holds it, hi here and lo kGHalf further)
        uint8_t *gsm = GLO ? smem + L.g + h * kSub + (r & 63) * 128 : smem + L.g + h * kGHalf + r * 128;
        const int sw = r & 7;                  // 128-byte swizzle: 16-byte chunk j sits at j ^ (row & 7)
        int i = 0;
        TileWalk w(p.units, cu);
        bool ok = true;
        while (ok && w.more()) {
            const int b = i & 1;
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[EB_LFULL + b], (i >> 1) & 1, abort_flag, p.err))) break;
            tc_fence_after();
            const uint32_t ta = lane_base + (uint32_t)(b * kComps + h * 64);
            float m = -INFINITY, z = 0.f;
            float mc[2];
            uint32_t ra[32], rb[32];
            // the second chunk's TMEM load is in flight while the first is
            // processed; a chunk's constants are requested before its wait
            tmem_ld32_issue(ta, ra);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t(&cur)[32] = c ? rb : ra;
                float4 ccur[8];
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) ccur[k4] = reinterpret_cast<const float4 *>(cl + c * 32)[k4];
                tmem_ld_wait(cur);
                if (c == 0) tmem_ld32_issue(ta + 32, rb);
                // y overwrites l in place; four independent max chains
                float cm0 = -INFINITY, cm1 = -INFINITY, cm2 = -INFINITY, cm3 = -INFINITY;
#pragma unroll
                for (int k4 = 0; k4 < 8; ++k4) {
                    const float y0 = fmaf(__uint_as_float(cur[4 * k4 + 0]), kLog2e, ccur[k4].x);
                    const float y1 = fmaf(__uint_as_float(cur[4 * k4 + 1]), kLog2e, ccur[k4].y);
                    const float y2 = fmaf(__uint_as_float(cur[4 * k4 + 2]), kLog2e, ccur[k4].z);
                    const float y3 = fmaf(__uint_as_float(cur[4 * k4 + 3]), kLog2e, ccur[k4].w);
                    cm0 = fmaxf(cm0, y0);
                    cm1 = fmaxf(cm1, y1);
                    cm2 = fmaxf(cm2, y2);
                    cm3 = fmaxf(cm3, y3);
                    cur[4 * k4 + 0] = __float_as_uint(y0);
                    cur[4 * k4 + 1] = __float_as_uint(y1);
                    cur[4 * k4 + 2] = __float_as_uint(y2);
                    cur[4 * k4 + 3] = __float_as_uint(y3);
                }
                const float mn = fmaxf(m, fmaxf(fmaxf(cm0, cm1), fmaxf(cm2, cm3)));
                const float mref = (mn == -INFINITY) ? 0.f : mn;
                float z0 = z * ex2_approx(m - mref), z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
                for (int k = 0; k < 32; k += 4) {
                    const float e0 = ex2_approx(__uint_as_float(cur[k + 0]) - mref);
                    const float e1 = ex2_approx(__uint_as_float(cur[k + 1]) - mref);
                    const float e2 = ex2_approx(__uint_as_float(cur[k + 2]) - mref);
                    const float e3 = ex2_approx(__uint_as_float(cur[k + 3]) - mref);
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
                mc[c] = mref;
                m = mn;
            }
            // the exponentials stay in registers (ra, rb) for pass B, so this
            // tile's log-likelihood buffer is free for the GEMM of tile i + 2
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[EB_LEMPTY + b]);
            // the row's two halves: (max, sum) of both, combined in half order
            // (bounded handshakes: the partner has read the previous tile's
            // value before this one is written, and written this tile's before
            // it is read)
            if (i > 0 && !__all_sync(0xffffffffu, mbar_wait(&bars[EB_HXFREE + q], (i - 1) & 1, abort_flag, p.err)))
                break;
            hx[h * kRows + r] = make_float2(m, z);
            __syncwarp();   // the warp's writes ordered before its one (release) arrive
            if (lane == 0) mbar_arrive(&bars[EB_HXFULL + q]);
            if (!__all_sync(0xffffffffu, mbar_wait(&bars[EB_HXFULL + q], i & 1, abort_flag, p.err))) break;
            const float2 h0 = hx[r], h1 = hx[kRows + r];
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[EB_HXFREE + q]);
            float mh, zh;
            {
                mh = fmaxf(h0.x, h1.x);
                const float ref = (mh == -INFINITY) ? 0.f : mh;
                zh = h0.y * ex2_approx(h0.x - ref) + h1.y * ex2_approx(h1.x - ref);
            }
            // (max, sum) over the cluster, combined in rank order so that every
            // CTA normalises with the same value. Exchange slot i % 2 of every
            // CTA receives the peers' values for tile i (counted in bytes on
            // XCHG, armed once per tile); warps 4-7 write their 32 rows into
            // their own rank's segment of the slot and send it to each peer as
            // one 256-byte bulk copy. A peer writes slot i % 2 again only for
            // tile i + 2, after this CTA's contribution to tile i + 1, which
            // warps 4-7 send only after the half handshake of tile i + 1, i.e.
            // after warps 8-11 have read tile i's values; likewise this CTA
            // rewrites its own segment (the copies' source) for tile i + 2 only
            // after every peer's tile i + 1 values arrived, which they send
            // after tile i's copies from here have landed.
            float M = -INFINITY, Z = 0.f;
            if (p.S > 1) {
                const int j = i & 1;
                float2 *xb = xbuf + j * p.S * kRows;
                if (h == 0) {
                    if (q == 0 && lane == 0)
                        mbar_arrive_expect_tx(&bars[EB_XCHG + j], (uint32_t)(p.S - 1) * kRows * 8u);
                    xb[rank * kRows + r] = make_float2(mh, zh);
                    fence_proxy_async_smem();   // the copy engine reads what the lanes wrote
                    __syncwarp();
                    if (lane < p.S && lane != (int)rank) {   // lane pr sends to peer pr
                        const uint32_t seg = smem_u32(&xb[rank * kRows + q * 32]);
                        bulk_s2cluster(mapa(seg, (uint32_t)lane), seg, 32u * 8u,
                                       mapa(smem_u32(&bars[EB_XCHG + j]), (uint32_t)lane));
                    }
                }
                if (!__all_sync(0xffffffffu,
                                mbar_wait(&bars[EB_XCHG + j], (i >> 1) & 1, abort_flag, p.err, true)))
                    break;
                for (int pr = 0; pr < p.S; ++pr) {
                    const float2 v = pr == (int)rank ? make_float2(mh, zh) : xb[pr * kRows + r];
                    const float Mn = fmaxf(M, v.x);
                    const float ref = (Mn == -INFINITY) ? 0.f : Mn;
                    Z = Z * ex2_approx(M - ref) + v.y * ex2_approx(v.x - ref);
                    M = Mn;
                }
            } else {
                M = mh;
                Z = zh;
            }
            const float Mref = (M == -INFINITY) ? 0.f : M;
            const float inv = 1.0f / Z;
            if constexpr (GLO) {
                // BF16X2: rows 0-63 (quadrants 0-1) go into the buffer once the
                // statistics GEMM has read rows 64-127 of the previous tile (and,
                // at a unit's first tile, once the previous unit's write-out,
                // which stages through this buffer, is over); rows 64-127 once
                // it has read rows 0-63 of this tile. Every phase is waited on.
                if (q < 2) {
                    if (w.first() && w.ui > 0 &&
                        !__all_sync(0xffffffffu, mbar_wait(&bars[EB_TEMPTY], (w.ui - 1) & 1, abort_flag, p.err)))
                        break;
                    if (i >= 1 &&
                        !__all_sync(0xffffffffu, mbar_wait(&bars[EB_GFREE2], (i - 1) & 1, abort_flag, p.err)))
                        break;
                } else if (!__all_sync(0xffffffffu, mbar_wait(&bars[EB_GFREE], i & 1, abort_flag, p.err))) {
                    break;
                }
            } else {
                // the statistics GEMM of the previous tile has read gamma^T (these
                // warps wait on every phase of GFREE in order, so none is skipped)
                if (i >= 1 &&
                    !__all_sync(0xffffffffu, mbar_wait(&bars[EB_GFREE], (i - 1) & 1, abort_flag, p.err))) break;
            }
            // pass B: normalised posteriors -> bf16 gamma^T from the registers of pass A
            bool row_nz = false;   // early termination: a posterior of this row and half above tau
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t(&cur)[32] = c ? rb : ra;
                const float sc = ex2_approx(mc[c] - Mref) * inv;
                if constexpr (SPARSE) {   // posteriors not above tau are dropped
                    const float tau = p.tau;
#pragma unroll
                    for (int k = 0; k < 32; ++k) {
                        const float g = __uint_as_float(cur[k]) * sc;
                        row_nz |= g > tau;
                        cur[k] = g > tau ? cur[k] : 0u;
                    }
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {   // 16-byte chunk c * 4 + k of the 128-byte row
                    if constexpr (GLO) {
                        // hi = RN_bf16(g), lo = RN_bf16(g - hi): g - hi is exact in FP32
                        uint32_t hv[4], lv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float g0 = __uint_as_float(cur[8 * k + 2 * e]) * sc;
                            const float g1 = __uint_as_float(cur[8 * k + 2 * e + 1]) * sc;
                            hv[e] = pack_bf16x2(g0, g1);
                            const float h0 = __uint_as_float(hv[e] << 16), h1 = __uint_as_float(hv[e] & 0xFFFF0000u);
                            lv[e] = pack_bf16x2(g0 - h0, g1 - h1);
                        }
                        *reinterpret_cast<uint4 *>(gsm + (((c * 4 + k) ^ sw) << 4)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
                        *reinterpret_cast<uint4 *>(gsm + kGHalf + (((c * 4 + k) ^ sw) << 4)) =
                            make_uint4(lv[0], lv[1], lv[2], lv[3]);
                    } else {
                        uint4 v;
                        v.x = pack_bf16x2(__uint_as_float(cur[8 * k + 0]) * sc, __uint_as_float(cur[8 * k + 1]) * sc);
                        v.y = pack_bf16x2(__uint_as_float(cur[8 * k + 2]) * sc, __uint_as_float(cur[8 * k + 3]) * sc);
                        v.z = pack_bf16x2(__uint_as_float(cur[8 * k + 4]) * sc, __uint_as_float(cur[8 * k + 5]) * sc);
                        v.w = pack_bf16x2(__uint_as_float(cur[8 * k + 6]) * sc, __uint_as_float(cur[8 * k + 7]) * sc);
                        *reinterpret_cast<uint4 *>(gsm + (((c * 4 + k) ^ sw) << 4)) = v;
                    }
                }
            }
            if constexpr (SPARSE) {   // marks of this warp's two 16-row K steps (its half of the components)
                const uint32_t bal = __ballot_sync(0xffffffffu, row_nz);
                if (lane == 0) {
                    smem[L.flags + h * 8 + 2 * q] = (bal & 0xFFFFu) != 0u;
                    smem[L.flags + h * 8 + 2 * q + 1] = (bal >> 16) != 0u;
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[GLO && q >= 2 ? EB_GFULL2 : EB_GFULL]);
            const bool last = w.last();
            const int uidx = w.ui, uslot = w.slot();
            w.next();
            ++i;
            if (!last) continue;
            // the unit's statistics: TMEM -> slot part[slot][j][Kp], centred
            // (write_stats); the warps of one lane quadrant split the
            // dimensions in 32-wide chunks
            if (!write_stats(&bars[EB_SDONE], uidx & 1, abort_flag, p.err, lane_base + kStatCol,
                             reinterpret_cast<float *>(smem + L.g + h * kGHalf + q * 32 * 128),
                             p.part + (size_t)uslot * p.Kp * p.P + (size_t)rank * kComps + q * 32, p.mu_t, h, p.D,
                             p.nkb * 16, p.Kp, (int)rank * kComps + q * 32 + lane, lane))
                break;
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bars[EB_TEMPTY]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (p.S > 1) cluster_sync();   // no remote access into a CTA that has exited
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kTmemCols);
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
// 16 x box_rows with the 32-byte swizzle; zero fill out of bounds.
bool make_map(CUtensorMap *m, const void *base, uint64_t cols, uint64_t rows, uint64_t pitch_elems, uint32_t box_rows) {
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {pitch_elems * 2};
    cuuint32_t box[2] = {16u, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

struct EncCfg {
    int nkb, S, nstage, ny;
    bool glo;
    size_t smem;
};

bool enc_config(const fv_gmm *g, EncCfg &c) {
    c.nkb = round_up(g->D, 16) / 16;
    c.S = g->Kp / kComps;
    c.ny = 3 * c.nkb * 16 + 16;
    c.glo = g->prec == FV_PREC_BF16X2;
    c.nstage = enc_smem(c.nkb, c.S, 2, c.glo).total <= (uint32_t)kMaxSmem ? 2 : 1;
    c.smem = enc_smem(c.nkb, c.S, c.nstage, c.glo).total;
    return g->Kp % kComps == 0 && c.S >= 1 && c.S <= 4 && c.ny <= 256 && c.nkb * kRows * 2 <= kHold * kBuilders &&
           c.smem <= (size_t)kMaxSmem;
}

void enc_launch_config(const EncCfg &c, int clusters, cudaStream_t st, cudaLaunchConfig_t &cfg,
                       cudaLaunchAttribute *attr) {
    cfg = cudaLaunchConfig_t{};
    cfg.gridDim = dim3((unsigned)(clusters * c.S));
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.S;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
}

}  // namespace

int bf16_max_shares(const fv_gmm *g, int sms) {
    // clusters of the encoder kernel resident at once (one CTA per SM; a
    // cluster's CTAs share a GPC, so larger clusters leave some SMs idle)
    EncCfg c;
    if (!enc_config(g, c)) return 1;
    if (c.S == 1) return std::max(1, sms);
    static std::mutex mu;
    static std::map<std::tuple<int, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_tuple(dev, c.S + (c.glo ? 1000 : 0), c.smem);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    int n = 0;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    enc_launch_config(c, std::max(1, sms / c.S), nullptr, cfg, attr);
    auto kern = c.glo ? bf16_encode_kernel<false, true> : bf16_encode_kernel<false, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem) != cudaSuccess ||
        cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess || n < 1) {
        cudaGetLastError();
        n = std::max(1, sms / c.S);
    }
    cache[key] = n;
    return n;
}

int bf16_shares(const fv_gmm *g, int64_t rows, int sms) {
    // persistent clusters over balanced row shares; a share of fewer than two
    // tiles would move more slot bytes than it saves time
    const int64_t tiles = (rows + kRows - 1) / kRows;
    return (int)std::max<int64_t>(1, std::min<int64_t>(bf16_max_shares(g, sms), (tiles + 1) / 2));
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

int bf16_max_stages(const fv_gmm *g) {
    EncCfg c;
    return enc_config(g, c) ? c.nstage : 1;
}

int run_bf16_encoder(const fv_gmm *g, const uint16_t *Xb, int64_t ldx, int64_t rows, const StatUnit *units,
                     const int2 *cl_units, int n_shares, float *part, int P, uint32_t *err, cudaStream_t st,
                     float tau, unsigned long long *skip_count, int nstage) {
    if (rows <= 0 || n_shares <= 0) return FV_OK;
    if (get_encoder() != cudaSuccess) return fail(FV_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
    EncCfg c;
    if (!enc_config(g, c)) return fail(FV_ERR_UNSUPPORTED, "BF16 form: shape does not fit the kernel's shared memory");
    if (nstage > 0 && nstage < c.nstage) {   // fewer stages than fit (the autotuner's choice)
        c.nstage = nstage;
        c.smem = enc_smem(c.nkb, c.S, c.nstage, c.glo).total;
    }
    if (P != 2 * g->D + 1) return fail(FV_ERR_INVALID, "BF16 form: slot width mismatch");
    if (rows > (int64_t)INT32_MAX - 256) return fail(FV_ERR_UNSUPPORTED, "BF16 form: too many rows for one call");

    CUtensorMap tmX, tmB;
    if (!make_map(&tmX, Xb, (uint64_t)g->D, (uint64_t)rows, (uint64_t)ldx, kRows) ||
        !make_map(&tmB, g->dev.bimg, (uint64_t)c.nkb * 16, (uint64_t)4 * g->Kp, (uint64_t)c.nkb * 16, kComps))
        return fail(FV_ERR_CUDA, "cuTensorMapEncodeTiled failed");

    EncArgs a;
    a.nkb = c.nkb;
    a.Kp = g->Kp;
    a.S = c.S;
    a.nstage = c.nstage;
    a.ny = c.ny;
    a.P = P;
    a.D = g->D;
    a.mu_t = g->dev.mu_t;
    a.cl2 = g->dev.cl2;
    a.units = units;
    a.cl_units = cl_units;
    a.part = part;
    a.err = err;
    a.glo = c.glo ? 1 : 0;
    a.tau = tau;
    a.skip_count = skip_count;
    auto kern = tau > 0.f ? (c.glo ? bf16_encode_kernel<true, true> : bf16_encode_kernel<true, false>)
                          : (c.glo ? bf16_encode_kernel<false, true> : bf16_encode_kernel<false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
    if (e != cudaSuccess) return cuda_fail(e, "bf16 encoder: smem attribute");
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    enc_launch_config(c, n_shares, st, cfg, attr);
    {
        KernelTimer kt_("bf16_encode", st);
        e = cudaLaunchKernelEx(&cfg, kern, tmX, tmB, a);
    }
    if (e != cudaSuccess) return cuda_fail(e, "bf16 encoder launch");
    return FV_OK;
}

}  // namespace fv
