// PCA projection and position append (Sec. 3.1): the step that turns a raw
// 128-dimensional descriptor into the encoder's input,
//   y_i = [ P (x_i - mean) ; xy_i ],   D = m + 2,
// run on the GPU as a prologue stage in front of the encoder.
//
// Plain FP32 form: a SIMT kernel, 64 rows per block, the centred rows and
// the basis staged in shared memory, 4 rows x 5 outputs per thread.
//
// BF16 form: one tcgen05 GEMM tile per CTA, M = 128 rows, N = m rounded up to
// 16, K = Din, FP32 accumulator in TMEM. The centred descriptors x - mean
// (FP32) and the basis are each split into bfloat16 hi + lo parts and three
// products accumulate, x_hi P_hi + x_hi P_lo + x_lo P_hi (the lo x lo term is
// below 2^-16 of the result), so the projection carries about 16 significant
// bits before it is rounded to the bfloat16 rows the encoder reads (row
// pitch a multiple of 16 elements, zero padded). Operands use the same
// shared-memory layout as the encoder: blocks of 16 bf16 columns stored as
// [rows][16] 32-byte rows with the 32-byte swizzle (the 16-byte half of row r
// sits at half ^ ((r >> 2) & 1)). The basis image is built once at load time
// in that layout and copied into shared memory by every CTA.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "fv_dsift.h"
#include "fv_internal.h"
#include "fv_sm100.cuh"

struct fv_pca {
    int m, Din, Npad, device;
    float *basis;      // [m][Din]
    float *mean;       // [Din]
    uint16_t *bimg;    // [2 terms][Din/16 blocks][Npad rows][16] bf16, swizzled (BF16 form operand)
    void *block;
};

namespace fv {
namespace {

using namespace sm100;

constexpr int kPcaRows = 128;
constexpr int kPcaThreads = 256;

__device__ __forceinline__ uint16_t bf16_rn(float f) {
    __nv_bfloat16 h = __float2bfloat16_rn(f);
    return *reinterpret_cast<uint16_t *>(&h);
}
__device__ __forceinline__ float bf16_val(uint16_t b) { return __uint_as_float(((uint32_t)b) << 16); }

// Byte offset of element (row, col) in a [rows][16]-block image with the
// 32-byte swizzle: block col/16, 32-byte row, 16-byte half swizzled by row.
__host__ __device__ __forceinline__ uint32_t sw32_offset(int row, int col, int rows_per_block) {
    const int blk = col >> 4, half = (col >> 3) & 1, e = col & 7;
    return (uint32_t)(blk * rows_per_block * 32 + row * 32 + ((half ^ ((row >> 2) & 1)) << 4) + e * 2);
}

// Basis hi/lo image in the swizzled operand layout (zero rows past m).
__global__ void pca_bimg_kernel(const float *__restrict__ P, int m, int Din, int Npad, uint16_t *__restrict__ img) {
    const int n = blockIdx.x;   // output dimension (row of the N x K operand)
    const size_t term = (size_t)(Din / 16) * Npad * 16;   // elements per term
    for (int k = threadIdx.x; k < Din; k += blockDim.x) {
        const float v = n < m ? P[(size_t)n * Din + k] : 0.f;
        const uint16_t hi = bf16_rn(v);
        const uint16_t lo = bf16_rn(v - bf16_val(hi));
        const uint32_t off = sw32_offset(n, k, Npad) / 2;
        img[off] = hi;
        img[term + off] = lo;
    }
}

// GATHER: the 8 values of bin `bin` (entries 8 bin .. 8 bin + 7) of dense-SIFT
// descriptor `row` (frames of dp.ndesc descriptors), read from the y-pass
// buffer before normalisation: bin (bx, by) of the descriptor at grid point
// (ix, iy) is lattice point (iy + by b/S, ix + bx b/S).
__device__ __forceinline__ void ds_gather(float (&v)[8], int64_t row, int bin, const float *__restrict__ yp,
                                          const DsPlan &dp) {
    const int64_t f = row / dp.ndesc, i = row - f * dp.ndesc;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < dp.n; ++q)
        if (i >= dp.s[q].desc_off) j = q;
    const DsScale &c = dp.s[j];
    const int64_t k = i - c.desc_off;
    const int iy = (int)(k / c.nx), ix = (int)(k - (int64_t)iy * c.nx);
    const int bs = dp.b / dp.S;
    const int mm = iy + (bin >> 2) * bs, t = ix + (bin & 3) * bs;
    const float4 *src = reinterpret_cast<const float4 *>(yp + (size_t)f * dp.yp + c.yp_off + ((size_t)mm * c.Tx + t) * 8);
    const float4 a = src[0], b = src[1];
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// grid ceil(N / 128), block 256, dynamic smem = basis image + A image.
// GATHER (Din = 128): row r is dense-SIFT descriptor r, assembled from the
// y-pass buffer yp (plan dp) and normalised here (L2, cap 0.2, L2; the 16
// chunks of a row sit in 16 consecutive lanes) instead of being read from X.
template <bool GATHER>
__global__ void __launch_bounds__(kPcaThreads)
pca_bf16_kernel(const float *__restrict__ X, int64_t N, int Din, const float *__restrict__ mean,
                const uint16_t *__restrict__ bimg, int Npad, int m, const float *__restrict__ xy,
                uint16_t *__restrict__ Y, int ld, uint32_t *__restrict__ err, const float *__restrict__ yp,
                const DsPlan dp) {
    extern __shared__ __align__(1024) uint8_t smem[];
    const int nkb = Din / 16;
    const uint32_t b_bytes = 2u * nkb * Npad * 32u;        // [hi | lo] basis image
    const uint32_t a_term = (uint32_t)nkb * kPcaRows * 32u;
    uint8_t *sB = smem, *sA = smem + b_bytes;
    uint64_t &bar = *reinterpret_cast<uint64_t *>(sA + 2 * a_term);       // MMAs complete
    uint64_t &lbar = *reinterpret_cast<uint64_t *>(sA + 2 * a_term + 8);  // bulk copies landed
    uint32_t &tslot = *reinterpret_cast<uint32_t *>(sA + 2 * a_term + 16);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t row0 = (int64_t)blockIdx.x * kPcaRows;
    const int nrows = (int)min((int64_t)kPcaRows, N - row0);
    const uint32_t ncols = Npad <= 32 ? 32u : (Npad <= 64 ? 64u : 128u);
    // X rows (pitch Din) of a tile are contiguous: with Din <= 128 (a thread
    // then holds its whole share of the tile in registers) one bulk copy lands
    // them, FP32, where the A image goes, and they are read out before the
    // image is written over them
    const bool bulk = !GATHER && Din <= 128 && (reinterpret_cast<uintptr_t>(X) & 15u) == 0;

    if ((smem_u32(smem) & 1023u) != 0u) {   // swizzle atoms need aligned blocks (same in every CTA)
        if (threadIdx.x == 0) atomicOr(err, kErrAlign);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_init(&lbar, 1);
        fence_mbar_init();
        const uint32_t xbytes = bulk ? (uint32_t)nrows * (uint32_t)Din * 4u : 0u;
        mbar_arrive_expect_tx(&lbar, b_bytes + xbytes);
        bulk_g2s(sB, bimg, b_bytes, &lbar);   // the basis image (built at load, L2-resident)
        if (bulk) bulk_g2s(sA, X + row0 * Din, xbytes, &lbar);
    }
    if (warp == 0) {
        __syncwarp();   // the allocation is warp-wide, after thread 0's branch
        tmem_alloc(&tslot, ncols);
        tmem_relinquish();
    }
    // a thread's chunks of 8 columns: c = tid + 256 u, row c / (Din / 8),
    // columns 8 (c % (Din / 8)) ..; all of them are requested before any is
    // converted (GATHER: rows tid / 16 + 16 u, bin tid % 16, each row then
    // normalised across the 16 lanes that hold it)
    constexpr int kGItems = kPcaRows * 16 / kPcaThreads;
    static_assert(kPcaRows * 16 % kPcaThreads == 0 && kPcaThreads % 32 == 0, "whole rows per half-warp");
    float gv[kGItems][8];
    if constexpr (GATHER) {
#pragma unroll
        for (int u = 0; u < kGItems; ++u) {
            const int c = threadIdx.x + u * kPcaThreads;
            const int64_t row = row0 + c / 16;
            if (row < N) {
                ds_gather(gv[u], row, c % 16, yp, dp);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) gv[u][e] = 0.f;
            }
        }
    }
    // requested before the waits: the thread's 8 column means (GATHER and bulk:
    // 256 is a multiple of Din / 8, so its columns are the same in every chunk)
    // and the position pair of its epilogue row (lane quadrant warp % 4)
    const int per = Din / 8, kt0 = (threadIdx.x % per) * 8;
    float mk[8];
    if (GATHER || bulk) {
#pragma unroll
        for (int e = 0; e < 8; ++e) mk[e] = mean[kt0 + e];
    }
    const int eq = warp & 3, ehalf = warp >> 2;
    const int er = eq * 32 + lane;
    const int64_t erow = row0 + er;
    float exy0 = 0.f, exy1 = 0.f;
    if (xy && erow < N) {
        exy0 = xy[2 * erow];
        exy1 = xy[2 * erow + 1];
    }
    __syncthreads();   // both mbarriers are initialised before any thread waits on one
    // the bulk copies have landed (bounded, about two seconds; on expiry the
    // tile is computed from whatever shared memory holds and flagged)
    {
        bool ok = mbar_try_wait(&lbar, 0);
        const long long t0 = clock64();
        while (!ok && clock64() - t0 < 4000000000ll) ok = mbar_try_wait_sleep(&lbar, 0, 2000u);
        if (!ok) atomicOr(err, kErrTimeout);
    }
    // hi + lo of 8 centred values into both A planes (swizzled row r, columns k0..k0+7)
    auto store_split = [&](int r, int k0, const float(&v)[8]) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const uint16_t h0 = bf16_rn(v[2 * e]), h1 = bf16_rn(v[2 * e + 1]);
            const uint16_t l0 = bf16_rn(v[2 * e] - bf16_val(h0)), l1 = bf16_rn(v[2 * e + 1] - bf16_val(h1));
            hw[e] = (uint32_t)h0 | ((uint32_t)h1 << 16);
            lw[e] = (uint32_t)l0 | ((uint32_t)l1 << 16);
        }
        const uint32_t off = sw32_offset(r, k0, kPcaRows);
        *reinterpret_cast<uint4 *>(sA + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
        *reinterpret_cast<uint4 *>(sA + a_term + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    };
    if constexpr (GATHER) {
#pragma unroll
        for (int u = 0; u < kGItems; ++u) {
            const int c = threadIdx.x + u * kPcaThreads;
            const int r = c / 16, k0 = kt0;
            const int64_t row = row0 + r;
            float(&v)[8] = gv[u];
            // every lane takes part in the half-warp reductions (rows past N are zeros)
            float ss = 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) ss = fmaf(v[e], v[e], ss);
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
            const float inv = ss > 0.f ? 1.f / sqrtf(ss) : 0.f;
            float s2 = 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                v[e] = fminf(v[e] * inv, 0.2f);
                s2 = fmaf(v[e], v[e], s2);
            }
#pragma unroll
            for (int o = 8; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            const float inv2 = s2 > 0.f ? 1.f / sqrtf(s2) : 0.f;
#pragma unroll
            for (int e = 0; e < 8; ++e) v[e] *= inv2;
            if (row < N) {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] -= mk[e];
            }
            store_split(r, k0, v);
        }
    } else if (bulk) {
        const int nit = Din / 16, k0 = kt0;
        const float *sX = reinterpret_cast<const float *>(sA);
#pragma unroll
        for (int u = 0; u < kGItems; ++u) {
            const int r = (threadIdx.x + u * kPcaThreads) / per;
            if (u < nit && r < nrows) {
                const float4 a = *reinterpret_cast<const float4 *>(sX + r * Din + k0);
                const float4 b = *reinterpret_cast<const float4 *>(sX + r * Din + k0 + 4);
                gv[u][0] = a.x - mk[0]; gv[u][1] = a.y - mk[1]; gv[u][2] = a.z - mk[2]; gv[u][3] = a.w - mk[3];
                gv[u][4] = b.x - mk[4]; gv[u][5] = b.y - mk[5]; gv[u][6] = b.z - mk[6]; gv[u][7] = b.w - mk[7];
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) gv[u][e] = 0.f;
            }
        }
        __syncthreads();   // every staged row is read before the image is written over it
#pragma unroll
        for (int u = 0; u < kGItems; ++u)
            if (u < nit) store_split((threadIdx.x + u * kPcaThreads) / per, k0, gv[u]);
    } else {
        // centred rows split into hi + lo, 8 columns per step
        for (int c = threadIdx.x; c < kPcaRows * (Din / 8); c += kPcaThreads) {
            const int r = c / (Din / 8), k0 = (c % (Din / 8)) * 8;
            const int64_t row = row0 + r;
            float v[8];
            if (row < N) {
                const float4 a = *reinterpret_cast<const float4 *>(X + row * Din + k0);
                const float4 b = *reinterpret_cast<const float4 *>(X + row * Din + k0 + 4);
                v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] -= mean[k0 + e];
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = 0.f;
            }
            store_split(r, k0, v);
        }
    }
    fence_proxy_async_smem();   // generic-proxy stores visible to the MMAs
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tslot;
    if (threadIdx.x == 0) {
        const uint32_t idesc = idesc_bf16(kPcaRows, Npad, false, false);
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        const uint32_t b_term = (uint32_t)nkb * Npad * 32u;
        for (int j = 0; j < nkb; ++j) {
            const uint64_t ah = sdesc_sw32(a0 + j * kPcaRows * 32, 16, 256);
            const uint64_t al = sdesc_sw32(a0 + a_term + j * kPcaRows * 32, 16, 256);
            const uint64_t bh = sdesc_sw32(b0 + j * Npad * 32, 16, 256);
            const uint64_t bl = sdesc_sw32(b0 + b_term + j * Npad * 32, 16, 256);
            mma_bf16(tmem, ah, bh, idesc, j > 0 ? 1u : 0u);
            mma_bf16(tmem, ah, bl, idesc, 1u);
            mma_bf16(tmem, al, bh, idesc, 1u);
        }
        mma_commit(&bar);
    }
    {
        // every warp: its TMEM lane quadrant's rows, 32-column chunks 32 ehalf + 64 j;
        // bounded wait for the MMAs (about two seconds); on expiry the rows become NaN
        bool ok = mbar_try_wait(&bar, 0);
        const long long t0 = clock64();
        while (!ok && clock64() - t0 < 4000000000ll) ok = mbar_try_wait_sleep(&bar, 0, 20000u);
        ok = __all_sync(0xffffffffu, ok);
        if (!ok && lane == 0) atomicOr(err, kErrTimeout);
        tc_fence_after();
        uint16_t *yr = Y + erow * ld;
        for (int c0 = ehalf * 32; c0 < Npad; c0 += 64) {
            uint32_t v[32];
            tmem_ld32_issue(tmem + ((uint32_t)(eq * 32) << 16) + (uint32_t)c0, v);
            tmem_ld_wait(v);
            if (erow < N) {
#pragma unroll
                for (int e = 0; e < 32; e += 8) {
                    const int n0 = c0 + e;
                    if (n0 >= ld) break;
                    uint32_t w4[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint16_t h[2];
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const int n = n0 + 2 * q + t;
                            float f = 0.f;
                            if (n < m) f = ok ? __uint_as_float(v[e + 2 * q + t]) : __int_as_float(0x7fc00000);
                            else if (n < m + 2) f = n == m ? exy0 : exy1;
                            h[t] = bf16_rn(f);
                        }
                        w4[q] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
                    }
                    *reinterpret_cast<uint4 *>(yr + n0) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
                }
            }
        }
        // columns past Npad (the position pair when m is a multiple of 16, and padding)
        if (ehalf == 0 && erow < N) {
            for (int n0 = Npad; n0 < ld; n0 += 8) {
                uint32_t w4[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint16_t h[2];
#pragma unroll
                    for (int t = 0; t < 2; ++t) {
                        const int n = n0 + 2 * q + t;
                        h[t] = bf16_rn(n == m ? exy0 : (n == m + 1 ? exy1 : 0.f));
                    }
                    w4[q] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
                }
                *reinterpret_cast<uint4 *>(yr + n0) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
        }
    }
    // the MMAs are complete before TMEM is released (bounded, also after an expired wait)
    if (threadIdx.x == 0) {
        mbar_drain(&bar, 0, 2000000000ll);
        mbar_drain(&lbar, 0, 2000000000ll);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, ncols);
    }
}

constexpr int kF32Rows = 64;

// grid ceil(N / 64), block 256: Y[row][0..m) = P (x - mean), then xy.
// Thread t: rows 4 (t / 16) .. +3, outputs (t % 16) + 16 j, j < 5 (m <= 80).
__global__ void __launch_bounds__(kPcaThreads)
pca_f32_kernel(const float *__restrict__ X, int64_t N, int Din, const float *__restrict__ mean,
               const float *__restrict__ P, int m, const float *__restrict__ xy, float *__restrict__ Y, int D) {
    extern __shared__ float fsm[];
    const int ldk = Din + 1;
    float *Xs = fsm, *Ps = fsm + kF32Rows * ldk;
    const int64_t row0 = (int64_t)blockIdx.x * kF32Rows;
    for (int i = threadIdx.x; i < kF32Rows * Din; i += kPcaThreads) {
        const int r = i / Din, k = i % Din;
        const int64_t row = row0 + r;
        Xs[r * ldk + k] = row < N ? X[row * Din + k] - mean[k] : 0.f;
    }
    for (int i = threadIdx.x; i < 80 * Din; i += kPcaThreads) {
        const int n = i / Din, k = i % Din;
        Ps[n * ldk + k] = n < m ? P[(size_t)n * Din + k] : 0.f;
    }
    __syncthreads();
    const int rb = (threadIdx.x >> 4) * 4, nb = threadIdx.x & 15;
    float acc[4][5];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 5; ++b) acc[a][b] = 0.f;
    for (int k = 0; k < Din; ++k) {
        float xv[4], pv[5];
#pragma unroll
        for (int a = 0; a < 4; ++a) xv[a] = Xs[(rb + a) * ldk + k];
#pragma unroll
        for (int b = 0; b < 5; ++b) pv[b] = Ps[(nb + 16 * b) * ldk + k];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 5; ++b) acc[a][b] = fmaf(xv[a], pv[b], acc[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t row = row0 + rb + a;
        if (row >= N) continue;
#pragma unroll
        for (int b = 0; b < 5; ++b) {
            const int n = nb + 16 * b;
            if (n < m) Y[row * D + n] = acc[a][b];
        }
        if (xy && nb < 2) Y[row * D + m + nb] = xy[2 * row + nb];
    }
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t bf16_smem(const fv_pca *p) {   // basis image, rows image, two mbarriers and the TMEM slot
    return (size_t)2 * (p->Din / 16) * p->Npad * 32 + (size_t)2 * (p->Din / 16) * kPcaRows * 32 + 32;
}

}  // namespace

// Project N rows into Y (device): FP32 rows of pitch D (bf16 = false) or
// bfloat16 rows of pitch ld (bf16 = true). err: device word (BF16 form).
cudaError_t launch_pca(const fv_pca *p, const float *X, const float *xy, int64_t N, bool bf16, void *Y, int ld,
                       uint32_t *err, cudaStream_t st, const float *yp, const DsPlan *dsp) {
    if (N <= 0) return cudaSuccess;
    if (!bf16) {
        const size_t smem = sizeof(float) * (size_t)(kF32Rows + 80) * (p->Din + 1);
        cudaError_t e = cudaFuncSetAttribute(pca_f32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        KernelTimer kt_("pca_f32", st);
        pca_f32_kernel<<<(unsigned)((N + kF32Rows - 1) / kF32Rows), kPcaThreads, smem, st>>>(
            X, N, p->Din, p->mean, p->basis, p->m, xy, (float *)Y, p->m + (xy ? 2 : 0));
        return cudaGetLastError();
    }
    const size_t smem = bf16_smem(p);
    const bool gather = yp != nullptr;
    if (gather && (p->Din != 128 || !dsp)) return cudaErrorInvalidValue;
    auto kern = gather ? pca_bf16_kernel<true> : pca_bf16_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const DsPlan none{};
    {
        KernelTimer kt_("pca_bf16", st);
        kern<<<(unsigned)((N + kPcaRows - 1) / kPcaRows), kPcaThreads, smem, st>>>(
            X, N, p->Din, p->mean, p->bimg, p->Npad, p->m, xy, (uint16_t *)Y, ld, err, yp, gather ? *dsp : none);
    }
    return cudaGetLastError();
}

}  // namespace fv

using namespace fv;

extern "C" int fv_pca_load(const float *basis, const float *mean, int m, int Din, fv_pca **out) {
    if (!out) return fail(FV_ERR_INVALID, "fv_pca_load: out is NULL");
    *out = nullptr;
    if (!basis) return fail(FV_ERR_INVALID, "fv_pca_load: NULL basis");
    if (m < 1 || m > 78) return fail(FV_ERR_UNSUPPORTED, "fv_pca_load: m must be in 1..78 (D = m + 2 <= 80)");
    if (Din < 16 || Din > 256 || Din % 16 != 0)
        return fail(FV_ERR_UNSUPPORTED, "fv_pca_load: Din must be a multiple of 16 in 16..256");
    for (size_t i = 0; i < (size_t)m * Din; ++i)
        if (!std::isfinite(basis[i])) return fail(FV_ERR_INVALID, "fv_pca_load: basis must be finite");
    if (mean)
        for (int i = 0; i < Din; ++i)
            if (!std::isfinite(mean[i])) return fail(FV_ERR_INVALID, "fv_pca_load: mean must be finite");
    fv_pca *p = new fv_pca();
    p->m = m;
    p->Din = Din;
    p->Npad = round_up(m, 16);
    cudaGetDevice(&p->device);
    const size_t b_basis = sizeof(float) * (size_t)m * Din, b_mean = sizeof(float) * Din;
    const size_t b_img = sizeof(uint16_t) * 2 * (size_t)(Din / 16) * p->Npad * 16;
    const size_t o_mean = (b_basis + 255) / 256 * 256, o_img = o_mean + (b_mean + 255) / 256 * 256;
    char *base = nullptr;
    cudaError_t e = cudaMalloc(&base, o_img + b_img);
    if (e != cudaSuccess) {
        delete p;
        return fail(FV_ERR_OOM, std::string("fv_pca_load: cudaMalloc: ") + cudaGetErrorString(e));
    }
    p->block = base;
    p->basis = (float *)base;
    p->mean = (float *)(base + o_mean);
    p->bimg = (uint16_t *)(base + o_img);
    std::vector<float> mz(Din, 0.f);
    e = cudaMemcpy(p->basis, basis, b_basis, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(p->mean, mean ? mean : mz.data(), b_mean, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        {
            KernelTimer kt_("pca_bimg", nullptr);
            pca_bimg_kernel<<<p->Npad, 128>>>(p->basis, m, Din, p->Npad, p->bimg);
        }
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(base);
        delete p;
        return cuda_fail(e, "fv_pca_load");
    }
    *out = p;
    return FV_OK;
}

extern "C" int fv_pca_info(const fv_pca *p, int *m, int *Din) {
    if (!p) return fail(FV_ERR_INVALID, "fv_pca_info: NULL handle");
    if (m) *m = p->m;
    if (Din) *Din = p->Din;
    return FV_OK;
}

extern "C" void fv_pca_free(fv_pca *p) {
    if (!p) return;
    cudaFree(p->block);
    delete p;
}

extern "C" int fv_pca_project(const fv_pca *p, const float *X, const float *xy, int64_t N, void *Y, int y_bf16,
                              int64_t ld_y, void *cuda_stream) {
    if (!p || !X || !Y) return fail(FV_ERR_INVALID, "fv_pca_project: NULL argument");
    if (N <= 0) return fail(FV_ERR_EMPTY, "fv_pca_project: no descriptors");
    const int D = p->m + (xy ? 2 : 0);
    if (!dev_ptr(X) || !dev_ptr(Y) || (xy && !dev_ptr(xy)))
        return fail(FV_ERR_INVALID, "fv_pca_project: X, xy and Y must be device memory");
    if (((uintptr_t)X) % 16 != 0) return fail(FV_ERR_INVALID, "fv_pca_project: X must be 16-byte aligned");
    if (y_bf16 && (ld_y < D || ld_y % 16 != 0 || ((uintptr_t)Y) % 16 != 0))
        return fail(FV_ERR_INVALID, "fv_pca_project: bfloat16 rows need ld_y >= D, a multiple of 16, 16-byte aligned");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    uint32_t *err = nullptr;
    cudaError_t e = cudaSuccess;
    if (y_bf16) {
        if ((e = cudaMallocAsync((void **)&err, 16, st)) != cudaSuccess) return cuda_fail(e, "fv_pca_project: scratch");
        cudaMemsetAsync(err, 0, 4, st);
    }
    e = launch_pca(p, X, xy, N, y_bf16 != 0, Y, (int)ld_y, err, st);
    if (err) cudaFreeAsync(err, st);
    if (e != cudaSuccess) return cuda_fail(e, "fv_pca_project: launch");
    return FV_OK;
}
