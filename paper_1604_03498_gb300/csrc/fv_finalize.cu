// Finalise: reduction of the per-range statistics copies (the paper's second
// Phase-2 kernel, Algorithm 3, adding the per-block copies of U and V)
// followed by the encoding scheme of Sec. 4: u = U/(N sqrt(w)),
// v = V/(N sqrt(2w)), signed square root, L2.
//
// Slots are component-fastest: part[slot][j][Kp], j indexing the statistic.
// Kernel R adds the frame's slots into its first slot in one canonical order:
// eight partial sums p_g over the slots s = g (mod 8) in increasing s, then
// p_0 + p_1 + ... + p_7 left to right. The order depends on nothing but the
// frame's own slots, so a frame's vector does not depend on what else was
// encoded with it. A block covers 32 components of one frame: with many
// slots, eight warps take one residue each for one statistic; with a few,
// each of eight warps takes a statistic and keeps the eight partials itself. Kernel A: one
// block per (32 components x 8 dimensions, frame) reads the totals, forms u
// and v, takes sign(z) sqrt|z|, and writes its [32][8] tiles through shared
// memory (runs of 8 contiguous floats); the block's sum of squares goes to
// sq. Kernel B: blocks of 1024 output values per frame each add the frame's
// block squares (the same fixed-order tree in every block) and scale their
// values by 1/||z||.
//
// All per-element arithmetic is FP32 (GB300's FP64 rate is a small fraction
// of its FP32 rate). Slots of both forms hold centred sums (the BF16 encoder
// centres its raw moments as it writes them out):
//   A = sum g (x - mu),  B = sum g (x - mu)^2,  S0 = sum g
//   u = A / sigma * alpha / N,    v = (B / sigma^2 - S0) * beta / N.
#include "fv_internal.h"

namespace fv {

namespace {

constexpr int FA_THREADS = 256;   // 32 components x 8 dimension lanes
constexpr int FB_THREADS = 256;   // one float4 each

__device__ __forceinline__ float ssqrtf(float v) { return v > 0.f ? sqrtf(v) : (v < 0.f ? -sqrtf(-v) : 0.f); }

// grid (ceil(P/J), Kp/32, frames), block 256: frame totals into the frame's
// first slot. split = true: J = 1, warp w sums residue w; split = false:
// J = 8, warp w sums statistic blockIdx.x * 8 + w over all residues.
__global__ void __launch_bounds__(256)
finalize_r_kernel(float *__restrict__ part, int P, int Kp, bool split, const FrameInfo *__restrict__ frames,
                  const int *__restrict__ B_dev) {
    __shared__ float red[8][32];
    pdl_wait();      // the statistics slots are complete
    pdl_trigger();
    const int f = blockIdx.z;
    if (B_dev && f >= *B_dev) return;
    const FrameInfo fr = frames[f];
    if (fr.n <= 0 || fr.nslots <= 1) return;   // nothing to add
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int n = fr.nslots;
    const size_t sstride = (size_t)P * Kp;
    if (split) {
        float *p = part + (size_t)fr.slot0 * sstride + (size_t)blockIdx.x * Kp + blockIdx.y * 32 + lane;
        float a = 0.f;
#pragma unroll 4
        for (int s = w; s < n; s += 8) a += p[(size_t)s * sstride];
        red[w][lane] = a;
        __syncthreads();
        if (w == 0) {
            float t = red[0][lane];
#pragma unroll
            for (int g = 1; g < 8; ++g) t += red[g][lane];
            p[0] = t;
        }
        return;
    }
    const int j = blockIdx.x * 8 + w;
    if (j >= P) return;
    float *p = part + (size_t)fr.slot0 * sstride + (size_t)j * Kp + blockIdx.y * 32 + lane;
    float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, a4 = 0.f, a5 = 0.f, a6 = 0.f, a7 = 0.f;
    int s = 0;
    for (; s + 8 <= n; s += 8) {
        a0 += p[(size_t)(s + 0) * sstride];
        a1 += p[(size_t)(s + 1) * sstride];
        a2 += p[(size_t)(s + 2) * sstride];
        a3 += p[(size_t)(s + 3) * sstride];
        a4 += p[(size_t)(s + 4) * sstride];
        a5 += p[(size_t)(s + 5) * sstride];
        a6 += p[(size_t)(s + 6) * sstride];
        a7 += p[(size_t)(s + 7) * sstride];
    }
    if (s + 0 < n) a0 += p[(size_t)(s + 0) * sstride];
    if (s + 1 < n) a1 += p[(size_t)(s + 1) * sstride];
    if (s + 2 < n) a2 += p[(size_t)(s + 2) * sstride];
    if (s + 3 < n) a3 += p[(size_t)(s + 3) * sstride];
    if (s + 4 < n) a4 += p[(size_t)(s + 4) * sstride];
    if (s + 5 < n) a5 += p[(size_t)(s + 5) * sstride];
    if (s + 6 < n) a6 += p[(size_t)(s + 6) * sstride];
    p[0] = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
}

// grid (Kp/32, ceil(D/8), frames); thread (lane -> component, grp -> dimension)
__global__ void __launch_bounds__(FA_THREADS)
finalize_a_kernel(const float *__restrict__ part, int P, int Kp, int K, int D, const FrameInfo *__restrict__ frames,
                  GmmDev g, double *__restrict__ sq, float *__restrict__ out, const int *__restrict__ B_dev) {
    __shared__ float tile[2][32][9];   // [u|v][component][dimension]
    __shared__ float red[FA_THREADS];
    pdl_wait();      // the frame totals are complete
    pdl_trigger();
    const int f = blockIdx.z;
    if (B_dev && f >= *B_dev) return;   // graph replay with fewer frames than the grid
    const int k0 = blockIdx.x * 32, d0 = blockIdx.y * 8;
    const int lane = threadIdx.x & 31, grp = threadIdx.x >> 5;
    const int k = k0 + lane, d = d0 + grp;
    const FrameInfo fr = frames[f];
    const size_t KD = (size_t)K * D;
    const size_t sstride = (size_t)P * Kp;
    float *o = out + (size_t)f * 2 * KD;

    float zu = 0.f, zv = 0.f;
    if (d < D && k < K && fr.n > 0) {
        const float *ps = part + (size_t)fr.slot0 * sstride + k;   // the frame totals
        const float S0 = ps[(size_t)(P - 1) * Kp];
        const float a = ps[(size_t)d * Kp];
        const float b = ps[(size_t)(D + d) * Kp];
        const float inv_n = 1.0f / (float)fr.n;
        const float al = g.alpha[k] * inv_n, be = g.beta[k] * inv_n;
        const float isd = g.s_t[(size_t)d * Kp + k], pr = g.prec_t[(size_t)d * Kp + k];
        const float u = a * isd * al;
        const float v = fmaf(b, pr, -S0) * be;
        zu = ssqrtf(u);
        zv = ssqrtf(v);
    }
    tile[0][lane][grp] = zu;
    tile[1][lane][grp] = zv;
    red[threadIdx.x] = fmaf(zu, zu, zv * zv);
    __syncthreads();
    // stores: 8 consecutive dimensions of one component per 8 lanes
    {
        const int dd = threadIdx.x & 7, kk = threadIdx.x >> 3;   // 32 components x 8 dimensions
        const int kw = k0 + kk, dw = d0 + dd;
        if (kw < K && dw < D) {
            o[(size_t)kw * D + dw] = tile[0][kk][dd];
            o[KD + (size_t)kw * D + dw] = tile[1][kk][dd];
        }
    }
    for (int s = FA_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) sq[((size_t)f * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = (double)red[0];
}

// grid (ceil(2KD / 1024), frames)
__global__ void __launch_bounds__(FB_THREADS)
finalize_b_kernel(int K, int D, int nb, const double *__restrict__ sq, float *__restrict__ out,
                  const uint32_t *__restrict__ err, const int *__restrict__ B_dev) {
    __shared__ float red[FB_THREADS];
    pdl_wait();      // the encoded values and block squares are complete
    const int f = blockIdx.y;
    if (B_dev && f >= *B_dev) return;
    // fixed-order FP32 tree over the frame's block sums (no FP64 on the hot path)
    float t = 0.f;
    for (int b = threadIdx.x; b < nb; b += FB_THREADS) t += (float)sq[(size_t)f * nb + b];
    red[threadIdx.x] = t;
    __syncthreads();
    for (int s = FB_THREADS / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    const float tot = red[0];
    const size_t n = (size_t)2 * K * D;
    float *o = out + (size_t)f * n;
    const size_t j0 = (size_t)blockIdx.x * FB_THREADS * 4 + threadIdx.x * 4;
    if (j0 >= n) return;
    const size_t j1 = j0 + 4 < n ? j0 + 4 : n;
    if (err && *err) {   // an earlier kernel of this call gave up: poison the output
        for (size_t j = j0; j < j1; ++j) o[j] = __int_as_float(0x7fc00000);
        return;
    }
    if (!(tot > 0.f)) return;   // all-zero vector stays zero
    const float inv = rsqrtf(tot);
    if (j1 == j0 + 4 && (reinterpret_cast<uintptr_t>(o + j0) & 15) == 0) {
        float4 v = *reinterpret_cast<float4 *>(o + j0);
        v.x *= inv;
        v.y *= inv;
        v.z *= inv;
        v.w *= inv;
        *reinterpret_cast<float4 *>(o + j0) = v;
    } else {
        for (size_t j = j0; j < j1; ++j) o[j] *= inv;
    }
}

}  // namespace

cudaError_t launch_slot_reduce(const fv_gmm *g, float *part, int P, const FrameInfo *frames, int B, int max_slots,
                               cudaStream_t st) {
    if (B <= 0) return cudaSuccess;
    const bool split = max_slots >= 16;
    const int J = split ? 1 : 8;
    {
        KernelTimer kt_("finalize_r", st);
        finalize_r_kernel<<<dim3((unsigned)((P + J - 1) / J), (unsigned)(g->Kp / 32), (unsigned)B), 256, 0, st>>>(
            part, P, g->Kp, split, frames, nullptr);
    }
    return cudaGetLastError();
}

cudaError_t launch_finalize(const fv_gmm *g, float *part, int P, const FrameInfo *frames,
                            int B, double *sq, float *out, cudaStream_t st, const uint32_t *err, const int *B_dev,
                            int max_slots, bool pdl) {
    if (B <= 0) return cudaSuccess;
    cudaError_t e;
    {
        // the split only changes which warps do the work, not the order
        const bool split = max_slots >= 16;
        const int J = split ? 1 : 8;
        KernelTimer kt_("finalize_r", st);
        e = launch_pdl(pdl, finalize_r_kernel, dim3((unsigned)((P + J - 1) / J), (unsigned)(g->Kp / 32), (unsigned)B),
                       dim3(256), 0, st, part, P, g->Kp, split, frames, B_dev);
    }
    if (e != cudaSuccess) return e;
    const int nbx = g->Kp / 32, nby = (g->D + 7) / 8, nb = nbx * nby;
    dim3 grid_a((unsigned)nbx, (unsigned)nby, (unsigned)B);
    {
        KernelTimer kt_("finalize_a", st);
        e = launch_pdl(pdl, finalize_a_kernel, grid_a, dim3(FA_THREADS),
                       0, st, (const float *)part, P, g->Kp, g->K, g->D, frames, g->dev, sq, out, B_dev);
    }
    if (e != cudaSuccess) return e;
    {
        KernelTimer kt_("finalize_b", st);
        const size_t n = (size_t)2 * g->K * g->D;
        const unsigned nbb = (unsigned)((n + FB_THREADS * 4 - 1) / (FB_THREADS * 4));
        e = launch_pdl(pdl, finalize_b_kernel, dim3(nbb, (unsigned)B), dim3(FB_THREADS), 0, st, g->K, g->D, nb,
                       (const double *)sq, out, err, B_dev);
    }
    return e;
}

}  // namespace fv
