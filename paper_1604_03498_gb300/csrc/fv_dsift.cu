// Dense SIFT on the GPU (the descriptor step of Sec. 3.1; "Dense SIFT on
// GPU" of Sec. 3.2; the 8-scale pyramid of Sec. 4), flat-window variant:
//
//   1. pyramid: scales s_j = 2^((e - j)/2), j < n (e = 1, n = 8 by default),
//      floor(H s + 1/2) x floor(W s + 1/2) pixels sampled bilinearly at
//      ((u + 0.5)/s - 0.5, (v + 0.5)/s - 0.5), coordinates clamped;
//   2. gradients: central differences inside, one-sided on the border;
//   3. 8 orientation bins: theta / (2 pi / 8) = t, the magnitude split
//      linearly between bins floor(t) and floor(t) + 1 (mod 8);
//   4. the separable triangle k(d) = 1 - |d|/b (f = 2b - 1 taps) along x,
//      then along y, zero outside the image;
//   5. descriptors on a stride-S grid, x0 = 2b + S i <= W - 2b, bin (bx, by)
//      read at (x0 + (bx - 1.5) b, y0 + (by - 1.5) b), entry (4 by + bx) 8 + o;
//   6. L2-normalise, cap at 0.2, L2-normalise (zero stays zero);
//   7. positions (x0 / W_s - 0.5, y0 / H_s - 0.5).
//
// The paper computes the triangular convolution as two passes in which every
// output point sums its f inputs directly (its "combined step" that replaces
// the four scans), and computes the second pass only at the pixels the
// descriptors read (its unused-pixel skip). Here both passes skip: with S
// dividing b every bin centre lies on the column lattice b/2 + S t and the
// row lattice b/2 + S t, so
//   kernel 1 resamples every scale of every frame (one launch),
//   kernel 2 computes, for every row and lattice column only, the gradients of
//            the 2b - 1 pixels around it, their orientation split and the
//            x-pass sum (8 channels),
//   kernel 3 computes the y-pass once at every lattice point (row
//            b/2 + S m, column b/2 + S t), the 8 channels' sums over the
//            2b - 1 rows around it (a bin centre is shared by up to 16
//            descriptors),
//   kernel 4 gives one warp to a descriptor: each lane reads 4 of the 128
//            entries (one 16-byte load from the y-pass buffer), then the warp
//            normalises.
// fv_encode_images in the BF16 form skips kernel 4: the PCA projection reads
// each descriptor's 16 bins from the y-pass buffer and normalises them itself,
// so the FP32 descriptors are never written out.
#include <cmath>
#include <string>
#include <vector>

#include "fv_dsift.h"
#include "fv_internal.h"

namespace fv {
namespace {

int plan_dsift(int H, int W, const fv_dsift_params *prm, DsPlan &p) {
    fv_dsift_params d{4, 4, 8, 1};
    if (prm) d = *prm;
    if (d.bin_size < 2 || d.bin_size > 16 || d.bin_size % 2 != 0)
        return fail(FV_ERR_INVALID, "dense SIFT: bin_size must be even, 2..16");
    if (d.stride < 1 || d.bin_size % d.stride != 0) return fail(FV_ERR_INVALID, "dense SIFT: stride must divide bin_size");
    if (d.n_scales < 1 || d.n_scales > kMaxScales) return fail(FV_ERR_INVALID, "dense SIFT: n_scales must be 1..9");
    if (d.top_scale < -16 || d.top_scale > 4) return fail(FV_ERR_INVALID, "dense SIFT: top_scale must be -16..4");
    if (H < 1 || W < 1 || H > 16384 || W > 16384) return fail(FV_ERR_INVALID, "dense SIFT: image size 1..16384");
    p.n = d.n_scales;
    p.b = d.bin_size;
    p.S = d.stride;
    p.pyr = p.tmp = p.ndesc = p.npix = p.yp = p.nlat = 0;
    for (int j = 0; j < p.n; ++j) {
        const double s = std::pow(2.0, (d.top_scale - j) / 2.0);
        DsScale &c = p.s[j];
        c.Hs = (int)std::floor(H * s + 0.5);
        c.Ws = (int)std::floor(W * s + 0.5);
        c.inv_s = (float)(1.0 / s);
        c.nx = c.Ws - 2 * p.b >= 2 * p.b ? (c.Ws - 4 * p.b) / p.S + 1 : 0;
        c.ny = c.Hs - 2 * p.b >= 2 * p.b ? (c.Hs - 4 * p.b) / p.S + 1 : 0;
        if (c.nx == 0 || c.ny == 0) c.nx = c.ny = 0;
        c.Tx = c.nx > 0 ? c.nx + 3 * p.b / p.S : 0;
        c.Ty = c.ny > 0 ? c.ny + 3 * p.b / p.S : 0;
        c.img_off = p.pyr;
        c.tmp_off = p.tmp;
        c.desc_off = p.ndesc;
        c.pix_off = p.npix;
        c.yp_off = p.yp;
        c.lat_off = p.nlat;
        p.pyr += (int64_t)c.Hs * c.Ws;
        p.tmp += (int64_t)8 * c.Hs * c.Tx;
        p.ndesc += (int64_t)c.ny * c.nx;
        p.npix += (int64_t)c.Hs * c.Tx;
        p.yp += (int64_t)8 * c.Ty * c.Tx;
        p.nlat += (int64_t)c.Ty * c.Tx;
    }
    return FV_OK;
}

// grid (ceil(pyr / 256), B): every pixel of every scale of every frame.
__global__ void __launch_bounds__(256)
dsift_resize_kernel(const float *__restrict__ img, int H, int W, DsPlan p, float *__restrict__ pyr) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= p.pyr) return;
    const int f = blockIdx.y;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < p.n; ++q)
        if (i >= p.s[q].img_off) j = q;
    const DsScale &c = p.s[j];
    const int64_t k = i - c.img_off;
    const int v = (int)(k / c.Ws), u = (int)(k - (int64_t)v * c.Ws);
    const float y = fminf(fmaxf((v + 0.5f) * c.inv_s - 0.5f, 0.f), (float)(H - 1));
    const float x = fminf(fmaxf((u + 0.5f) * c.inv_s - 0.5f, 0.f), (float)(W - 1));
    const int y0 = (int)floorf(y), x0 = (int)floorf(x);
    const int y1 = min(y0 + 1, H - 1), x1 = min(x0 + 1, W - 1);
    const float fy = y - (float)y0, fx = x - (float)x0;
    const float *im = img + (size_t)f * H * W;
    const float top = (1.f - fx) * im[(size_t)y0 * W + x0] + fx * im[(size_t)y0 * W + x1];
    const float bot = (1.f - fx) * im[(size_t)y1 * W + x0] + fx * im[(size_t)y1 * W + x1];
    pyr[(size_t)f * p.pyr + i] = (1.f - fy) * top + fy * bot;
}

// grid (ceil(npix / 256), B): x-pass at every (row, lattice column).
__global__ void __launch_bounds__(256)
dsift_xpass_kernel(const float *__restrict__ pyr, DsPlan p, float *__restrict__ tmp) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= p.npix) return;
    const int f = blockIdx.y;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < p.n; ++q)
        if (i >= p.s[q].pix_off) j = q;
    const DsScale &c = p.s[j];
    const int64_t k = i - c.pix_off;
    const int y = (int)(k / c.Tx), t = (int)(k - (int64_t)y * c.Tx);
    const int b = p.b, Hs = c.Hs, Ws = c.Ws;
    const int cx = b / 2 + p.S * t;
    const float *im = pyr + (size_t)f * p.pyr + c.img_off;
    const float *row = im + (size_t)y * Ws;
    const float *up = im + (size_t)(y > 0 ? y - 1 : y) * Ws;
    const float *dn = im + (size_t)(y < Hs - 1 ? y + 1 : y) * Ws;
    const float ys = (y > 0 && y < Hs - 1) ? 0.5f : 1.f;   // central or one-sided difference
    const float k2pi = 1.27323954473516268615f;             // 8 / (2 pi)
    float acc[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) acc[o] = 0.f;
    for (int d = -(b - 1); d <= b - 1; ++d) {
        const int x = cx + d;
        if (x < 0 || x >= Ws) continue;
        float gx;
        if (Ws == 1) gx = 0.f;
        else if (x == 0) gx = row[1] - row[0];
        else if (x == Ws - 1) gx = row[Ws - 1] - row[Ws - 2];
        else gx = 0.5f * (row[x + 1] - row[x - 1]);
        const float gy = Hs == 1 ? 0.f : ys * (dn[x] - up[x]);
        const float m = sqrtf(gx * gx + gy * gy);
        float th = atan2f(gy, gx);
        if (th < 0.f) th += 6.28318530717958647692f;
        const float tt = th * k2pi;
        const float fl = floorf(tt);
        const float fr = tt - fl;
        const int b0 = ((int)fl) & 7, b1 = (b0 + 1) & 7;
        const float kw = 1.f - fabsf((float)d) / (float)b;
        const float w0 = kw * m * (1.f - fr), w1 = kw * m * fr;
#pragma unroll
        for (int o = 0; o < 8; ++o) acc[o] += (o == b0 ? w0 : 0.f) + (o == b1 ? w1 : 0.f);
    }
    float *out = tmp + (size_t)f * p.tmp + c.tmp_off + (size_t)y * c.Tx + t;
#pragma unroll
    for (int o = 0; o < 8; ++o) out[(size_t)o * Hs * c.Tx] = acc[o];
}

// grid (ceil(nlat / 256), B): y-pass at every lattice point (m, t), all 8
// channels, the taps in the same order as a per-descriptor sum would take them.
__global__ void __launch_bounds__(256)
dsift_ypass_kernel(const float *__restrict__ tmp, DsPlan p, float *__restrict__ yp) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= p.nlat) return;
    const int f = blockIdx.y;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < p.n; ++q)
        if (i >= p.s[q].lat_off) j = q;
    const DsScale &c = p.s[j];
    const int64_t k = i - c.lat_off;
    const int m = (int)(k / c.Tx), t = (int)(k - (int64_t)m * c.Tx);
    const int b = p.b, cy = b / 2 + p.S * m;
    const float *src = tmp + (size_t)f * p.tmp + c.tmp_off + t;
    float v[8];
#pragma unroll
    for (int o = 0; o < 8; ++o) v[o] = 0.f;
    for (int d = -(b - 1); d <= b - 1; ++d) {
        const int y = cy + d;
        if (y < 0 || y >= c.Hs) continue;
        const float kw = 1.f - fabsf((float)d) / (float)b;
#pragma unroll
        for (int o = 0; o < 8; ++o) v[o] = fmaf(kw, src[((size_t)o * c.Hs + y) * c.Tx], v[o]);
    }
    float4 *out = reinterpret_cast<float4 *>(yp + (size_t)f * p.yp + c.yp_off + (size_t)k * 8);
    out[0] = make_float4(v[0], v[1], v[2], v[3]);
    out[1] = make_float4(v[4], v[5], v[6], v[7]);
}

// grid (ceil(ndesc / 8), B), block 256: one warp per descriptor.
__global__ void __launch_bounds__(256)
dsift_desc_kernel(const float *__restrict__ yp, DsPlan p, float *__restrict__ desc, float *__restrict__ xy) {
    const int64_t i = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= p.ndesc) return;
    const int f = blockIdx.y;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < p.n; ++q)
        if (i >= p.s[q].desc_off) j = q;
    const DsScale &c = p.s[j];
    const int64_t k = i - c.desc_off;
    const int iy = (int)(k / c.nx), ix = (int)(k - (int64_t)iy * c.nx);
    const int b = p.b, bs = b / p.S;
    const int bin = lane >> 1, by = bin >> 2, bx = bin & 3, o0 = (lane & 1) * 4;
    // the bin's centre (x0 + (bx - 1.5) b, y0 + (by - 1.5) b) is lattice point (iy + by bs, ix + bx bs)
    const int m = iy + by * bs, t = ix + bx * bs;
    const float4 w4 = *reinterpret_cast<const float4 *>(yp + (size_t)f * p.yp + c.yp_off + ((size_t)m * c.Tx + t) * 8 + o0);
    float v[4] = {w4.x, w4.y, w4.z, w4.w};
    float ss = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (ss > 0.f) {
        const float inv = 1.f / sqrtf(ss);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = fminf(v[e] * inv, 0.2f);
        float s2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
        const float inv2 = 1.f / sqrtf(s2);
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] *= inv2;
    }
    const size_t row = (size_t)f * p.ndesc + i;
    *reinterpret_cast<float4 *>(desc + row * 128 + lane * 4) = make_float4(v[0], v[1], v[2], v[3]);
    if (xy && lane == 0) {
        const int x0 = 2 * b + p.S * ix, y0 = 2 * b + p.S * iy;
        xy[row * 2] = (float)x0 / (float)c.Ws - 0.5f;
        xy[row * 2 + 1] = (float)y0 / (float)c.Hs - 0.5f;
    }
}

// grid (ceil(ndesc / 256), B): positions only (the fused images path, whose
// descriptors are assembled inside the PCA projection).
__global__ void __launch_bounds__(256)
dsift_xy_kernel(DsPlan p, float *__restrict__ xy) {
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= p.ndesc) return;
    const int f = blockIdx.y;
    int j = 0;
#pragma unroll 1
    for (int q = 1; q < p.n; ++q)
        if (i >= p.s[q].desc_off) j = q;
    const DsScale &c = p.s[j];
    const int64_t k = i - c.desc_off;
    const int iy = (int)(k / c.nx), ix = (int)(k - (int64_t)iy * c.nx);
    const int x0 = 2 * p.b + p.S * ix, y0 = 2 * p.b + p.S * iy;
    const size_t row = (size_t)f * p.ndesc + i;
    xy[row * 2] = (float)x0 / (float)c.Ws - 0.5f;
    xy[row * 2 + 1] = (float)y0 / (float)c.Hs - 0.5f;
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Scratch of the lattice stages for B frames: pyramid, x-pass, y-pass (16-byte aligned).
size_t lattice_floats(const DsPlan &p, int B) { return (size_t)B * (p.pyr + p.tmp + p.yp) + 4; }
float *lattice_yp(float *buf, const DsPlan &p, int B) {
    float *tmp_end = buf + (size_t)B * (p.pyr + p.tmp);
    return reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(tmp_end) + 15) & ~uintptr_t(15));
}

// Resampling, x-pass and y-pass of B device frames into buf (lattice_floats floats).
cudaError_t run_lattice(const float *img, int B, int H, int W, const DsPlan &p, float *buf, cudaStream_t st) {
    float *pyr = buf, *tmp = buf + (size_t)B * p.pyr, *yp = lattice_yp(buf, p, B);
    {
        KernelTimer kt_("dsift_resize", st);
        dsift_resize_kernel<<<dim3((unsigned)((p.pyr + 255) / 256), (unsigned)B), 256, 0, st>>>(img, H, W, p, pyr);
    }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        KernelTimer kt_("dsift_xpass", st);
        dsift_xpass_kernel<<<dim3((unsigned)((p.npix + 255) / 256), (unsigned)B), 256, 0, st>>>(pyr, p, tmp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        KernelTimer kt_("dsift_ypass", st);
        dsift_ypass_kernel<<<dim3((unsigned)((p.nlat + 255) / 256), (unsigned)B), 256, 0, st>>>(tmp, p, yp);
        e = cudaGetLastError();
    }
    return e;
}

// The four kernels over B device frames into device desc / xy.
int run_dsift(const float *img, int B, int H, int W, const DsPlan &p, float *desc, float *xy, cudaStream_t st) {
    if (p.ndesc == 0) return FV_OK;
    float *buf = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(float) * lattice_floats(p, B), st);
    if (e != cudaSuccess) return cuda_fail(e, "dense SIFT: cudaMallocAsync(scratch)");
    e = run_lattice(img, B, H, W, p, buf, st);
    if (e == cudaSuccess) {
        KernelTimer kt_("dsift_desc", st);
        dsift_desc_kernel<<<dim3((unsigned)((p.ndesc + 7) / 8), (unsigned)B), 256, 0, st>>>(lattice_yp(buf, p, B), p,
                                                                                           desc, xy);
        e = cudaGetLastError();
    }
    cudaFreeAsync(buf, st);
    if (e != cudaSuccess) return cuda_fail(e, "dense SIFT: launch");
    return FV_OK;
}

// Frames on the device: the caller's, or a stream-ordered copy of host frames.
int stage_frames(const float *images, int B, int H, int W, int on_device, cudaStream_t st, const float **d,
                 float **owned) {
    *owned = nullptr;
    if (on_device) {
        if (!dev_ptr(images)) return fail(FV_ERR_INVALID, "images_on_device=1 but images is not device memory");
        *d = images;
        return FV_OK;
    }
    const size_t bytes = sizeof(float) * (size_t)B * H * W;
    cudaError_t e = cudaMallocAsync((void **)owned, bytes, st);
    if (e != cudaSuccess) return cuda_fail(e, "dense SIFT: cudaMallocAsync(images)");
    if ((e = cudaMemcpyAsync(*owned, images, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
        return cuda_fail(e, "dense SIFT: cudaMemcpyAsync(images)");
    *d = *owned;
    return FV_OK;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" int fv_dsift_count(int H, int W, const fv_dsift_params *params, int64_t *n_per_image) {
    DsPlan p;
    int rc = plan_dsift(H, W, params, p);
    if (rc != FV_OK) return rc;
    if (n_per_image) *n_per_image = p.ndesc;
    return FV_OK;
}

extern "C" int fv_dsift(const float *images, int B, int H, int W, int images_on_device, const fv_dsift_params *params,
                        float *desc, float *xy, void *cuda_stream) {
    if (!images || !desc) return fail(FV_ERR_INVALID, "fv_dsift: NULL images or descriptor output");
    if (B < 1) return fail(FV_ERR_INVALID, "fv_dsift: B must be >= 1");
    DsPlan p;
    int rc = plan_dsift(H, W, params, p);
    if (rc != FV_OK) return rc;
    if (!dev_ptr(desc) || (xy && !dev_ptr(xy)) || ((uintptr_t)desc) % 16 != 0)
        return fail(FV_ERR_INVALID, "fv_dsift: desc (16-byte aligned) and xy must be device memory");
    if (p.ndesc == 0) return fail(FV_ERR_EMPTY, "fv_dsift: the image is too small for one descriptor");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float *d = nullptr;
    float *owned = nullptr;
    rc = stage_frames(images, B, H, W, images_on_device, st, &d, &owned);
    if (rc == FV_OK) rc = run_dsift(d, B, H, W, p, desc, xy, st);
    if (owned) cudaFreeAsync(owned, st);
    return rc;
}

extern "C" int fv_encode_images(const fv_gmm *gmm, const fv_pca *pca, const float *images, int B, int H, int W,
                                int images_on_device, const fv_dsift_params *params, float *fv_out, int out_on_device,
                                void *cuda_stream) {
    if (!gmm || !pca || !images || !fv_out) return fail(FV_ERR_INVALID, "fv_encode_images: NULL argument");
    if (B < 1) return fail(FV_ERR_INVALID, "fv_encode_images: B must be >= 1");
    int m = 0, Din = 0;
    fv_pca_info(pca, &m, &Din);
    if (Din != 128) return fail(FV_ERR_INVALID, "fv_encode_images: the PCA must take 128-dimensional descriptors");
    DsPlan p;
    int rc = plan_dsift(H, W, params, p);
    if (rc != FV_OK) return rc;
    if (p.ndesc == 0) return fail(FV_ERR_EMPTY, "fv_encode_images: the image is too small for one descriptor");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    const float *d = nullptr;
    float *owned = nullptr, *buf = nullptr;
    rc = stage_frames(images, B, H, W, images_on_device, st, &d, &owned);
    const size_t n = (size_t)B * p.ndesc;
    std::vector<int64_t> offs(B + 1);
    for (int b = 0; b <= B; ++b) offs[b] = (int64_t)b * p.ndesc;
    if (is_bf16(gmm->prec)) {
        // BF16 form: the PCA projection assembles and normalises each descriptor
        // from the y-pass buffer itself; only the positions are written here
        const size_t lat = lattice_floats(p, B);
        if (rc == FV_OK) {
            cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(float) * (lat + n * 2), st);
            if (e != cudaSuccess) rc = cuda_fail(e, "fv_encode_images: cudaMallocAsync(scratch)");
        }
        float *xy = buf ? buf + lat : nullptr;
        if (rc == FV_OK) {
            cudaError_t e = run_lattice(d, B, H, W, p, buf, st);
            if (e == cudaSuccess) {
                KernelTimer kt_("dsift_xy", st);
                dsift_xy_kernel<<<dim3((unsigned)((p.ndesc + 255) / 256), (unsigned)B), 256, 0, st>>>(p, xy);
                e = cudaGetLastError();
            }
            if (e != cudaSuccess) rc = cuda_fail(e, "fv_encode_images: dense SIFT launch");
        }
        if (rc == FV_OK)
            rc = encode_pca_impl(gmm, pca, nullptr, xy, offs.data(), B, 1, fv_out, out_on_device, cuda_stream,
                                 lattice_yp(buf, p, B), &p);
    } else {
        if (rc == FV_OK) {
            cudaError_t e = cudaMallocAsync((void **)&buf, sizeof(float) * n * 130, st);
            if (e != cudaSuccess) rc = cuda_fail(e, "fv_encode_images: cudaMallocAsync(descriptors)");
        }
        if (rc == FV_OK) rc = run_dsift(d, B, H, W, p, buf, buf + n * 128, st);
        if (rc == FV_OK)
            rc = fv_encode_pca(gmm, pca, buf, buf + n * 128, offs.data(), B, 1, fv_out, out_on_device, cuda_stream);
    }
    if (buf) cudaFreeAsync(buf, st);
    if (owned) cudaFreeAsync(owned, st);
    return rc;
}
