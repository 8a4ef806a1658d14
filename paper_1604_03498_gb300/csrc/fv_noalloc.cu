// fv_encode_noalloc: the plain FP32 encoder for callers that cannot allocate
// device memory.
//
// Some callers may not allocate at all. Examples: an application whose own
// allocator already owns (nearly) all device memory, where an extra pool
// allocation fails or fragments; a latency-critical loop where growing a
// memory pool could stall; a process under a fixed device-memory quota. For
// them this entry point takes its scratch (posteriors, per-range statistics,
// work list, squared norms) from one file-scope __device__ array of
// kNoAllocScratchBytes and calls no allocating routine (no cudaMalloc,
// cudaMallocAsync, cudaHostAlloc, cudaFree or library allocation).
//
// The array lives in every GPU that loads this library until the process
// exits. Every call shares it and it keeps the last call's contents: calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it and must be serialised by the caller. Nothing in it has
// to start at zero: the kernels write every element they later read.
//
// In host code the array's name is only a host-side stand-in, so the device
// address is looked up once per device with cudaGetSymbolAddress, with that
// device current, on the first call made on the device.
#include <algorithm>
#include <mutex>
#include <string>

#include "fv_internal.h"

namespace fv {
namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_na_mu;
void *g_na_ptr[64] = {nullptr};

// Device address of the scratch array on `dev` (the current device).
cudaError_t scratch_address(int dev, void **ptr) {
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev & 63]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_na_ptr[dev & 63] = p;
    }
    *ptr = g_na_ptr[dev & 63];
    return cudaSuccess;
}

// Work list of one frame: ranges of rpr rows, one statistics slot each.
__global__ void noalloc_plan_kernel(int64_t n, int64_t rpr, int nslots, FrameInfo *frame, StatUnit *units) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        frame->row0 = 0;
        frame->n = n;
        frame->slot0 = 0;
        frame->nslots = nslots;
    }
    if (i < nslots) {
        units[i].row0 = (int64_t)i * rpr;
        units[i].nrows = (int32_t)min(rpr, n - (int64_t)i * rpr);
        units[i].slot = i;
    }
}

size_t al256(size_t b) { return (b + 255) / 256 * 256; }

size_t scratch_bytes(int64_t N, int Kp, int K, int D, int P, int64_t nslots) {
    return al256(f32_gamma_bytes(N, Kp)) + al256(sizeof(float) * (size_t)nslots * Kp * P) +
           al256(sizeof(FrameInfo)) + al256(sizeof(StatUnit) * (size_t)nslots) + al256(sizeof(double) * (size_t)(Kp / 32) * ((D + 7) / 8));
}

bool device_pointer(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace fv

using namespace fv;

extern "C" int fv_encode_noalloc(const fv_gmm *gmm, const float *X, int64_t N, float *fv_out, void *cuda_stream) {
    if (!gmm || !fv_out) return fail(FV_ERR_INVALID, "fv_encode_noalloc: NULL GMM handle or output");
    if (gmm->prec != FV_PREC_FP32) return fail(FV_ERR_INVALID, "fv_encode_noalloc: needs an FV_PREC_FP32 GMM");
    if (N < 0 || (N > 0 && !X)) return fail(FV_ERR_INVALID, "fv_encode_noalloc: bad N or NULL descriptors");
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != gmm->device) return fail(FV_ERR_INVALID, "fv_encode_noalloc: GMM handle belongs to another device");
    if ((N > 0 && !device_pointer(X)) || !device_pointer(fv_out))
        return fail(FV_ERR_INVALID, "fv_encode_noalloc: descriptors and output must be device memory");

    const int K = gmm->K, D = gmm->D, Kp = gmm->Kp, P = 2 * D + 1;
    // statistics ranges: about three blocks per SM, widened until the scratch fits
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t rows = N > 0 ? N : 1;
    const int64_t per_range = (int64_t)(Kp / 64) * ((D + 63) / 64);
    int64_t rpr = std::max<int64_t>(64, round_up64((rows * per_range + 3LL * sms - 1) / (3LL * sms), 32));
    int64_t nslots = (rows + rpr - 1) / rpr;
    while (scratch_bytes(rows, Kp, K, D, P, nslots) > kNoAllocScratchBytes && nslots > 1) {
        rpr *= 2;
        nslots = (rows + rpr - 1) / rpr;
    }
    if (scratch_bytes(rows, Kp, K, D, P, nslots) > kNoAllocScratchBytes)
        return fail(FV_ERR_UNSUPPORTED,
                    "fv_encode_noalloc: N=" + std::to_string(N) + " with K=" + std::to_string(K) + ", D=" +
                        std::to_string(D) + " needs more than the fixed 32 MiB scratch (posteriors alone take N*" +
                        std::to_string(Kp) + "*4 bytes); use fv_encode");

    void *base = nullptr;
    cudaError_t e = scratch_address(dev, &base);
    if (e != cudaSuccess) return cuda_fail(e, "fv_encode_noalloc: cudaGetSymbolAddress");
    char *b = (char *)base;
    float *gam = (float *)b;
    b += al256(f32_gamma_bytes(rows, Kp));
    float *part = (float *)b;
    b += al256(sizeof(float) * (size_t)nslots * Kp * P);
    FrameInfo *frame = (FrameInfo *)b;
    b += al256(sizeof(FrameInfo));
    StatUnit *units = (StatUnit *)b;
    b += al256(sizeof(StatUnit) * (size_t)nslots);
    double *sq = (double *)b;

    const int nunits = N > 0 ? (int)nslots : 0;
    {
        KernelTimer kt_("noalloc_plan", st);
        noalloc_plan_kernel<<<(unsigned)((nslots + 127) / 128), 128, 0, st>>>(N, rpr, nunits, frame, units);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fv_encode_noalloc: plan launch");
    if (N > 0) {
        if ((e = launch_f32_posteriors(gmm, X, N, gam, st)) != cudaSuccess)
            return cuda_fail(e, "fv_encode_noalloc: posteriors launch");
        if ((e = launch_f32_stats(gmm, X, gam, N, units, nunits, part, P, st)) != cudaSuccess)
            return cuda_fail(e, "fv_encode_noalloc: statistics launch");
    }
    if ((e = launch_finalize(gmm, part, P, frame, 1, sq, fv_out, st, nullptr, nullptr, (int)nunits)) !=
        cudaSuccess)
        return cuda_fail(e, "fv_encode_noalloc: finalise launch");
    if (N == 0) return fail(FV_ERR_EMPTY, "no descriptors (N == 0)");
    return FV_OK;
}
