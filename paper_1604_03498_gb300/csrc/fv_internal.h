// Internal declarations shared by the CUDA translation units of the encoder.
// Nothing here is part of the public ABI (include/fv.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fv.h"

namespace fv {

// ---- error reporting -------------------------------------------------------
void set_error(const std::string &msg);
int fail(int status, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define FV_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t e_ = (expr);                            \
        if (e_ != cudaSuccess) return ::fv::cuda_fail(e_, #expr); \
    } while (0)

// ---- instrumentation: launch counting and optional per-kernel event timing --
// Construct one KernelTimer right before each kernel launch and let it go out
// of scope right after: it counts the launch and, while profiling is enabled,
// records start/stop events on the launch stream.
class KernelTimer {
  public:
    KernelTimer(const char *name, cudaStream_t st);
    ~KernelTimer();
  private:
    int slot_;
    cudaStream_t st_;
};

// Adds kernel launches made by a graph replay to the launch counter.
void count_launches(int n);

// ---- limits ----------------------------------------------------------------
constexpr int kMaxK_F32 = 512;    // posteriors keep a BM x Kp row block in shared memory
constexpr int kMaxD_F32 = 1024;
constexpr int kMaxK_BF16 = 512;   // one 128-lane x K-column TMEM accumulator
constexpr int kMaxD_BF16 = 80;    // stats GEMM N = 3D + 16 <= 256
constexpr int kMaxD_BF16X2 = 64;  // hi + lo posteriors: the doubled gamma^T tile fits shared memory up to D = 64

inline int round_up(int a, int b) { return (a + b - 1) / b * b; }
// The tensor-core forms (FV_PREC_BF16 and FV_PREC_BF16X2) share operands and kernels.
inline bool is_bf16(int prec) { return prec == FV_PREC_BF16 || prec == FV_PREC_BF16X2; }
inline int64_t round_up64(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

// ---- GMM handle ------------------------------------------------------------
// Per-component operands, all computed on the device in FP64 from the FP32
// inputs by the preparation kernel (Algorithm 1, "compute sqrt(sigma^-1)").
struct GmmDev {
    // FP32 form
    float *s_t;      // [D][Kp]  1/sigma, component-contiguous (posteriors)
    float *nms_t;    // [D][Kp]  -mu/sigma
    float *cst;      // [Kp]     log w - 1/2 sum_d log sigma^2 (-inf on padding)
    float *s_kd;     // [Kp][Dp] 1/sigma, dimension-contiguous (statistics)
    float *mu_kd;    // [Kp][Dp] mu (statistics: t = (x - mu) / sigma)
    // shared by both forms (finalise), component-contiguous, FP32 rounded from
    // FP64 (zero on padding); 1/sigma of the finalise is s_t
    float *mu_t;     // [D][Kp] mu
    float *prec_t;   // [D][Kp] 1/sigma^2
    float *alpha;    // [Kp] 1/sqrt(w)
    float *beta;     // [Kp] 1/sqrt(2w)
    // BF16 form: B operands of the log-likelihood GEMM, [term][Kp][D16] bf16,
    // terms = Q_hi, Q_lo, R_hi, R_lo with Q = mu/sigma^2, R = -1/(2 sigma^2)
    uint16_t *bimg;
    float *cfull;    // [Kp] log w - 1/2 sum log sigma^2 - 1/2 sum mu^2/sigma^2 (FP64 -> FP32; -inf on padding)
    float *cl2;      // [Kp] cfull * log2(e), formed in FP64
    // the same constants before rounding: [0, Kp) log w - 1/2 sum log sigma^2,
    // [Kp, 2 Kp) minus 1/2 sum mu^2/sigma^2 (FP64; -inf on padding)
    double *c64;
    // the parameters as loaded (FP32): [K] weights, [K][D] means, [K][D]
    // variances (the preparation kernel's input)
    float *params;
};

}  // namespace fv

struct fv_pca;

struct fv_gmm {
    int K, D;
    int Kp;     // components padded (64 for FP32, 128 for BF16)
    int Dp;     // dimensions padded to 8 (FP32 statistics) / 16 (BF16)
    int prec;   // fv_precision
    int device;
    fv::GmmDev dev;
    void *block;   // single device allocation backing dev.*
    size_t block_bytes;
};

namespace fv {

// ---- work description shared by the kernels ---------------------------------
struct FrameInfo {
    int64_t row0;    // first row in the packed descriptor array
    int64_t n;       // descriptors in the frame
    int32_t slot0;   // first statistics slot of the frame
    int32_t nslots;  // number of row ranges (slots) of the frame
};

struct StatUnit {
    int64_t row0;    // first row of the range
    int32_t nrows;   // rows in the range
    int32_t slot;    // statistics slot written by this range
};

// Balanced work plan of the BF16 statistics (see fv_api.cu): G row shares,
// cut at frame boundaries into units; cta[c] = (first unit, count).
void build_balanced_plan(const int64_t *offsets, int B, int G, std::vector<FrameInfo> &frames,
                         std::vector<StatUnit> &units, std::vector<int2> &cta);

// ---- kernels' host launchers --------------------------------------------------
cudaError_t launch_prep(const fv_gmm *g, const float *w, const float *mu, const float *var, cudaStream_t st);

// Programmatic dependent launch (PDL): a kernel launched with launch_pdl may
// begin while the previous kernel on the stream is still running; it calls
// pdl_wait() before it reads anything that kernel writes (griddepcontrol.wait
// returns once the previous grid has completed and its memory is visible; it
// is a no-op for a normal launch). pdl_trigger() lets the next PDL kernel
// start launching early. The first kernel of a call is always launched
// normally, so nothing of a previous call can overlap it.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// The FP32 posteriors buffer: rows x Kp floats, then one 32-bit mask per row
// (bit j set when some posterior of components 16j .. 16j+15 is non-zero).
// Only the 16-component groups with a set bit are written; the statistics
// kernel reads only those and takes the others as the exact zeros they are.
inline size_t f32_gamma_bytes(int64_t rows, int Kp) {
    return sizeof(float) * (size_t)rows * Kp + sizeof(uint32_t) * (size_t)rows;
}
inline uint32_t *f32_gamma_mask(float *gamma, int64_t rows, int Kp) {
    return reinterpret_cast<uint32_t *>(gamma + (size_t)rows * Kp);
}

// lse (nullable): per-row log sum_k exp(l_ik), natural log (EM log-likelihood).
cudaError_t launch_f32_posteriors(const fv_gmm *g, const float *X, int64_t rows, float *gamma,
                                  cudaStream_t st, float *lse = nullptr);
// gamma: the posteriors buffer of all `rows` rows the units index.
// tau > 0: early termination (terms with posterior <= tau dropped, all-small
// rows skipped); skip_count (device, nullable): [skipped, visited] counters.
cudaError_t launch_f32_stats(const fv_gmm *g, const float *X, const float *gamma, int64_t rows,
                             const StatUnit *units, int n_units, float *part, int P, cudaStream_t st,
                             bool pdl = false, float tau = 0.f, unsigned long long *skip_count = nullptr);

// Statistics slots are component-fastest: part[slot][j][Kp], j < P.
// Finalise: reduce per-range statistics in a fixed order, scale, signed sqrt,
// L2. Slots of both forms hold the centred [A, B, S0] layout (blocks of D,
// P = 2D+1).
// sq needs B * (Kp / 32) * ceil(D / 8) doubles. Each frame's first slot is
// overwritten with the frame's totals (three launches: slot reduction,
// encode, normalise). max_slots: the most slots a frame has (any value is
// correct; it picks the reduction's split).
// err (nullable): device error word of the call; when a kernel set it, every
// output element becomes NaN so a failed encode can never look valid.
// Only the slot reduction of launch_finalize: every frame's slots summed
// into its first slot in the canonical order.
cudaError_t launch_slot_reduce(const fv_gmm *g, float *part, int P, const FrameInfo *frames, int B, int max_slots,
                               cudaStream_t st);
// PCA projection + position append (Sec. 3.1) of N rows into device Y:
// FP32 rows of pitch D (bf16 = false) or bfloat16 rows of pitch ld (bf16 =
// true, ld a multiple of 16); err: device word set if an MMA wait expired.
// yp / dsp (BF16 form, Din = 128): the rows are dense-SIFT descriptors
// assembled from the y-pass buffer yp of plan dsp instead of read from X.
struct DsPlan;
cudaError_t launch_pca(const fv_pca *p, const float *X, const float *xy, int64_t N, bool bf16, void *Y, int ld,
                       uint32_t *err, cudaStream_t st, const float *yp = nullptr, const DsPlan *dsp = nullptr);
// fv_encode_pca, or (yp != nullptr) the same on rows gathered from a dense-SIFT
// y-pass buffer (BF16 form, device memory, offsets = B frames of dsp->ndesc).
int encode_pca_impl(const fv_gmm *gmm, const fv_pca *pca, const float *X, const float *xy, const int64_t *offsets,
                    int B, int x_on_device, float *fv_out, int out_on_device, void *cuda_stream, const float *yp,
                    const DsPlan *dsp);
cudaError_t launch_finalize(const fv_gmm *g, float *part, int P,
                            const FrameInfo *frames, int B, double *sq, float *out, cudaStream_t st,
                            const uint32_t *err = nullptr, const int *B_dev = nullptr, int max_slots = 1,
                            bool pdl = false);

}  // namespace fv
