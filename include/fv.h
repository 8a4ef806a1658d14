/*
 * fv.h - C ABI of the GB300 Fisher-vector encoder.
 *
 * The library encodes sets of local descriptors against a diagonal-covariance
 * Gaussian mixture model into improved Fisher vectors, as stated in
 * "GPU-FV: Realtime Fisher Vector and Its Applications in Video Monitoring"
 * (Ma et al., ICMR 2016):
 *   - the problem statement, Sec. 3.1 and Algorithm 1: inputs are the
 *     descriptors and the GMM (means, "covariances" = diagonal variances,
 *     priors), output the Fisher vector {U, V};
 *   - posteriors (Algorithm 1 first loop; Algorithm 2 on the GPU);
 *   - first/second-order statistics U, V (Algorithm 1 second loop;
 *     Algorithm 3 with per-block copies and a reduction kernel);
 *   - the encoding scheme of Sec. 4 ("the same encoding scheme as VLFeat"):
 *     u_kd = U_kd / (N sqrt(w_k)), v_kd = V_kd / (N sqrt(2 w_k)), then the
 *     signed square root and L2 normalisation of z = [u; v].
 *
 * Notation: N descriptors of dimension D, K mixture components.
 * Fisher-vector layout (2*K*D floats): [u_0 .. u_{K-1}, v_0 .. v_{K-1}],
 * each u_k / v_k block D-contiguous. The paper writes the vector as {V, U};
 * the order here is a fixed permutation and is documented as such.
 *
 * Conventions for every call:
 *   - every entry point returns an fv_status and never aborts; on error
 *     fv_last_error() gives a thread-local message;
 *   - the caller owns all input and output buffers; the library copies what
 *     it keeps (the GMM at load time, submitted frames at submit time);
 *   - "on_device" flags say whether a pointer is device memory (1) or host
 *     memory (0). Host buffers may be pageable; pinned ones copy faster;
 *   - cuda_stream is a cudaStream_t (NULL = the legacy default stream).
 *     Device work is ordered on it. A call returns only after the result is
 *     in a host output buffer; with device outputs it returns as soon as the
 *     work is queued;
 *   - a GMM handle is immutable after load and may be shared by threads;
 *   - N == 0 gives FV_ERR_EMPTY and a zero-filled Fisher vector.
 */
#ifndef FV_H_
#define FV_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FV_API __attribute__((visibility("default")))
#else
#define FV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FV_OK = 0,
    FV_PENDING = 1,           /* fv_server_poll: result not ready yet */
    FV_ERR_INVALID = -1,      /* bad argument or GMM parameter */
    FV_ERR_OOM = -2,          /* device or host allocation failed */
    FV_ERR_CUDA = -3,         /* a CUDA call failed */
    FV_ERR_BUSY = -4,         /* server admission refused (slots or memory) */
    FV_ERR_TIMEOUT = -5,      /* poll deadline passed */
    FV_ERR_NOTFOUND = -6,     /* unknown ticket */
    FV_ERR_EMPTY = -7,        /* N == 0: output is zero-filled */
    FV_ERR_DEVICE = -8,       /* a kernel reported an error flag */
    FV_ERR_UNSUPPORTED = -9   /* shape outside the implemented limits */
} fv_status;

typedef enum {
    FV_PREC_FP32 = 0,    /* plain FP32 form: SIMT kernels, centred statistics */
    FV_PREC_BF16 = 1,    /* precision form: BF16 tensor-core GEMMs, hi+lo split */
    FV_PREC_BF16X2 = 2   /* the precision form with the posteriors entering the
                            statistics GEMM as bf16 hi + lo pairs (about 2^-16
                            relative instead of 2^-9): the accurate choice when a
                            component's 1/sqrt(w) is large; one Y stage, slower */
} fv_precision;

/* GMM parameters, all host memory, float32:
 *   weights   K priors w_k > 0 with |sum_k w_k - 1| <= 1e-5 (renormalised in
 *             FP64 on load),
 *   means     K x D row-major mu_kd (finite),
 *   variances K x D row-major diagonal sigma^2_kd > 0 (finite).
 * Source: the GMM model "means, covariances, priors" of Algorithm 1. */
typedef struct {
    int K;
    int D;
    const float *weights;
    const float *means;
    const float *variances;
} fv_gmm_desc;

typedef struct fv_gmm fv_gmm;
typedef struct fv_server fv_server;

/* Load a GMM onto the current CUDA device and precompute, once and in FP64,
 * everything the encoder needs (the "compute sqrt(sigma^-1)" step of
 * Algorithm 1, run by "a simple GPU kernel" per Sec. 3.2): 1/sigma, the
 * per-component log-constants, 1/sqrt(w), 1/sqrt(2w), and for FV_PREC_BF16
 * the hi+lo split operand images. Copies every input; *out owns device
 * memory until fv_gmm_free. Errors: FV_ERR_INVALID (parameter checks above),
 * FV_ERR_OOM, FV_ERR_CUDA, FV_ERR_UNSUPPORTED (K or D beyond the limits of
 * the chosen precision, see fv_limits). */
FV_API int fv_gmm_load(const fv_gmm_desc *desc, fv_precision precision, fv_gmm **out);

/* Free a handle from fv_gmm_load (NULL is a no-op). The caller must make sure
 * no queued work still uses it (synchronise the streams it was used on). */
FV_API void fv_gmm_free(fv_gmm *gmm);

/* Report K, D and precision of a loaded GMM (any pointer may be NULL). */
FV_API int fv_gmm_info(const fv_gmm *gmm, int *K, int *D, int *precision);

/* The per-component constants of the log-likelihood as the loader computed
 * them on the device in FP64 (Sec. 3.1, Algorithm 1: the constant part of the
 * log posterior, log prior plus the Gaussian's normaliser; the -D/2 log 2pi
 * term is common to every component and left out):
 *   c_direct[k]   = log w_k - 1/2 sum_d log sigma^2_kd          (w renormalised to sum 1)
 *   c_expanded[k] = c_direct[k] - 1/2 sum_d mu_kd^2 / sigma^2_kd
 * The FP32 form uses c_direct with the centred distance, the BF16 form
 * c_expanded with the expanded [x, x^2] product; both are rounded to FP32
 * from these values. Host arrays of K doubles owned by the caller, either may
 * be NULL. Synchronous (waits for the load to finish). FV_ERR_INVALID on a
 * NULL handle, FV_ERR_CUDA if the copy fails. */
FV_API int fv_gmm_constants(const fv_gmm *gmm, double *c_direct, double *c_expanded);

/* Largest K and D the given precision supports. */
FV_API int fv_limits(fv_precision precision, int *max_K, int *max_D);

/* Encode one descriptor set (Algorithm 1 end to end).
 *   X        N x D float32 row-major descriptors (host or device),
 *   fv_out   2*K*D float32 normalised Fisher vector (host or device).
 * With an FV_PREC_BF16 handle the descriptors are rounded to bfloat16 on the
 * device before encoding. Scratch is taken stream-ordered from the device's
 * default memory pool and returned before the call's work ends.
 * Errors: FV_ERR_INVALID, FV_ERR_EMPTY (N == 0; fv_out zero-filled),
 * FV_ERR_OOM, FV_ERR_CUDA. */
FV_API int fv_encode(const fv_gmm *gmm, const float *X, int64_t N, int x_on_device,
              float *fv_out, int out_on_device, void *cuda_stream);

/* Encode B descriptor sets packed back to back (frame b owns rows
 * offsets[b] .. offsets[b+1]-1 of X_packed, offsets[0] == 0) in one pass:
 * one set of kernels over every frame, frames of uneven size sharing the GPU.
 *   offsets  B+1 int64, HOST memory, non-decreasing,
 *   fv_out   B x 2*K*D float32.
 * Empty frames get a zero vector; the call still returns FV_OK when at least
 * one frame is non-empty, else FV_ERR_EMPTY. */
FV_API int fv_encode_batch(const fv_gmm *gmm, const float *X_packed, const int64_t *offsets, int B,
                    int x_on_device, float *fv_out, int out_on_device, void *cuda_stream);

/* Precision form with descriptors already stored as bfloat16 on the device
 * (uint16 bit patterns, row pitch ld_x >= D elements, ld_x a multiple of 8).
 * Otherwise as fv_encode_batch; gmm must be an FV_PREC_BF16 handle and X,
 * fv_out device pointers. offsets is a host array. */
FV_API int fv_encode_batch_bf16(const fv_gmm *gmm, const uint16_t *X_bf16, int64_t ld_x,
                         const int64_t *offsets, int B, float *fv_out, void *cuda_stream);

/* Options of fv_encode_batch_opts.
 *   posterior_threshold  tau in [0, 1). 0 (the default of every other entry
 *            point) is the exact encoding. tau > 0 is the paper's early
 *            termination (Sec. 3.3, Algorithm 5, with 1e-6 in the paper):
 *            statistics terms whose posterior gamma_ik is not above tau are
 *            dropped (the threshold test of Algorithm 1's second loop), and
 *            blocks of work whose posteriors are all at or below tau are
 *            skipped: in the FP32 form a warp's row of 16 components, in the
 *            BF16 form a 16-row x 128-component K step of the statistics
 *            GEMM. The result is the thresholded Fisher vector.
 *   skip_counts  NULL, or DEVICE memory of two uint64 counters to which the
 *            call adds (skipped blocks, visited blocks) when tau > 0 (the
 *            caller zeroes them). */
typedef struct {
    float posterior_threshold;
    void *skip_counts;
} fv_encode_options;

/* fv_encode_batch / fv_encode_batch_bf16 with options (opts may be NULL).
 *   X          N x D row-major float32 (x_is_bf16 = 0; host or device per
 *              x_on_device, ld_x ignored) or bfloat16 bit patterns with row
 *              pitch ld_x (x_is_bf16 = 1; device only, FV_PREC_BF16 handle,
 *              ld_x >= D and a multiple of 8, 16-byte aligned),
 *   offsets    B+1 host int64 as in fv_encode_batch.
 * Errors as fv_encode_batch, and FV_ERR_INVALID for a threshold outside
 * [0, 1) or skip_counts not in device memory. */
FV_API int fv_encode_batch_opts(const fv_gmm *gmm, const void *X, int x_is_bf16, int64_t ld_x, const int64_t *offsets,
                                int B, int x_on_device, float *fv_out, int out_on_device, const fv_encode_options *opts,
                                void *cuda_stream);

/* ---- descriptor step before the encoding: PCA + positions (Sec. 3.1) ---------
 * The paper reduces each 128-dimensional dense-SIFT descriptor to m
 * dimensions with PCA and appends the descriptor's normalised X and Y
 * position, D = m + 2 (D = 82 in Sec. 4):
 *   y_i = [ P (x_i - mean) ; xy_i ].
 * The projection runs on the GPU as a prologue of the encoder: an FP32 SIMT
 * kernel for FV_PREC_FP32 handles, a tcgen05 GEMM for FV_PREC_BF16 handles
 * (x - mean and P split into bfloat16 hi + lo parts, three products with
 * FP32 accumulation, the result rounded to the bfloat16 rows the encoder
 * reads). */
typedef struct fv_pca fv_pca;

/* Load a projection onto the current device. basis: m x Din row-major host
 * floats (rows are the principal directions), mean: Din host floats the PCA
 * was centred on (NULL = zeros). 1 <= m <= 78 (so that D = m + 2 fits the
 * BF16 form's D <= 80), Din a multiple of 16 in 16..256. Copies its inputs.
 * Errors: FV_ERR_INVALID (NULL, non-finite), FV_ERR_UNSUPPORTED (sizes),
 * FV_ERR_OOM, FV_ERR_CUDA. */
FV_API int fv_pca_load(const float *basis, const float *mean, int m, int Din, fv_pca **out);
FV_API int fv_pca_info(const fv_pca *pca, int *m, int *Din);
FV_API void fv_pca_free(fv_pca *pca);

/* Project N descriptors (X: N x Din float32, device, 16-byte aligned; xy:
 * N x 2 float32 normalised positions, device, or NULL) into Y (device):
 * float32 rows of pitch m + 2 (m without xy) when y_bf16 = 0, or bfloat16
 * rows of pitch ld_y (a multiple of 16, >= D, 16-byte aligned; padding
 * zeroed) with the tcgen05 kernel when y_bf16 = 1. Stream-ordered. Errors:
 * FV_ERR_INVALID, FV_ERR_EMPTY (N == 0), FV_ERR_CUDA. */
FV_API int fv_pca_project(const fv_pca *pca, const float *X, const float *xy, int64_t N, void *Y, int y_bf16,
                          int64_t ld_y, void *cuda_stream);

/* Encode B frames of raw descriptors: the PCA step above, then the encoder
 * of the GMM's precision on the projected rows (the projected rows never
 * leave the device). X: offsets[B] x Din float32, xy: offsets[B] x 2 (or
 * NULL), both on the host or both on the device per x_on_device; the GMM's
 * D must be m + 2 (m when xy is NULL). offsets and fv_out as in
 * fv_encode_batch. Errors as fv_encode_batch, and FV_ERR_DEVICE (host
 * output only) if the projection gave up on a bounded wait. */
FV_API int fv_encode_pca(const fv_gmm *gmm, const fv_pca *pca, const float *X, const float *xy, const int64_t *offsets,
                         int B, int x_on_device, float *fv_out, int out_on_device, void *cuda_stream);

/* ---- dense SIFT: the descriptors of an image (Sec. 3.1-3.2, Sec. 4) ----------
 * Flat-window dense SIFT on the GPU over an image pyramid:
 *   scales s_j = 2^((top_scale - j)/2), j < n_scales (the paper's 8 scales
 *   from sqrt 2 down to 1/8: top_scale 1, n_scales 8; its 9-scale setting:
 *   top_scale 2, n_scales 9), each floor(H s + 1/2) x floor(W s + 1/2) pixels
 *   resampled bilinearly; central-difference gradients (one-sided on the
 *   border); each gradient's magnitude split linearly between its two nearest
 *   of 8 orientation bins; the triangular filter k(d) = 1 - |d|/b (2b - 1
 *   taps) along x then y, each output summing its inputs directly and only
 *   at the pixels the descriptors read (Sec. 3.2); 4 x 4 spatial bins of
 *   b x b pixels x 8 orientations = 128 entries, entry (4 by + bx) 8 + o, on a
 *   grid of centres x0 = 2b + stride i <= W_s - 2b (likewise y0); each
 *   descriptor L2-normalised, capped at 0.2 and renormalised (zero stays
 *   zero); positions (x0 / W_s - 0.5, y0 / H_s - 0.5). Descriptors of an
 *   image come scale by scale, row-major by (y0, x0) within a scale. */
typedef struct {
    int bin_size;    /* b: even, 2..16 (default 4) */
    int stride;      /* grid spacing in pixels; must divide bin_size (default 4, Sec. 4) */
    int n_scales;    /* 1..9 (default 8) */
    int top_scale;   /* the largest scale is 2^(top_scale/2) (default 1: sqrt 2) */
} fv_dsift_params;

/* Descriptors per image of size H x W (params NULL = the defaults above).
 * Errors: FV_ERR_INVALID for parameters or sizes outside the ranges. */
FV_API int fv_dsift_count(int H, int W, const fv_dsift_params *params, int64_t *n_per_image);

/* Dense SIFT of B grey-level images (B x H x W float32, row-major, host or
 * device per images_on_device) into desc (DEVICE, B x n x 128 float32,
 * 16-byte aligned) and xy (DEVICE, B x n x 2 float32, or NULL), n from
 * fv_dsift_count. Stream-ordered. Errors: FV_ERR_INVALID, FV_ERR_EMPTY (no
 * descriptor fits the image), FV_ERR_OOM, FV_ERR_CUDA. */
FV_API int fv_dsift(const float *images, int B, int H, int W, int images_on_device, const fv_dsift_params *params,
                    float *desc, float *xy, void *cuda_stream);

/* Images in, Fisher vectors out: fv_dsift, then fv_encode_pca with the
 * descriptors and positions of each image as one frame (the PCA takes
 * 128-dimensional descriptors; the GMM's D must be m + 2). fv_out: B x 2KD,
 * host or device per out_on_device. Every intermediate stays on the device.
 * Errors as fv_dsift and fv_encode_pca. */
FV_API int fv_encode_images(const fv_gmm *gmm, const fv_pca *pca, const float *images, int B, int H, int W,
                            int images_on_device, const fv_dsift_params *params, float *fv_out, int out_on_device,
                            void *cuda_stream);

/* ---- GMM training: expectation-maximisation on the GPU -----------------------
 * The paper encodes with a GMM trained beforehand (Sec. 3.1). These calls
 * train one on the GPU with the encoder's own kernels: the E-step is the
 * plain FP32 form's posteriors and centred statistics (Algorithm 1), the
 * M-step the closed form for a diagonal GMM,
 *   N_k = sum_i gamma_ik + 10 eps (eps = 2^-52),  w'_k = N_k / N,
 *   mu'_kd = sum_i gamma_ik x_id / N_k,
 *   var'_kd = sum_i gamma_ik (x_id - mu'_kd)^2 / N_k + reg_covar,
 * formed in FP64 from the FP32 sums centred on the current means. */

/* One EM step. gmm: an FV_PREC_FP32 handle (the current model). X: N x D
 * float32 (host or device per x_on_device). Outputs w_out (K), mu_out and
 * var_out (K x D row-major), host or device per out_on_device. mean_loglik
 * (host, nullable) receives 1/N sum_i log p(x_i) under the CURRENT model
 * (the E-step's value). Synchronous when an output is on the host or
 * mean_loglik is given. reg_covar >= 0 is added to every new variance.
 * Errors: FV_ERR_INVALID, FV_ERR_EMPTY (N == 0), FV_ERR_OOM, FV_ERR_CUDA. */
FV_API int fv_gmm_em_step(const fv_gmm *gmm, const float *X, int64_t N, int x_on_device, double reg_covar,
                          float *w_out, float *mu_out, float *var_out, int out_on_device, double *mean_loglik,
                          void *cuda_stream);

/* EM from the initial model `init` (host parameters, checked as by
 * fv_gmm_load) for at most max_iter steps, stopping early once the mean
 * log-likelihood changes by less than tol between steps; every step runs on
 * the device (the GMM preparation kernel re-derives the encoder's operands
 * from the new parameters between steps). Outputs (host): the final
 * w_out (K), mu_out and var_out (K x D), n_iter (steps run, nullable) and
 * mean_loglik (nullable: the last E-step's mean log-likelihood, i.e. under
 * the model before the last M-step). Synchronous. A variance that collapses
 * to zero (reg_covar = 0 and a component on a single point) makes the
 * log-likelihood non-finite: FV_ERR_INVALID. */
FV_API int fv_gmm_fit(const fv_gmm_desc *init, const float *X, int64_t N, int x_on_device, int max_iter, double tol,
                      double reg_covar, float *w_out, float *mu_out, float *var_out, int *n_iter, double *mean_loglik,
                      void *cuda_stream);

/* ---- batched form: one CUDA-graph launch per batch ---------------------------
 * A plan owns every device buffer a batch of up to max_frames frames and
 * max_rows descriptors needs (bfloat16 input rows, statistics slots, work
 * lists, output vectors; the fused encoder keeps the posteriors on chip) and
 * a CUDA graph of the whole kernel sequence (fused posteriors + statistics,
 * slot reduction, finalise), captured once against those buffers. The kernels read the batch's row and frame counts from device
 * memory, so a run uploads one small work list and launches the graph once:
 * frames of uneven size share the persistent kernels (Algorithm 1 for every
 * frame; the per-block copies and reduction of Algorithm 3 become per-share
 * statistics slots reduced per frame). FV_PREC_BF16 and FV_PREC_BF16X2
 * handles only.
 *
 * The tile pipeline is chosen by a measured autotune at creation (when
 * requested): every pair of Y-stage count (1, or 2 where two fit shared
 * memory) and share count (1, 2, 3 and 4 times the clusters resident at
 * once; the share count sets the tiles per share) is timed on a synthetic
 * batch of the plan's capacity; the fastest pair is kept and written to
 * tune_cache (one line per GPU model, SM count, K, D, capacity and
 * precision), which later plans read back. Rows per tile are the MMA's M. */
typedef struct fv_batch_plan fv_batch_plan;

typedef struct {
    int max_frames;          /* >= 1 */
    int64_t max_rows;        /* >= 1: total descriptors of a batch */
    int autotune;            /* 1: time candidate statistics grids at creation */
    const char *tune_cache;  /* file of tuned grids (read, then appended); NULL: none */
} fv_batch_plan_config;

typedef struct {
    int stat_ctas;           /* persistent clusters = row shares of a batch */
    int tuned;               /* 1: chosen by timing now, 2: read from tune_cache, 0: default */
    double tuned_ms;         /* best candidate's time (ms) when tuned now */
    int64_t max_rows;
    int max_frames;
    int ld_x;                /* row pitch (elements) of the plan's input buffer */
    int rows_per_tile;       /* M of the log-likelihood MMA (128) */
    int y_stages;            /* tiles whose [X | X^2 | 1] planes are in flight per CTA (1 or 2) */
    int candidates;          /* (stages, shares) pairs timed by the autotune */
    double tiles_per_share;  /* at the plan's capacity */
} fv_batch_plan_info;

FV_API int fv_batch_plan_create(const fv_gmm *gmm, const fv_batch_plan_config *cfg, fv_batch_plan **out);
/* Device pointers of the plan's input rows (bfloat16, max_rows x ld_x; write
 * a batch's descriptors packed back to back, rows D..ld_x-1 ignored) and of
 * its output (max_frames x 2KD float32). Valid until fv_batch_plan_destroy. */
FV_API int fv_batch_plan_buffers(fv_batch_plan *plan, uint16_t **x_bf16, float **fv_out);
/* Copy `rows` bfloat16 descriptor rows (device, row pitch ld_x >= D) into the
 * plan's input buffer (stream-ordered). */
FV_API int fv_batch_plan_load_bf16(fv_batch_plan *plan, const uint16_t *X_bf16, int64_t ld_x, int64_t rows,
                                   void *cuda_stream);
/* Encode B frames (offsets: B+1 host int64, offsets[0] == 0, offsets[B] <=
 * max_rows) already in the plan's input buffer with one graph launch; the
 * vectors land in the plan's output buffer (rows 0..B-1) and, when fv_out is
 * not NULL, are copied to fv_out (B x 2KD, host or device per out_on_device;
 * a host copy waits for the result). Ordered on cuda_stream. A plan must not
 * run on two streams at once. Errors: FV_ERR_INVALID, FV_ERR_EMPTY (every
 * frame empty; zero vectors), FV_ERR_DEVICE (host output only: a kernel gave
 * up on a bounded wait), FV_ERR_CUDA. */
FV_API int fv_batch_plan_run(fv_batch_plan *plan, const int64_t *offsets, int B, float *fv_out, int out_on_device,
                             void *cuda_stream);
/* Convert B frames of FP32 descriptors (device, packed N x D rows) into the
 * plan's input buffer, then run as fv_batch_plan_run. */
FV_API int fv_batch_plan_run_f32(fv_batch_plan *plan, const float *X, const int64_t *offsets, int B, float *fv_out,
                                 int out_on_device, void *cuda_stream);
FV_API int fv_batch_plan_get_info(const fv_batch_plan *plan, fv_batch_plan_info *info);
FV_API void fv_batch_plan_destroy(fv_batch_plan *plan);

/* ---- serving form: continuous batching of frames from many streams --------
 * A server keeps the GMM and two batch plans resident on the device. Client
 * threads submit frames (host FP32 descriptors) as they arrive; a frame is
 * admitted only while the device memory of admitted, unfinished frames stays
 * within hbm_budget_bytes and fewer than max_slots frames are in flight,
 * otherwise submit answers FV_ERR_BUSY at once. A scheduler thread gathers
 * the admitted frames into the next batch while the previous batch runs on
 * the GPU (two plans on two streams alternate), so frames that arrive while
 * others are being encoded join the next batch instead of waiting for a
 * queue to drain. Every frame is encoded exactly as fv_encode_batch would
 * encode it (a frame's vector does not depend on the other frames of its
 * batch beyond rounding of the per-share partial sums).
 * FV_PREC_BF16 handles only. */
typedef struct {
    int max_slots;                   /* frames admitted and not yet polled */
    int64_t hbm_budget_bytes;        /* device bytes for admitted frames' descriptors */
    int64_t max_batch_descriptors;   /* capacity of one GPU batch (rows) */
    int max_batch_frames;            /* capacity of one GPU batch (frames) */
    int64_t max_frame_descriptors;   /* largest accepted frame */
    int64_t batch_window_ns;         /* a batch that is not full waits at most this long
                                        after its oldest frame's submit (0: launch at once) */
} fv_server_config;

typedef struct {
    int status;             /* FV_OK, or the error of the frame's batch */
    int stream_id;
    int64_t n;              /* descriptors */
    int64_t latency_ns;     /* submit -> result ready on the host */
    int64_t queue_ns;       /* submit -> its batch launched */
    int batch_frames;       /* frames in the batch that encoded it */
} fv_result_info;

FV_API int fv_server_create(const fv_gmm *gmm, const fv_server_config *cfg, fv_server **out);
/* Copy a frame (X: host float32 N x D, 1 <= N <= max_frame_descriptors) into
 * the server; returns when X may be reused. *ticket identifies the result.
 * Errors: FV_ERR_BUSY (budget or slots exhausted: retry later),
 * FV_ERR_INVALID, FV_ERR_CUDA. */
FV_API int fv_server_submit(fv_server *srv, int stream_id, const float *X, int64_t N, uint64_t *ticket);
/* Wait up to timeout_ns (0: do not wait, < 0: wait without limit) for a
 * ticket's result; on FV_OK writes the 2KD vector to fv_out (host) and info,
 * and releases the ticket. FV_PENDING when not ready, FV_ERR_NOTFOUND for an
 * unknown or already released ticket, FV_ERR_TIMEOUT when the wait expired. */
FV_API int fv_server_poll(fv_server *srv, uint64_t ticket, float *fv_out, fv_result_info *info, int64_t timeout_ns);
/* Counters: admitted, refused (busy), completed frames, batches launched. */
FV_API int fv_server_stats(const fv_server *srv, int64_t *admitted, int64_t *refused, int64_t *completed,
                           int64_t *batches);
FV_API void fv_server_destroy(fv_server *srv);

/* Allocation-free variant of fv_encode (plain FP32 form, one descriptor set).
 * The paper has no counterpart: this entry point exists for callers that must
 * not allocate device memory, e.g. an application whose own allocator already
 * owns nearly all of it, a latency-critical loop that cannot risk a memory
 * pool growing, or a process under a fixed memory quota. Instead of taking
 * scratch from the memory pool, it uses one fixed 32 MiB __device__ array
 * inside the library (held on every GPU that loads the library until the
 * process exits) and calls no allocating routine.
 *   gmm      an FV_PREC_FP32 handle on the current device,
 *   X        N x D float32 row-major descriptors, DEVICE memory,
 *   fv_out   2*K*D float32, DEVICE memory.
 * The scratch needs about N*Kp*4 bytes for the posteriors (Kp = K rounded up
 * to 64), N*4 bytes of posterior group masks, plus the per-range statistics; larger inputs are rejected with
 * FV_ERR_UNSUPPORTED and a message giving the limit (e.g. N=19200, K=256,
 * D=64 fits). The first call on a device looks up the array's device address
 * (make that first call before any stream capture). All calls share the
 * array and it keeps the last call's contents; calls whose GPU work overlaps
 * (other streams, other threads) race on it, so serialise them. Returns after
 * queuing the work on cuda_stream. Errors: FV_ERR_INVALID, FV_ERR_UNSUPPORTED,
 * FV_ERR_EMPTY (N == 0; zero vector), FV_ERR_CUDA. */
FV_API int fv_encode_noalloc(const fv_gmm *gmm, const float *X, int64_t N, float *fv_out, void *cuda_stream);

/* Thread-local description of the last error on this thread ("" if none). */
FV_API const char *fv_last_error(void);

/* ---- instrumentation (not part of the method) -------------------------------
 * While enabled, every kernel launch of the library is bracketed by two CUDA
 * events recorded on the stream it is launched on; fv_prof_collect waits for
 * the recorded events, returns per-kernel launch counts and summed device
 * time, and clears them. fv_launch_count counts every kernel launched by the
 * library since it was loaded, profiling or not. */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} fv_kernel_stat;

FV_API int fv_prof_enable(int on);
/* Throughput probes of the SM units the plain FP32 form and the softmax use:
 * every SM runs long independent chains of scalar FP32 fused multiply-adds,
 * of packed f32x2 fused multiply-adds and of ex2.approx, each timed with CUDA
 * events on cuda_stream (best of five launches after a warm-up). Outputs
 * (each nullable): FP32 TFLOP/s counting a multiply-add as 2 flops for the
 * scalar and packed forms, and ex2 results per second in G/s. Synchronous.
 * Errors: FV_ERR_CUDA. */
FV_API int fv_probe_peaks(double *ffma_tflops, double *ffma2_tflops, double *ex2_gops, void *cuda_stream);
FV_API int fv_prof_collect(fv_kernel_stat *out, int max, int *n_out);
FV_API int64_t fv_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* FV_H_ */
