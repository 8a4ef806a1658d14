// Internal declarations of the BF16 (tensor-core) form of the encoder.
#pragma once

#include "fv_internal.h"

namespace fv {

// Clusters of the fused encoder kernel resident at once on the current device.
int bf16_max_shares(const fv_gmm *g, int sms);

// Number of row shares (persistent clusters) for a call over `rows` packed rows.
int bf16_shares(const fv_gmm *g, int64_t rows, int sms);

// FP32 descriptors (rows x D) -> bfloat16 rows of pitch Dp (zero padded).
cudaError_t launch_bf16_convert(const fv_gmm *g, const float *X, int64_t rows, uint16_t *Xb, cudaStream_t st);

// Posteriors and statistics of the BF16 form in one kernel; returns an fv_status.
// Xb: bf16 rows of pitch ldx; rows: rows addressable in Xb (rows past it read as zero).
// units: row ranges (one frame each) grouped per share; cl_units[c] = (first
// unit, count) of share c, which one cluster of the kernel walks.
// part: [slot][P][Kp] statistics slots, P = 2D + 1 (centred [A | B | S0]).
// err: device word a kernel sets when a bounded wait gives up (zeroed by the caller).
// tau > 0: early termination (posteriors <= tau dropped, all-zero 16-row
// K steps of the statistics GEMM skipped); skip_count (device, nullable):
// [skipped, visited] K steps.
// nstage: Y-plane stages of the tile pipeline (0 = the most that fit shared
// memory; 1 or 2 to choose, e.g. by the batched form's autotuner).
int run_bf16_encoder(const fv_gmm *g, const uint16_t *Xb, int64_t ldx, int64_t rows, const StatUnit *units,
                     const int2 *cl_units, int n_shares, float *part, int P, uint32_t *err, cudaStream_t st,
                     float tau = 0.f, unsigned long long *skip_count = nullptr, int nstage = 0);

// Y-plane stages that fit shared memory for this GMM (1 or 2).
int bf16_max_stages(const fv_gmm *g);

}  // namespace fv
