// Internal declarations of the BF16 (tensor-core) form of the encoder.
#pragma once

#include "fv_internal.h"

namespace fv {

// Number of persistent statistics CTAs (row shares) for `rows` packed rows.
int bf16_stat_ctas(const fv_gmm *g, int64_t rows, int sms);

// FP32 descriptors (rows x D) -> bfloat16 rows of pitch Dp (zero padded).
cudaError_t launch_bf16_convert(const fv_gmm *g, const float *X, int64_t rows, uint16_t *Xb, cudaStream_t st);

// Posteriors and statistics of the BF16 form; returns an fv_status.
// err: device word a kernel sets when a bounded wait gives up (zeroed by the caller).
// units: row segments (one frame each) grouped per statistics CTA;
// cta_units[c] = (first unit, count) of CTA c.
// rows_dev (nullable): device row count read by the kernels at start; rows is
// then the capacity of Xb/gamma (graph replays with a varying row count).
int run_bf16_encoder(const fv_gmm *g, const uint16_t *Xb, int64_t ldx, int64_t rows, uint16_t *gamma,
                     const StatUnit *units, const int2 *cta_units, int n_ctas, float *part, int P, int sms,
                     uint32_t *err, cudaStream_t st, const int64_t *rows_dev = nullptr);

}  // namespace fv
