// BF16 form (placeholder until the tensor-core kernels land).
#include "fv_bf16.h"

namespace fv {

int64_t bf16_rows_per_range(const fv_gmm *, int64_t rows, int) { return rows > 0 ? rows : 1; }

cudaError_t launch_bf16_convert(const fv_gmm *, const float *, int64_t, uint16_t *, cudaStream_t) {
    return cudaErrorNotSupported;
}

int run_bf16_encoder(const fv_gmm *, const uint16_t *, int64_t, int64_t, uint16_t *, const StatUnit *, int, float *,
                     int, int, cudaStream_t) {
    return fail(FV_ERR_UNSUPPORTED, "BF16 form not built yet");
}

}  // namespace fv
