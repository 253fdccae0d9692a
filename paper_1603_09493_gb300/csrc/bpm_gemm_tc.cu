// tcgen05 BF16 split demag GEMM (placeholder until the tensor-core kernel lands).
#include "bpm_internal.cuh"

namespace bpm {

int gemm_bf16x3_tc(cudaStream_t, int, int, int, const __nv_bfloat16*, const __nv_bfloat16*,
                   const __nv_bfloat16*, const __nv_bfloat16*, float*, int, int*, int) {
    set_error("tensor-core demag GEMM not built in this version");
    return BPM_ERR_STATE;
}

}  // namespace bpm
