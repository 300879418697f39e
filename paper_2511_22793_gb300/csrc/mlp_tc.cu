// Attribute network on the tensor cores (BF16 operands, FP32 accumulation).

#include "internal.cuh"

namespace gsparc {

int attr_mlp_bf16(int32_t, int32_t, const float*, const float*, const float*, const float*, const float*,
                  const gsparc_mlp*, int32_t, float*, cudaStream_t) {
    return GSPARC_ERR_INVALID;
}

}  // namespace gsparc
