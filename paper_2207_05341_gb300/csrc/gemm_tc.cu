// Tensor-core (tcgen05) complex products for the mixed-precision path.
#include "impl.h"

namespace qst {

bool tc_available() { return false; }

cudaError_t split_bf16_G(int, const float2*, void*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_herm_square(int, const void*, float2*, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_gt_product(int, const void*, const void*, float*, float*, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace qst
