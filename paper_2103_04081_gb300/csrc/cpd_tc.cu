// Tensor-core gradient engine (tcgen05, TMEM accumulators) for BF16 tensors.
#include "cpd_internal.h"

namespace cpd {

bool tc_supported(int R, int rb) { return false && R <= 64 && rb == 128; }

cudaError_t launch_grad_tc(const Problem<float> &, int, cudaStream_t) { return cudaErrorNotSupported; }

size_t tc_smem_bytes(const Problem<float> &) { return 0; }

}  // namespace cpd
