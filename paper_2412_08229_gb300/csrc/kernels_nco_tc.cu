// kernels_nco_tc.cu - the neural-collision step with the network on the tcgen05 tensor cores
// (BF16 operands, FP32 accumulation in tensor memory).
#include "cell.cuh"

namespace lbm {

bool nco_tc_supported(int, int) { return false; }
size_t nco_tc_weight_bytes() { return 16; }
void nco_tc_pack_weights(const float*, void*) {}
cudaError_t launch_step_nco_tc(const StepArgs&, int, int, const void*, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace lbm
