// k_tc.cu -- placeholder: the tcgen05 engine is not built yet.
#include "nst_kernels.h"
namespace nst {
bool tc_available() { return false; }
cudaError_t launch_conv_tc(const ConvArgs &, cudaStream_t) { return cudaErrorNotSupported; }
}  // namespace nst
