// Multislice per-position pass instantiated for the 16, 32 and 64 windows.
#include "kernels_ms.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1_ms<16>(const MsArgs&, cudaStream_t);
template cudaError_t launch_pass1_ms<32>(const MsArgs&, cudaStream_t);
template cudaError_t launch_pass1_ms<64>(const MsArgs&, cudaStream_t);
template cudaError_t launch_step_ms<16>(const MsStepArgs&, cudaStream_t);
template cudaError_t launch_step_ms<32>(const MsStepArgs&, cudaStream_t);
template cudaError_t launch_step_ms<64>(const MsStepArgs&, cudaStream_t);
}  // namespace ptycho
