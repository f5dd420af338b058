// Multislice per-position pass instantiated for the 128 x 128 window.
#include "kernels_ms.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1_ms<128>(const MsArgs&, cudaStream_t);
template cudaError_t launch_step_ms<128>(const MsStepArgs&, cudaStream_t);
}  // namespace ptycho
