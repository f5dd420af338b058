// Per-position kernels instantiated for the 32 x 32 window.
#include "kernels.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1<32>(const BatchArgs&, cudaStream_t, int);
template cudaError_t launch_pass2<32>(const Pass2Args&, cudaStream_t, int);
}  // namespace ptycho
