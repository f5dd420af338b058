// Per-position kernels instantiated for the 64 x 64 window.
#include "kernels.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1<64>(const BatchArgs&, cudaStream_t, int);
template cudaError_t launch_pass2<64>(const Pass2Args&, cudaStream_t, int);
}  // namespace ptycho
