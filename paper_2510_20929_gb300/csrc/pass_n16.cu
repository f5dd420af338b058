// Per-position kernels instantiated for the 16 x 16 window.
#include "kernels.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1<16>(const BatchArgs&, cudaStream_t, int);
template cudaError_t launch_pass2<16>(const Pass2Args&, cudaStream_t, int);
}  // namespace ptycho
