// Per-position kernels instantiated for the 128 x 128 window.
#include "kernels.cuh"
#include "launch.h"

namespace ptycho {
template cudaError_t launch_pass1<128>(const BatchArgs&, cudaStream_t, int);
template cudaError_t launch_pass2<128>(const Pass2Args&, cudaStream_t, int);
}  // namespace ptycho
