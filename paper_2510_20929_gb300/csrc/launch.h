// Host-side launch wrappers of the per-position kernels, one translation unit
// per window size (pass_n<N>.cu) so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

namespace ptycho {
struct BatchArgs;
struct Pass2Args;
template <int N> cudaError_t launch_pass1(const BatchArgs& a, cudaStream_t s);
template <int N> cudaError_t launch_pass2(const Pass2Args& a, cudaStream_t s);
}  // namespace ptycho
