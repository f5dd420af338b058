// Host-side launch wrappers of the per-position kernels, one translation unit
// per window size (pass_n<N>.cu) so that they compile in parallel.
#pragma once
#include <cuda_runtime.h>

namespace ptycho {
struct BatchArgs;
struct Pass2Args;
struct MsArgs;
// variant 0 = default CTA size, 1 = the alternative CTA size (autotuner)
template <int N> cudaError_t launch_pass1(const BatchArgs& a, cudaStream_t s, int variant);
template <int N> cudaError_t launch_pass2(const Pass2Args& a, cudaStream_t s, int variant);
// multislice per-position pass
template <int N> cudaError_t launch_pass1_ms(const MsArgs& a, cudaStream_t s);
template <> cudaError_t launch_pass1_ms<192>(const MsArgs& a, cudaStream_t s);
template <> cudaError_t launch_pass1_ms<256>(const MsArgs& a, cudaStream_t s);
}  // namespace ptycho
