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
// multislice LSQML tangent pass (step-size Gram entries); Q CTAs per position
// (ms_cluster_ctas(N), at most 8)
struct MsStepArgs;
int ms_cluster_ctas(int N);
template <int N> cudaError_t launch_step_ms(const MsStepArgs& a, cudaStream_t s);
template <> cudaError_t launch_step_ms<192>(const MsStepArgs& a, cudaStream_t s);
template <> cudaError_t launch_step_ms<256>(const MsStepArgs& a, cudaStream_t s);
// split-BF16 DFT-GEMM form (N = 32, 64, 128): bytes of the DFT chunks, their
// fill, the two parts of the per-position pass (part 1: exit waves, part 2:
// overlap-add) and the tensor-core far-field stage between them
template <int N> size_t dft_plane_bytes();
template <int N> cudaError_t launch_dft_planes(void* dft, cudaStream_t s);
template <int N> cudaError_t launch_pass1_part(const BatchArgs& a, cudaStream_t s, int part);
template <int N> cudaError_t launch_far_tc(const BatchArgs& a, const void* dft, cudaStream_t s);
}  // namespace ptycho
