// Opt-in per-launch timing of the library's kernels: when enabled, every
// launch site records a CUDA event pair on the launching stream; reading the
// profile synchronises the events and sums the elapsed time per kernel name.
#pragma once
#include <cuda_runtime.h>

namespace ptycho {
enum KernelId : int {
  K_PASS1 = 0, K_PASS2, K_PROBE_REDUCE, K_NORM_PROBE, K_UPDATE, K_INIT, K_OPR_REDUCE, K_OPR_WEIGHTS, K_TILE_MAX, K_TILE_CLEAR,
  K_PASS1_MS, K_CLEAR_PLANE, K_PASS1_EXIT, K_FAR_TC, K_PASS1_OVERLAP, K_DFT_PLANES, K_COUNT
};
const char* kernel_name(int id);
bool profiling_on();
// Returns an event to record before the launch (or null when profiling is off).
cudaEvent_t profile_begin(int id, cudaStream_t s);
void profile_end(int id, cudaEvent_t start, cudaStream_t s);
}  // namespace ptycho
