// Multislice per-position pass for the cluster windows: 256 x 256 (eight CTAs)
// and 192 x 192 (six CTAs).
#include "kernels_ms_cluster.cuh"
#include "launch.h"

namespace ptycho {

int ms_cluster_ctas(int N) { return N == 256 ? cl::Cfg256::Q : N == 192 ? cl::Cfg192::Q : 1; }

template <>
cudaError_t launch_pass1_ms<256>(const MsArgs& a, cudaStream_t s) {
  static unsigned long long done[2] = {0, 0};
  return launch_ms_cluster<cl::Cfg256>(a, s, done);
}

template <>
cudaError_t launch_pass1_ms<192>(const MsArgs& a, cudaStream_t s) {
  static unsigned long long done[2] = {0, 0};
  return launch_ms_cluster<cl::Cfg192>(a, s, done);
}

template <>
cudaError_t launch_step_ms<256>(const MsStepArgs& a, cudaStream_t s) {
  static unsigned long long done = 0;
  return launch_step_ms_cluster<cl::Cfg256>(a, s, &done);
}

template <>
cudaError_t launch_step_ms<192>(const MsStepArgs& a, cudaStream_t s) {
  static unsigned long long done = 0;
  return launch_step_ms_cluster<cl::Cfg192>(a, s, &done);
}

}  // namespace ptycho
