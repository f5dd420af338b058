// Per-position kernels for the 256 x 256 window: the eight-CTA cluster pass 1
// and the step-size pass 2.
#include "kernels_cluster.cuh"
#include "launch.h"

namespace ptycho {

template <class C, bool OPR>
static cudaError_t launch_cluster(const BatchArgs& a, cudaStream_t s, unsigned long long* done) {
  cudaError_t e = smem_optin(cl::k_pass1_cluster<C, OPR>, C::Smem::bytes, done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C::Q * a.nb));
  cfg.blockDim = dim3(C::T);
  cfg.dynamicSmemBytes = C::Smem::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C::Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, cl::k_pass1_cluster<C, OPR>, a);
}

template <>
cudaError_t launch_pass1<256>(const BatchArgs& a, cudaStream_t s, int) {
  static unsigned long long done = 0, done_opr = 0;
  if (a.opr_U) return launch_cluster<cl::Cfg256, true>(a, s, &done_opr);
  return launch_cluster<cl::Cfg256, false>(a, s, &done);
}

template cudaError_t launch_pass2<256>(const Pass2Args&, cudaStream_t, int);

}  // namespace ptycho
