// Per-position kernels for the 256 x 256 window: the four-CTA cluster pass 1
// and the step-size pass 2.
#include "kernels256.cuh"
#include "launch.h"

namespace ptycho {

template <>
cudaError_t launch_pass1<256>(const BatchArgs& a, cudaStream_t s, int) {
  static unsigned long long done = 0;
  cudaError_t e = smem_optin(n256::k_pass1_c256, n256::Smem::bytes, &done);
  if (e != cudaSuccess) return e;
  if (a.nb <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n256::Q * a.nb));
  cfg.blockDim = dim3(n256::T);
  cfg.dynamicSmemBytes = n256::Smem::bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = n256::Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, n256::k_pass1_c256, a);
}

template cudaError_t launch_pass2<256>(const Pass2Args&, cudaStream_t, int);

}  // namespace ptycho
