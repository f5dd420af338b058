// Per-position kernels instantiated for the 128 x 128 window. The per-position
// pass has three variants the autotuner chooses from: 1024 and 512 threads on
// one CTA (variants 0 and 1), and a pair of CTAs of 512 threads holding 64
// rows each (variant 2: the column transforms exchange through distributed
// shared memory, and two pairs fit on an SM, so a minibatch of 256 positions
// runs as 512 CTAs instead of 256 on 152 SMs).
#include "kernels_cluster.cuh"
#include "launch.h"

namespace ptycho {

template <>
cudaError_t launch_pass1<128>(const BatchArgs& a, cudaStream_t s, int variant) {
  if (a.opr_U) return launch_pass1_t<128, Threads<128>::T, true>(a, s);
  if (variant == 2) {
    using C = cl::Cfg128;
    static unsigned long long done = 0;
    cudaError_t e = smem_optin(cl::k_pass1_cluster<C, false>, C::Smem::bytes, &done);
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
    return cudaLaunchKernelEx(&cfg, cl::k_pass1_cluster<C, false>, a);
  }
  return variant == 1 ? launch_pass1_t<128, Threads<128>::ALT, false>(a, s)
                      : launch_pass1_t<128, Threads<128>::T, false>(a, s);
}

template cudaError_t launch_pass2<128>(const Pass2Args&, cudaStream_t, int);
}  // namespace ptycho
