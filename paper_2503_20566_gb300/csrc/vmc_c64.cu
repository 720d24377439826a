// Instantiation of the persistent VMC kernel for scalar type cfloat.
#include "launch.h"
#include "vmc_kernel.cuh"

namespace gcf {
template <>
cudaError_t launch_vmc<cfloat>(const KParams<cfloat>& k, int grid, int block, size_t smem,
                              cudaStream_t st) {
  vmc_kernel<cfloat><<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
}  // namespace gcf
