// Instantiation of the persistent VMC kernel for scalar type float.
#include "launch.h"
#include "vmc_kernel.cuh"

namespace gcf {
template <>
cudaError_t launch_vmc<float>(const KParams<float>& k, int grid, int block, size_t smem,
                              cudaStream_t st) {
  vmc_kernel<float><<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
}  // namespace gcf
