// Instantiation of the persistent VMC kernel for scalar type double.
#include "launch.h"
#include "vmc_kernel.cuh"

namespace gcf {
template <>
cudaError_t launch_vmc<double>(const KParams<double>& k, int grid, int block, size_t smem,
                              cudaStream_t st) {
  vmc_kernel<double><<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
}  // namespace gcf
