// Instantiation of the persistent VMC kernel for scalar type cdouble.
#include "launch.h"
#include "vmc_kernel.cuh"

namespace gcf {
template <>
cudaError_t launch_vmc<cdouble>(const KParams<cdouble>& k, int grid, int block, size_t smem,
                              cudaStream_t st) {
  vmc_kernel<cdouble><<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
}  // namespace gcf
