// Instantiation of the persistent VMC kernel for scalar type cfloat.
#include "launch.h"
#include "vmc_kernel.cuh"

namespace gcf {
template <>
cudaError_t launch_vmc<cfloat>(const KParams<cfloat>& k, int grid, int block, size_t smem,
                              cudaStream_t st) {
  {
    // static + dynamic shared memory above 48 KB needs the opt-in attribute
    cudaError_t e = cudaFuncSetAttribute(vmc_kernel<cfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  vmc_kernel<cfloat><<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
template <>
int occupancy_vmc<cfloat>(int block, size_t smem) {
  cudaFuncSetAttribute(vmc_kernel<cfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, vmc_kernel<cfloat>, block, smem) != cudaSuccess) return 1;
  return n > 0 ? n : 1;
}
template <>
cudaError_t launch_vmc_grouped<cfloat>(const KParams<cfloat>& k, int grid, int block, size_t smem,
                                 cudaStream_t st) {
  // 256 threads: two chain groups per CTA; 512: four (one CTA per SM)
  auto* fn = block == 512 ? vmc_kernel_grouped4<cfloat> : vmc_kernel_grouped<cfloat>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  fn<<<grid, block, smem, st>>>(k);
  return cudaGetLastError();
}
template <>
int occupancy_vmc_grouped<cfloat>(int block, size_t smem) {
  auto* fn = block == 512 ? vmc_kernel_grouped4<cfloat> : vmc_kernel_grouped<cfloat>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) return 0;
  return n;
}
template <>
cudaError_t launch_vmc_multi<cfloat>(const KParams<cfloat>* ks, int n_ctx, const long long* start, long long total,
                                  cfloat* arena, long long ws_stride, int grid, int block, long long group_bytes,
                                  unsigned long long* queue, size_t smem, cudaStream_t st) {
  if (block == 512) {
    cudaError_t e = cudaFuncSetAttribute(vmc_kernel_multi4<cfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    vmc_kernel_multi4<cfloat><<<grid, 512, smem, st>>>(ks, n_ctx, start, total, arena, ws_stride, group_bytes, queue);
    return cudaGetLastError();
  }
  cudaError_t e = cudaFuncSetAttribute(vmc_kernel_multi<cfloat>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  vmc_kernel_multi<cfloat><<<grid, 256, smem, st>>>(ks, n_ctx, start, total, arena, ws_stride, queue);
  return cudaGetLastError();
}
template <>
int occupancy_vmc_multi<cfloat>(int block, size_t smem) {
  const void* fn = block == 512 ? (const void*)vmc_kernel_multi4<cfloat> : (const void*)vmc_kernel_multi<cfloat>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) return 0;
  return n;
}
}  // namespace gcf
