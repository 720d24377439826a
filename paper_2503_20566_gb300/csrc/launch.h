// Launch entry points of the per-type VMC kernels (one translation unit each).
#pragma once

#include <cuda_runtime.h>

#include "common.cuh"

namespace gcf {
template <class T> struct KParams;
template <class T>
cudaError_t launch_vmc(const KParams<T>& k, int grid, int block, size_t smem, cudaStream_t st);
// resident blocks per SM of vmc_kernel<T> for this block size and dynamic smem
template <class T>
int occupancy_vmc(int block, size_t smem);
// several chains per CTA (groups of 128 threads; block 256 = two groups, 512 = four);
// smem = groups x per-group bytes
template <class T>
cudaError_t launch_vmc_grouped(const KParams<T>& k, int grid, int block, size_t smem, cudaStream_t st);
// resident blocks per SM of vmc_kernel_grouped<T>; 0 if the launch cannot fit
template <class T>
int occupancy_vmc_grouped(int block, size_t smem);
// chains of several contexts in one launch (one chain per CTA of 256 threads)
// block 256: one chain per CTA (vmc_kernel_multi); block 512: four chains per
// CTA of group_bytes shared memory each (vmc_kernel_multi4)
template <class T>
cudaError_t launch_vmc_multi(const KParams<T>* ks, int n_ctx, const long long* start, long long total, T* arena,
                             long long ws_stride, int grid, int block, long long group_bytes,
                             unsigned long long* queue, size_t smem, cudaStream_t st);
template <class T>
int occupancy_vmc_multi(int block, size_t smem);
// bytes of the per-chain shared state of the VMC kernels (16-byte aligned)
size_t sharedv_bytes();
cudaError_t launch_init_configs(int N, int Lx, int Ly, int matter, const int* Q, int n_chains,
                                const int8_t* occ, const int8_t* powers, int8_t* configs,
                                int* status, cudaStream_t st);
}  // namespace gcf
