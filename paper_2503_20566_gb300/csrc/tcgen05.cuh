// Fifth-generation tensor-core GEMM of one chain (tcgen05.mma, accumulator in
// tensor memory) for the environment contractions of the BF16 form.
//
// C[M x N] = A[M x K] B[K x N] with FP32 data read through (row stride,
// column stride) views, FP32 accumulation.  Each operand x is split into two
// BF16 parts, hi = bf16(x) and lo = bf16(x - hi), and the product is
// A_lo B_hi + A_hi B_lo + A_hi B_hi (the split-precision scheme of Markidis
// et al. 2018 and Ootomo & Yokota 2022 with BF16 parts), about 16
// significant bits; a single BF16 pass (8 bits) measured 0.5-12 % E_loc
// error on random-tensor networks, above the 1e-2 bound.
//   1. the chain's threads stage A_hi, A_lo (rows m0..m0+127 of the current
//      M tile) and B_hi^T, B_lo^T into its shared-memory staging area in the
//      K-major no-swizzle core-matrix layout (8 rows x 16 bytes per core
//      matrix; core matrices adjacent along K are 128 bytes apart, 8-row
//      groups Kp/8 core matrices apart), zero outside M, N, K;
//   2. one thread issues 3 Kp/16 tcgen05.mma.cta_group::1.kind::f16 (M =
//      128, N = Np, K = 16 each) into the chain's TMEM columns and commits
//      them to the chain's mbarrier;
//   3. all threads wait on the mbarrier (bounded), and the chain's four warps
//      read the 128 x N accumulator with tcgen05.ld (warp w reads TMEM lanes
//      32 (w % 4) .. + 31, i.e. rows of its quarter) into C.
// A wait that runs out of iterations marks the chain's tensor path unusable
// for the rest of the launch, records a status the host reads, and the GEMM
// is computed on the CUDA cores instead (results stay correct).
//
// Encodings (PTX ISA, tcgen05 "Instruction descriptor" and "Shared memory
// descriptor"): instruction descriptor bits 4-5 D format (1 = F32), 7-9 /
// 10-12 A / B format (1 = BF16), 15 / 16 A / B major (0 = K), 17-22 N >> 3,
// 24-28 M >> 4; shared-memory descriptor bits 0-13 start address >> 4,
// 16-29 leading-dimension byte offset >> 4 (between core matrices along K),
// 32-45 stride-dimension byte offset >> 4 (between 8-row groups), 46-47
// version 1, 61-63 layout 0 (no swizzle).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"

namespace gcf {

// Tensor-memory state of the chain groups of a CTA (at most four).
struct TcGroup {
  unsigned long long mbar;  // completion barrier of the group's MMAs
  unsigned tmem;            // TMEM address of the group's accumulator columns
  unsigned parity;          // phase parity the next completion flips to
  int ok;                   // 0 once a wait ran out: the group uses the CUDA cores
};
__shared__ __align__(8) TcGroup g_tc[4];
__shared__ unsigned g_tc_base;
__shared__ unsigned char* g_tc_stage[4];  // staging area of each chain group (null: no tensor-core path)
__shared__ long long g_tc_cap;            // bytes of each staging area
__shared__ int* g_tc_status;              // counter of waits that ran out
// Bulk-copy (tensor memory accelerator, 1-D form) state of the chain groups.
struct BulkGroup {
  unsigned long long mbar;  // completion barrier of the group's bulk copies
  unsigned parity;          // phase parity the next completion flips to
  int ok;                   // 0 once a wait ran out: the group copies with its threads
};
__shared__ __align__(8) BulkGroup g_bulk[4];
constexpr int kTcCols = 128;            // TMEM columns per chain group (N <= 128)
constexpr int kTcSpinLimit = 1 << 22;   // bounded mbarrier wait

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long tc_sdesc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (unsigned long long)((addr >> 4) & 0x3FFF) | ((unsigned long long)((lbo >> 4) & 0x3FFF) << 16) |
         ((unsigned long long)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ unsigned tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(N >> 3) << 17) | ((unsigned)(M >> 4) << 24);
}

// Allocate kTcCols TMEM columns per group (called by every thread of the CTA
// at kernel entry; warp 0 allocates) and initialise the groups' barriers.
__device__ inline void tc_setup(int n_groups) {
  const int cols = kTcCols * n_groups;  // 128, 256 or 512: a power of two
  if (threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&g_tc_base)),
                 "r"(cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x < n_groups) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&g_tc[threadIdx.x].mbar)));
    g_tc[threadIdx.x].parity = 0;
    g_tc[threadIdx.x].ok = 1;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x < n_groups) g_tc[threadIdx.x].tmem = g_tc_base + (unsigned)(kTcCols * threadIdx.x);
  __syncthreads();
}

// Bounded wait for completion `parity` of barrier `mbar`; true if it completed.
__device__ __forceinline__ bool tc_wait(unsigned mbar, unsigned parity) {
  unsigned done = 0;
  for (int it = 0; it < kTcSpinLimit && !done; ++it)
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity)
                 : "memory");
  return done != 0;
}

// Release the CTA's TMEM (every thread calls it once, at kernel exit).  A
// group whose last wait ran out first waits (bounded) for its MMAs in flight.
__device__ inline void tc_teardown(int n_groups) {
  if (threadIdx.x < n_groups && !g_tc[threadIdx.x].ok)
    tc_wait(smem_addr(&g_tc[threadIdx.x].mbar), g_tc[threadIdx.x].parity ^ 1u);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (threadIdx.x < 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(g_tc_base), "r"(kTcCols * n_groups));
}

// Initialise the groups' bulk-copy barriers (every thread of the CTA calls it).
__device__ inline void bulk_setup(int n_groups) {
  if (threadIdx.x < n_groups) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&g_bulk[threadIdx.x].mbar)));
    g_bulk[threadIdx.x].parity = 0;
    g_bulk[threadIdx.x].ok = 1;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
}

// At kernel exit: a group whose bulk-copy wait ran out waits (bounded) for
// that copy before the block's shared memory is released.
__device__ inline void bulk_teardown(int n_groups) {
  if (threadIdx.x < n_groups && !g_bulk[threadIdx.x].ok)
    tc_wait(smem_addr(&g_bulk[threadIdx.x].mbar), g_bulk[threadIdx.x].parity ^ 1u);
  __syncthreads();
}

// Copy n0 bytes from global src0 to shared dst0 and n1 bytes from src1 to
// dst1 with cp.async.bulk (addresses 16-byte aligned, sizes multiples of 16,
// n0 + n1 < 2^20), completing on the group's barrier; every thread of the
// executor calls it.  Returns false, with nothing known about the
// destination, if the wait ran out (the caller then copies with its threads).
template <class X>
__device__ __noinline__ bool bulk_copy2(const X ex, void* dst0, const void* src0, unsigned n0, void* dst1,
                                        const void* src1, unsigned n1, int* status_flag) {
  BulkGroup& bg = g_bulk[ex.slot()];
  if (!bg.ok) return false;
  const unsigned mbar = smem_addr(&bg.mbar);
  // the sources were written by this group's threads through the generic
  // proxy; the copy reads them through the async proxy
  asm volatile("fence.proxy.async;" ::: "memory");
  ex.sync();
  if (ex.leader()) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(n0 + n1) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst0)),
                 "l"(src0), "r"(n0), "r"(mbar)
                 : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst1)),
                 "l"(src1), "r"(n1), "r"(mbar)
                 : "memory");
  }
  const bool done = tc_wait(mbar, bg.parity);
  ex.sync();
  if (ex.leader()) {
    if (done) {
      bg.parity ^= 1u;
    } else {
      bg.ok = 0;
      atomicAdd(status_flag, 1);
    }
  }
  ex.sync();
  return done;
}

// Staging bytes a GEMM of these dimensions needs (hi and lo parts of an A
// tile of 128 rows and of B).
__host__ __device__ inline long long tc_stage_bytes(int N, int K) {
  const int Kp = (K + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
  return (long long)(128 + Np) * Kp * 2 * 2;
}

// x = hi + lo with hi = bf16(x), lo = bf16(x - hi), stored at byte offset
// `off` of the hi and lo planes.
__device__ __forceinline__ void tc_put_split(unsigned char* hi_plane, unsigned char* lo_plane, unsigned off,
                                             float x) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  *(__nv_bfloat16*)(hi_plane + off) = h;
  *(__nv_bfloat16*)(lo_plane + off) = __float2bfloat16_rn(x - __bfloat162float(h));
}

// C = A B on the tensor cores (see the top of this file).  Every thread of
// the executor calls it with the same arguments; `stage` is the group's
// staging area (16-byte aligned, tc_stage_bytes(N, K) bytes), N <= 128.
// Returns this thread's largest |C| written.  On a wait that runs out,
// returns -1 with C unwritten (the caller computes C another way).
template <class X>
__device__ __noinline__ float tc_gemm_bf16(const X ex, int M, int N, int K, const float* __restrict__ A, int sAm,
                                           int sAk, const float* __restrict__ B, int sBk, int sBn,
                                           float* __restrict__ C, int ldc, unsigned char* stage, int* status_flag) {
  TcGroup& tg = g_tc[ex.slot()];
  const int Kp = (K + 15) / 16 * 16, Np = (N + 15) / 16 * 16;
  const unsigned SBO = (unsigned)(Kp / 8) * 128u, LBO = 128u;
  unsigned char* sA = stage;                       // A_hi; A_lo follows
  unsigned char* sAl = stage + 128 * Kp * 2;
  unsigned char* sB = stage + 2 * 128 * Kp * 2;    // B_hi^T; B_lo^T follows
  unsigned char* sBl = sB + Np * Kp * 2;
  // B^T: row n, column k -> (n/8) SBO + (k/8) LBO + (n%8) 16 + (k%8) 2
#pragma unroll 1
  for (int idx = ex.tid(); idx < Np * Kp; idx += ex.size()) {
    const int n = idx / Kp, k = idx - (idx / Kp) * Kp;
    const float v = (n < N && k < K) ? B[k * sBk + n * sBn] : 0.f;
    tc_put_split(sB, sBl, (n >> 3) * SBO + (k >> 3) * LBO + (n & 7) * 16 + (k & 7) * 2, v);
  }
  const unsigned idesc = tc_idesc_bf16(128, Np);
  const unsigned mbar = smem_addr(&tg.mbar);
  const int quarter = ex.warp() & 3, cgrp = ex.warp() >> 2, ncg = (ex.nwarps() + 3) >> 2;
  float mx = 0.f;
  for (int m0 = 0; m0 < M; m0 += 128) {
#pragma unroll 1
    for (int idx = ex.tid(); idx < 128 * Kp; idx += ex.size()) {
      const int r = idx / Kp, k = idx - (idx / Kp) * Kp;
      const float v = (m0 + r < M && k < K) ? A[(m0 + r) * sAm + k * sAk] : 0.f;
      tc_put_split(sA, sAl, (r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2, v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    ex.sync();
    if (ex.leader()) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // small products first: lo x hi, hi x lo, then hi x hi
      const unsigned char* pa[3] = {sAl, sA, sA};
      const unsigned char* pb[3] = {sB, sBl, sB};
      for (int ks = 0; ks < Kp / 16; ++ks)
        for (int part = 0; part < 3; ++part) {
          const unsigned long long ad = tc_sdesc(smem_addr(pa[part]) + ks * 2 * LBO, LBO, SBO);
          const unsigned long long bd = tc_sdesc(smem_addr(pb[part]) + ks * 2 * LBO, LBO, SBO);
          const unsigned acc = (ks > 0 || part > 0) ? 1u : 0u;
          asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                       "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tg.tmem),
                       "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
        }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                   : "memory");
    }
    const bool done = tc_wait(mbar, tg.parity);
    ex.sync();
    if (!done) {
      if (ex.leader()) {
        tg.ok = 0;
        tg.parity ^= 1u;  // the pending completion, waited for at teardown
        atomicAdd(status_flag, 1);
      }
      ex.sync();
      return -1.f;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int row = quarter * 32 + ex.lane();
    for (int c0 = cgrp * 16; c0 < Np; c0 += 16 * ncg) {
      unsigned r[16];
      const unsigned taddr = tg.tmem + ((unsigned)(quarter * 32) << 16) + (unsigned)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m0 + row < M) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < N) {
            const float v = __uint_as_float(r[j]);
            C[(m0 + row) * ldc + c0 + j] = v;
            mx = fmaxf(mx, fabsf(v));
          }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (ex.leader()) tg.parity ^= 1u;
    ex.sync();
  }
  return mx;
}

}  // namespace gcf
