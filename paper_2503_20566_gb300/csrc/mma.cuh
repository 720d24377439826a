// Tensor-core GEMM tiles for the mixed-precision contraction forms.
//
// One warp computes a 16 x 8 output tile with mma.sync (m16n8k8 for TF32
// operands, m16n8k16 for BF16 operands), accumulating in FP32.  Operands are
// read straight from their (row stride, column stride) views in shared or
// global memory and rounded on the way into the fragment registers, so the
// stored tensors stay FP32 and the strided-view GEMM interface of the CUDA-
// core form is kept.  Modes:
//   GEMM_TF32X3: each FP32 operand x is split as x = hi + lo with hi, lo TF32
//     (lo = tf32(x - hi)); the product is hi*hi + hi*lo + lo*hi, which keeps
//     about 21 significant bits (the split-precision scheme of Markidis et
//     al., "NVIDIA Tensor Core Programmability, Performance & Precision",
//     2018, as refined for TF32 by Ootomo & Yokota, 2022).
//   GEMM_BF16: the same split with BF16 parts (hi = bf16(x), lo =
//     bf16(x - hi), products lo*hi + hi*lo + hi*hi, about 16 significant
//     bits), FP32 accumulation.  A single BF16 pass (8 bits) measured 0.5-12 %
//     E_loc error on random-tensor networks, above the 1e-2 bound.
// Complex operands use four real products, Re C = Ar Br - Ai Bi and
// Im C = Ar Bi + Ai Br.
//
// Fragment ownership (PTX ISA, "Matrix fragments for mma.m16n8k8 / k16"):
// lane = 4 g + t.  A rows g and g + 8; C holds (g, 2t), (g, 2t+1),
// (g+8, 2t), (g+8, 2t+1).  TF32 k8: A columns t, t+4; B rows t, t+4,
// column g.  BF16 k16: A columns (2t, 2t+1) and (2t+8, 2t+9), two per
// register, lower k in the low half; B rows likewise, column g.
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace gcf {

enum GemmMode { GEMM_FFMA = 0, GEMM_TF32X3 = 1, GEMM_BF16 = 2 };

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t u;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
  return u;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo_k, float hi_k) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo_k, hi_k);  // .x (low half) = lo_k
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma_tf32(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// c += a b for FP32 fragments a (4 values), b (2 values) with the 3-pass
// TF32 split.
__device__ __forceinline__ void mma_tf32x3(float* c, const float* a, const float* b) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) split_tf32(a[i], ah[i], al[i]);
#pragma unroll
  for (int i = 0; i < 2; ++i) split_tf32(b[i], bh[i], bl[i]);
  mma_tf32(c, al, bh);
  mma_tf32(c, ah, bl);
  mma_tf32(c, ah, bh);
}
// c += a b for FP32 fragments a (8 values: regs x (lo k, hi k)), b (4 values),
// each value split into two BF16 parts (3 products).
__device__ __forceinline__ void mma_bf16f(float* c, const float* a, const float* b) {
  uint32_t ah[4], al[4], bh[2], bl[2];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(a[2 * i]));
    const float h1 = __bfloat162float(__float2bfloat16_rn(a[2 * i + 1]));
    ah[i] = pack_bf16(h0, h1);
    al[i] = pack_bf16(a[2 * i] - h0, a[2 * i + 1] - h1);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float h0 = __bfloat162float(__float2bfloat16_rn(b[2 * i]));
    const float h1 = __bfloat162float(__float2bfloat16_rn(b[2 * i + 1]));
    bh[i] = pack_bf16(h0, h1);
    bl[i] = pack_bf16(b[2 * i] - h0, b[2 * i + 1] - h1);
  }
  mma_bf16(c, al, bh);
  mma_bf16(c, ah, bl);
  mma_bf16(c, ah, bh);
}

// scalar types with a tensor-core form (FP32 storage)
template <class T> struct MmaOk { static constexpr bool value = false; };
template <> struct MmaOk<float> { static constexpr bool value = true; };
template <> struct MmaOk<cfloat> { static constexpr bool value = true; };

template <class T> struct MmaParts;
template <> struct MmaParts<float> {
  static constexpr bool cplx = false;
  __device__ static float re(float v) { return v; }
  __device__ static float im(float) { return 0.f; }
};
template <> struct MmaParts<cfloat> {
  static constexpr bool cplx = true;
  __device__ static float re(cfloat v) { return v.x; }
  __device__ static float im(cfloat v) { return v.y; }
};

// Warp-tiled C = [C +] A B on tensor cores (T = float or cfloat).  Every
// thread of the executor calls it; warps take 16 x 8 tiles round-robin.
// Returns this thread's largest |component| of the C values it wrote (for
// the caller's rescale).  Out-of-range rows / columns / k read as zero.
template <class T, int MODE, class X>
__device__ __noinline__ float mma_gemm(const X ex, int M, int N, int K, const T* __restrict__ A, int sAm,
                                       int sAk, const T* __restrict__ B, int sBk, int sBn, T* __restrict__ C,
                                       int sCm, int sCn, bool accumulate) {
  using P = MmaParts<T>;
  constexpr int KS = MODE == GEMM_BF16 ? 16 : 8;
  const int lane = ex.lane(), g = lane >> 2, t = lane & 3;
  const int tN = (N + 7) >> 3, tiles = ((M + 15) >> 4) * tN;
  float mx = 0.f;
  for (int tile = ex.warp(); tile < tiles; tile += ex.nwarps()) {
    const int m0 = (tile / tN) << 4, n0 = (tile % tN) << 3;
    const int r0 = m0 + g, r1 = m0 + g + 8, cn = n0 + g;
    float cr[4] = {0.f, 0.f, 0.f, 0.f}, ci[4] = {0.f, 0.f, 0.f, 0.f};
    if (accumulate) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = (i < 2) ? r0 : r1, c = n0 + 2 * t + (i & 1);
        if (r < M && c < N) {
          const T v = C[r * sCm + c * sCn];
          cr[i] = P::re(v);
          ci[i] = P::im(v);
        }
      }
    }
    for (int k0 = 0; k0 < K; k0 += KS) {
      // fragment element -> k index
      float ar[2 * (KS / 4)], ai[2 * (KS / 4)], br[KS / 4], bi[KS / 4];
#pragma unroll
      for (int e = 0; e < KS / 4; ++e) {
        // A: register e of the fragment pair for rows r0 / r1
        int kk;
        if constexpr (MODE == GEMM_BF16) kk = k0 + 2 * t + (e & 1) + ((e >> 1) << 3);
        else kk = k0 + t + (e << 2);
        const bool kin = kk < K;
        const T a0 = (kin && r0 < M) ? A[r0 * sAm + kk * sAk] : zero<T>();
        const T a1 = (kin && r1 < M) ? A[r1 * sAm + kk * sAk] : zero<T>();
        const T bv = (kin && cn < N) ? B[kk * sBk + cn * sBn] : zero<T>();
        // element order: (row r0 | row r1) for each k slot
        ar[2 * e] = P::re(a0); ar[2 * e + 1] = P::re(a1);
        ai[2 * e] = P::im(a0); ai[2 * e + 1] = P::im(a1);
        br[e] = P::re(bv); bi[e] = P::im(bv);
      }
      // reorder into the fragment register order
      float fa[2 * (KS / 4)], fb[KS / 4];
      auto frag = [&](const float* av, const float* bv, float* oa, float* ob) {
        if constexpr (MODE == GEMM_BF16) {
          // regs: a0 = (r0, k 2t / 2t+1), a1 = (r1, ...), a2 = (r0, k+8 ...), a3 = (r1, k+8 ...)
          // slots e: 0 -> k 2t, 1 -> 2t+1, 2 -> 2t+8, 3 -> 2t+9
          oa[0] = av[0]; oa[1] = av[2];  // a0 = r0: (e0, e1)
          oa[2] = av[1]; oa[3] = av[3];  // a1 = r1: (e0, e1)
          oa[4] = av[4]; oa[5] = av[6];  // a2 = r0: (e2, e3)
          oa[6] = av[5]; oa[7] = av[7];  // a3 = r1: (e2, e3)
          ob[0] = bv[0]; ob[1] = bv[1]; ob[2] = bv[2]; ob[3] = bv[3];
        } else {
          // a0 = (r0, t), a1 = (r1, t), a2 = (r0, t+4), a3 = (r1, t+4)
          oa[0] = av[0]; oa[1] = av[1]; oa[2] = av[2]; oa[3] = av[3];
          ob[0] = bv[0]; ob[1] = bv[1];
        }
      };
      auto run = [&](float* c, const float* av, const float* bv) {
        frag(av, bv, fa, fb);
        if constexpr (MODE == GEMM_BF16) mma_bf16f(c, fa, fb);
        else mma_tf32x3(c, fa, fb);
      };
      run(cr, ar, br);
      if (P::cplx) {
        float nai[2 * (KS / 4)];
#pragma unroll
        for (int e = 0; e < 2 * (KS / 4); ++e) nai[e] = -ai[e];
        run(cr, nai, bi);
        run(ci, ar, bi);
        run(ci, ai, br);
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = (i < 2) ? r0 : r1, c = n0 + 2 * t + (i & 1);
      if (r < M && c < N) {
        T v;
        if constexpr (P::cplx) v = T{cr[i], ci[i]};
        else v = cr[i];
        C[r * sCm + c * sCn] = v;
        mx = fmaxf(mx, absmax1(v));
      }
    }
  }
  return mx;
}

}  // namespace gcf
