// Environment steps of the strip (4-layer) and row (3-layer) contractions,
// written as GEMM -> column-operator contraction -> GEMM.
//
// Strip, left step (columns absorbed left to right):
//   L'[a2][i2][j2][b2] = sum L[a][i][j][b] Bs[a][d][a2] W1[i][i2][d][m]
//                            W2[j][j2][m][u] Ts[b][u][b2]
//   C[(i j d)][(u i2 j2)] = sum_m W1[i][i2][d][m] W2[j][j2][m][u]   (column operator)
//   G1: X1[(i j b)][(d a2)] = sum_a L[a][(i j b)] Bs[a][(d a2)]          GEMM
//   G2: X2[(a2 i2 j2)][(b u)] = sum_{(i j d)} X1 . C                      per (b, a2)
//   G3: L'[(a2 i2 j2)][b2] = sum_{(b u)} X2[(a2 i2 j2)][(b u)] Ts[(b u)][b2]  GEMM
// and the mirrored right step; the row steps are the same with one PEPS row.
// The third stage divides its output by its largest |component| and returns
// the log of that factor (log-space rescaling keeps FP32 in range).
#pragma once

#include "common.cuh"
#include "mma.cuh"
#include "tcgen05.cuh"

namespace gcf {

// ---------------------------------------------------------------------------
// Register-tiled CTA GEMM: C[m][n] (row-major, ldc) = sum_k A(m,k) B(k,n),
// A(m,k) = A[m*sAm + k*sAk], B(k,n) = B[k*sBk + n*sBn].  Each thread owns
// TM x TN outputs per tile.  If rescale, the output is divided by its
// largest |component| (CTA-wide) and log(max) is returned.
// ---------------------------------------------------------------------------
template <class T, int TM, int TN, class X>
__device__ __forceinline__ float gemm_tiles(const X ex, int M, int N, int K, const T* __restrict__ A, int sAm,
                                            int sAk, const T* __restrict__ B, int sBk, int sBn,
                                            T* __restrict__ C, int ldc) {
  const int tilesN = (N + TN - 1) / TN;
  const int tiles = ((M + TM - 1) / TM) * tilesN;
  float mx = 0.f;
#pragma unroll 1
  for (int t = ex.tid(); t < tiles; t += ex.size()) {
    const int tm = t / tilesN;
    const int m0 = tm * TM, n0 = (t - tm * tilesN) * TN;
    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = zero<T>();
    const T* a = A + m0 * sAm;
    const T* b = B + n0 * sBn;
    const bool full = (m0 + TM <= M) && (n0 + TN <= N);
    if (full) {
#pragma unroll 4
      for (int k = 0; k < K; ++k) {
        T av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = a[i * sAm + k * sAk];
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = b[k * sBk + j * sBn];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmac(acc[i][j], av[i], bv[j]);
      }
    } else {
#pragma unroll 1
      for (int k = 0; k < K; ++k) {
        T av[TM], bv[TN];
#pragma unroll
        for (int i = 0; i < TM; ++i) av[i] = (m0 + i < M) ? a[i * sAm + k * sAk] : zero<T>();
#pragma unroll
        for (int j = 0; j < TN; ++j) bv[j] = (n0 + j < N) ? b[k * sBk + j * sBn] : zero<T>();
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) acc[i][j] = fmac(acc[i][j], av[i], bv[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j)
        if (m0 + i < M && n0 + j < N) {
          C[(m0 + i) * ldc + n0 + j] = acc[i][j];
          mx = fmaxf(mx, (float)absmax1(acc[i][j]));
        }
  }
  return mx;
}

// Dispatch on the output size so that typically one tile per thread.  With
// rescale, the output is multiplied by 2^-e (exact) with e the binary
// exponent of its largest |component|, and e is returned.
template <class T, class X>
__device__ __noinline__ int cta_gemm_scaled(const X ex, int M, int N, int K, const T* A, int sAm, int sAk,
                                              const T* B, int sBk, int sBn, T* C, int ldc,
                                              bool rescale) {
  float mx;
  const int MN = M * N;
  const int nt = ex.size();
  bool done = false;
  if constexpr (std::is_same<T, float>::value) {
    // BF16 form of a real chain: the fifth-generation tensor cores when the
    // launch set them up and the operands fit the chain's staging area
    const int slot = ex.slot();
    if (g_gemm_mode[slot] == GEMM_BF16 && g_tc_stage[slot] && N <= kTcCols &&
        tc_stage_bytes(N, K) <= g_tc_cap && g_tc[slot].ok) {
      mx = tc_gemm_bf16(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, g_tc_stage[slot], g_tc_status);
      done = mx >= 0.f;
      if (!done) mx = 0.f;
    }
  }
  if (done) {
  } else if constexpr (MmaOk<T>::value) {
    const int mode = g_gemm_mode[ex.slot()];
    if (mode != GEMM_FFMA) {
      if (mode == GEMM_BF16)
        mx = mma_gemm<T, GEMM_BF16>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, 1, false);
      else
        mx = mma_gemm<T, GEMM_TF32X3>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc, 1, false);
      done = true;
    }
  }
  if (done) {
  } else if (MN >= 8 * nt && M % 4 == 0 && N % 2 == 0)
    mx = gemm_tiles<T, 4, 2>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc);
  else if (MN >= 4 * nt && M % 2 == 0 && N % 2 == 0)
    mx = gemm_tiles<T, 2, 2>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc);
  else
    mx = gemm_tiles<T, 1, 1>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, ldc);
  if (!rescale) {
    ex.sync();
    return 0;
  }
  mx = ex.maxf(mx);
  if (mx > 0.f && isfinite(mx)) {
    using R = typename Traits<T>::R;
    const int e = exp2_of(mx);
    const R s = pow2r<R>(-e);
    if (ldc == N) {
#pragma unroll 1
      for (int i = ex.tid(); i < MN; i += nt) C[i] = scale(C[i], s);
    } else {
#pragma unroll 1
      for (int i = ex.tid(); i < MN; i += nt) {
        const int m = i / N, n = i - m * N;
        C[m * ldc + n] = scale(C[m * ldc + n], s);
      }
    }
    ex.sync();
    return e;
  }
  ex.sync();
  return 0;
}

// ---------------------------------------------------------------------------
// Strip steps
// ---------------------------------------------------------------------------
struct SDims {
  int nA, nI, nJ, nB;     // left cut: B bond, row-r bond, row-(r+1) bond, T bond
  int nA2, nI2, nJ2, nB2; // right cut
  int pB, pM, pT;         // B-physical, middle vertical bond, T-physical
};

// C[(i j d)][(u i2 j2)] = sum_m W1[i][i2][d][m] W2[j][j2][m][u], stored with
// padded D_k strides: row (i*DK + j)*DK + d, column (u*DK + i2)*DK + j2.
template <class T, int DK, class X>
__device__ __forceinline__ void build_column_op(const X ex, const SDims& d, const T* W1, const T* W2, T* Cop) {
  constexpr int D3 = DK * DK * DK;
#pragma unroll 1
  for (int idx = ex.tid(); idx < D3 * D3; idx += ex.size()) {
    const int k = idx / D3, n = idx % D3;
    const int i = k / (DK * DK), j = (k / DK) % DK, dd = k % DK;
    const int u = n / (DK * DK), i2 = (n / DK) % DK, j2 = n % DK;
    T s = zero<T>();
    if (i < d.nI && j < d.nJ && dd < d.pB && u < d.pT && i2 < d.nI2 && j2 < d.nJ2) {
#pragma unroll
      for (int m = 0; m < DK; ++m)
        if (m < d.pM)
          s = fmac(s, W1[((i * DK + i2) * DK + dd) * DK + m], W2[((j * DK + j2) * DK + m) * DK + u]);
    }
    Cop[idx] = s;
  }
}

// left step; returns log of the rescale factor of the output
template <class T, int DK, class X>
__device__ __noinline__ int strip_left(const X ex, const SDims& d, const T* L, const T* Bs, const T* W1,
                                         const T* W2, const T* Ts, T* out, T* X1, T* X2, T* Cop) {
  build_column_op<T, DK>(ex, d, W1, W2, Cop);
  // G1: X1[(i j b)][(d a2)] = sum_a L[a][(i j b)] Bs[a][(d a2)]
  const int Mij = d.nI * d.nJ * d.nB, N1 = d.pB * d.nA2;
  cta_gemm_scaled<T>(ex, Mij, N1, d.nA, L, 1, Mij, Bs, N1, 1, X1, N1, false);
  // G2: X2[(a2 i2 j2)][(b u)] = sum_{(i j d)} X1[(i j b)][(d a2)] C[(i j d)][(u i2 j2)]
  {
    constexpr int D3 = DK * DK * DK;
    const int ldx2 = d.nB * d.pT;
    const int sI = d.nJ * d.nB * N1, sJ = d.nB * N1;
#pragma unroll 1
    for (int p = ex.tid(); p < d.nB * d.nA2; p += ex.size()) {
      const int b = p / d.nA2, a2 = p - (p / d.nA2) * d.nA2;
      const T* x1 = X1 + b * N1 + a2;
      T x[D3];
#pragma unroll
      for (int i = 0; i < DK; ++i)
#pragma unroll
        for (int j = 0; j < DK; ++j)
#pragma unroll
          for (int dd = 0; dd < DK; ++dd)
            x[(i * DK + j) * DK + dd] =
                (i < d.nI && j < d.nJ && dd < d.pB) ? x1[i * sI + j * sJ + dd * d.nA2] : zero<T>();
      T* x2 = X2 + a2 * d.nI2 * d.nJ2 * ldx2 + b * d.pT;
#pragma unroll
      for (int u = 0; u < DK; ++u)
#pragma unroll
        for (int i2 = 0; i2 < DK; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < DK; ++j2) {
            if (u < d.pT && i2 < d.nI2 && j2 < d.nJ2) {
              const int n = (u * DK + i2) * DK + j2;
              T s = zero<T>();
#pragma unroll
              for (int k = 0; k < D3; ++k) s = fmac(s, x[k], Cop[k * D3 + n]);
              x2[(i2 * d.nJ2 + j2) * ldx2 + u] = s;
            }
          }
    }
    ex.sync();
  }
  // G3: out[(a2 i2 j2)][b2] = sum_{(b u)} X2 Ts
  return cta_gemm_scaled<T>(ex, d.nA2 * d.nI2 * d.nJ2, d.nB2, d.nB * d.pT, X2, d.nB * d.pT, 1, Ts, d.nB2, 1,
                            out, d.nB2, true);
}

// right step: R[a][i][j][b] from R2[a2][i2][j2][b2]
template <class T, int DK, class X>
__device__ __noinline__ int strip_right(const X ex, const SDims& d, const T* R2, const T* Bs, const T* W1,
                                          const T* W2, const T* Ts, T* out, T* Y1, T* Y2, T* Cop) {
  build_column_op<T, DK>(ex, d, W1, W2, Cop);
  // G1: Y1[(a2 i2 j2)][(b u)] = sum_b2 R2[(a2 i2 j2)][b2] Ts[(b u)][b2]
  const int M1 = d.nA2 * d.nI2 * d.nJ2, N1 = d.nB * d.pT;
  cta_gemm_scaled<T>(ex, M1, N1, d.nB2, R2, d.nB2, 1, Ts, 1, d.nB2, Y1, N1, false);
  // G2: Y2[(d a2)][(i j b)] = sum_{(u i2 j2)} C[(i j d)][(u i2 j2)] Y1[(a2 i2 j2)][(b u)]
  {
    constexpr int D3 = DK * DK * DK;
    const int ldy2 = d.nI * d.nJ * d.nB;
#pragma unroll 1
    for (int p = ex.tid(); p < d.nA2 * d.nB; p += ex.size()) {
      const int a2 = p / d.nB, b = p - (p / d.nB) * d.nB;
      const T* y1 = Y1 + a2 * d.nI2 * d.nJ2 * N1 + b * d.pT;
      T y[D3];
#pragma unroll
      for (int u = 0; u < DK; ++u)
#pragma unroll
        for (int i2 = 0; i2 < DK; ++i2)
#pragma unroll
          for (int j2 = 0; j2 < DK; ++j2)
            y[(u * DK + i2) * DK + j2] = (u < d.pT && i2 < d.nI2 && j2 < d.nJ2)
                                             ? y1[(i2 * d.nJ2 + j2) * N1 + u]
                                             : zero<T>();
#pragma unroll
      for (int i = 0; i < DK; ++i)
#pragma unroll
        for (int j = 0; j < DK; ++j)
#pragma unroll
          for (int dd = 0; dd < DK; ++dd) {
            if (i < d.nI && j < d.nJ && dd < d.pB) {
              const int k = (i * DK + j) * DK + dd;
              T s = zero<T>();
#pragma unroll
              for (int n = 0; n < D3; ++n) s = fmac(s, Cop[k * D3 + n], y[n]);
              Y2[(dd * d.nA2 + a2) * ldy2 + (i * d.nJ + j) * d.nB + b] = s;
            }
          }
    }
    ex.sync();
  }
  // G3: R[a][(i j b)] = sum_{(d a2)} Bs[a][(d a2)] Y2[(d a2)][(i j b)]
  return cta_gemm_scaled<T>(ex, d.nA, d.nI * d.nJ * d.nB, d.pB * d.nA2, Bs, d.pB * d.nA2, 1, Y2,
                            d.nI * d.nJ * d.nB, 1, out, d.nI * d.nJ * d.nB, true);
}

// ---------------------------------------------------------------------------
// Row (3-layer) steps.  E[a][l][b] = (nA, nH, nB).
// ---------------------------------------------------------------------------
struct RDims {
  int nA, nH, nB;
  int nA2, nH2, nB2;
  int pB, pT;
};

template <class T, int DK, class X>
__device__ __noinline__ int row_left(const X ex, const RDims& d, const T* L, const T* Bs, const T* W, const T* Ts,
                                       T* out, T* X1, T* X2, bool rescale = true) {
  // G1: X1[(l b)][(d a2)] = sum_a L[a][(l b)] Bs[a][(d a2)]
  const int Mlb = d.nH * d.nB, N1 = d.pB * d.nA2;
  cta_gemm_scaled<T>(ex, Mlb, N1, d.nA, L, 1, Mlb, Bs, N1, 1, X1, N1, false);
  // G2: X2[(a2 r)][(b u)] = sum_{l,d} X1[(l b)][(d a2)] W[l][r][d][u]
  {
    const int ldx2 = d.nB * d.pT;
#pragma unroll 1
    for (int p = ex.tid(); p < d.nB * d.nA2; p += ex.size()) {
      const int b = p / d.nA2, a2 = p - (p / d.nA2) * d.nA2;
      T x[DK][DK];
#pragma unroll
      for (int l = 0; l < DK; ++l)
#pragma unroll
        for (int dd = 0; dd < DK; ++dd)
          x[l][dd] = (l < d.nH && dd < d.pB) ? X1[(l * d.nB + b) * N1 + dd * d.nA2 + a2] : zero<T>();
      for (int r = 0; r < d.nH2; ++r)
        for (int u = 0; u < d.pT; ++u) {
          T s = zero<T>();
#pragma unroll
          for (int l = 0; l < DK; ++l)
#pragma unroll
            for (int dd = 0; dd < DK; ++dd)
              if (l < d.nH && dd < d.pB) s = fmac(s, x[l][dd], W[((l * DK + r) * DK + dd) * DK + u]);
          X2[(a2 * d.nH2 + r) * ldx2 + b * d.pT + u] = s;
        }
    }
    ex.sync();
  }
  // G3: out[(a2 r)][b2] = sum_{(b u)} X2[(a2 r)][(b u)] Ts[(b u)][b2]
  return cta_gemm_scaled<T>(ex, d.nA2 * d.nH2, d.nB2, d.nB * d.pT, X2, d.nB * d.pT, 1, Ts, d.nB2, 1, out,
                            d.nB2, rescale);
}

template <class T, int DK, class X>
__device__ __noinline__ int row_right(const X ex, const RDims& d, const T* R2, const T* Bs, const T* W, const T* Ts,
                                        T* out, T* Y1, T* Y2) {
  // G1: Y1[(a2 r)][(b u)] = sum_b2 R2[(a2 r)][b2] Ts[(b u)][b2]
  const int M1 = d.nA2 * d.nH2, N1 = d.nB * d.pT;
  cta_gemm_scaled<T>(ex, M1, N1, d.nB2, R2, d.nB2, 1, Ts, 1, d.nB2, Y1, N1, false);
  // G2: Y2[(d a2)][(l b)] = sum_{r,u} Y1[(a2 r)][(b u)] W[l][r][d][u]
  {
    const int ldy2 = d.nH * d.nB;
#pragma unroll 1
    for (int p = ex.tid(); p < d.nA2 * d.nB; p += ex.size()) {
      const int a2 = p / d.nB, b = p - (p / d.nB) * d.nB;
      T y[DK][DK];
#pragma unroll
      for (int r = 0; r < DK; ++r)
#pragma unroll
        for (int u = 0; u < DK; ++u)
          y[r][u] = (r < d.nH2 && u < d.pT) ? Y1[(a2 * d.nH2 + r) * N1 + b * d.pT + u] : zero<T>();
      for (int l = 0; l < d.nH; ++l)
        for (int dd = 0; dd < d.pB; ++dd) {
          T s = zero<T>();
#pragma unroll
          for (int r = 0; r < DK; ++r)
#pragma unroll
            for (int u = 0; u < DK; ++u)
              if (r < d.nH2 && u < d.pT) s = fmac(s, y[r][u], W[((l * DK + r) * DK + dd) * DK + u]);
          Y2[(dd * d.nA2 + a2) * ldy2 + l * d.nB + b] = s;
        }
    }
    ex.sync();
  }
  // G3: R[a][(l b)] = sum_{(d a2)} Bs[a][(d a2)] Y2[(d a2)][(l b)]
  return cta_gemm_scaled<T>(ex, d.nA, d.nH * d.nB, d.pB * d.nA2, Bs, d.pB * d.nA2, 1, Y2, d.nH * d.nB, 1,
                            out, d.nH * d.nB, true);
}

// Open tensor of one row vertex: G[l][r][d][u] = sum_{b,a2} X1[(l b)][(d a2)] Y1[(a2 r)][(b u)]
// with X1 = L.Bs (left G1) and Y1 = R2.Ts (right G1); written over the actual dims.
template <class T, int DK, class X>
__device__ __noinline__ void row_open(const X ex, const RDims& d, const T* L, const T* Bs, const T* Ts, const T* R2,
                                      T* G, T* X1, T* Y1) {
  const int Mlb = d.nH * d.nB, N1 = d.pB * d.nA2;
  cta_gemm_scaled<T>(ex, Mlb, N1, d.nA, L, 1, Mlb, Bs, N1, 1, X1, N1, false);
  const int M2 = d.nA2 * d.nH2, N2 = d.nB * d.pT;
  cta_gemm_scaled<T>(ex, M2, N2, d.nB2, R2, d.nB2, 1, Ts, 1, d.nB2, Y1, N2, false);
  const int lane = ex.lane(), wid = ex.warp(), nw = ex.nwarps();
  const int nout = d.nH * d.nH2 * d.pB * d.pT;
  const int K = d.nB * d.nA2;
  for (int o = wid; o < nout; o += nw) {
    int t = o;
    const int u = t % d.pT; t /= d.pT;
    const int dd = t % d.pB; t /= d.pB;
    const int r = t % d.nH2; t /= d.nH2;
    const int l = t;
    T s = zero<T>();
    for (int q = lane; q < K; q += 32) {
      const int b = q / d.nA2, a2 = q - (q / d.nA2) * d.nA2;
      s = fmac(s, X1[(l * d.nB + b) * N1 + dd * d.nA2 + a2], Y1[(a2 * d.nH2 + r) * N2 + b * d.pT + u]);
    }
    s = warp_sum_scalar(s);
    if (lane == 0) G[o] = s;
  }
  ex.sync();
}

}  // namespace gcf
