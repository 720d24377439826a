// CTA-cooperative dense linear algebra on small matrices (one chain per CTA):
// strided GEMM, Householder QR / LQ and one-sided Jacobi SVD.
//
// Every routine is called by all threads of the CTA with identical arguments;
// matrices live in global scratch or shared memory and are addressed through
// (row stride, column stride), so transposed views cost nothing.  Routines
// end with ex.sync() so their results are visible on return.
//
// The algorithms are the textbook ones: Householder QR (Golub & Van Loan,
// "Matrix Computations", Alg. 5.1.1 / 5.2.1, with the complex reflector that
// maps x to -sign(Re x_1) |x| e_1) and the one-sided (Hestenes) Jacobi SVD
// with the round-robin pair schedule.
#pragma once

#include "common.cuh"
#include "mma.cuh"

namespace gcf {

// C (M x N) = A (M x K) B (K x N) in FP32, strided operands in shared or
// global memory: each thread accumulates 4 x 4 tiles of C in registers, so a
// multiply-add costs half a load instead of two.  C must not overlap A or B.
template <class X>
__device__ __noinline__ void tile_gemm_f32(const X ex, int M, int N, int K, const float* A, int sAm, int sAk,
                                           const float* B, int sBk, int sBn, float* C, int sCm, int sCn) {
  const int tm = (M + 3) >> 2, tn = (N + 3) >> 2;
#pragma unroll 1
  for (int t = ex.tid(); t < tm * tn; t += ex.size()) {
    const int i0 = (t / tn) << 2, j0 = (t - (t / tn) * tn) << 2;
    const float* ap[4];
    const float* bp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      ap[q] = A + min(i0 + q, M - 1) * sAm;  // rows / columns past the edge repeat the last one
      bp[q] = B + min(j0 + q, N - 1) * sBn;
    }
    float acc[4][4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[q][r] = 0.f;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      float a[4], b[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        a[q] = ap[q][k * sAk];
        b[q] = bp[q][k * sBk];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[q][r] = fmaf(a[q], b[r], acc[q][r]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (i0 + q < M && j0 + r < N) C[(i0 + q) * sCm + (j0 + r) * sCn] = acc[q][r];
  }
  ex.sync();
}

// C(i,j) = [C(i,j) +] sum_k op(A)(i,k) op(B)(k,j); op = optional conjugation.
// TC = false keeps the product in the scalar's own precision whatever the
// chain's GEMM mode (the factorisations' own products).
template <class T, bool CA = false, bool CB = false, bool TC = true, class X>
__device__ __noinline__ void cta_gemm(const X ex, int M, int N, int K, const T* A, int sAm, int sAk, const T* B,
                         int sBk, int sBn, T* C, int sCm, int sCn, bool accumulate) {
  if constexpr (TC && !CA && !CB && MmaOk<T>::value) {
    const int mode = g_gemm_mode[ex.slot()];
    if (mode != GEMM_FFMA) {
      if (mode == GEMM_BF16)
        mma_gemm<T, GEMM_BF16>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, sCm, sCn, accumulate);
      else
        mma_gemm<T, GEMM_TF32X3>(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, sCm, sCn, accumulate);
      ex.sync();
      return;
    }
  }
  if constexpr (std::is_same<T, float>::value) {
    // the same sum over k in the same order, from register tiles, when the
    // product has a 4 x 4 tile for every thread
    if (!accumulate && M >= 4 && (long long)M * N >= 16LL * ex.size()) {
      tile_gemm_f32(ex, M, N, K, A, sAm, sAk, B, sBk, sBn, C, sCm, sCn);
      return;
    }
  }
  const int MN = M * N;
#pragma unroll 1
  for (int idx = ex.tid(); idx < MN; idx += ex.size()) {
    const int i = idx / N, j = idx - (idx / N) * N;
    T s = accumulate ? C[i * sCm + j * sCn] : zero<T>();
    const T* a = A + i * sAm;
    const T* b = B + j * sBn;
    for (int k = 0; k < K; ++k) {
      T av = a[k * sAk], bv = b[k * sBk];
      if (CA) av = conjg(av);
      if (CB) bv = conjg(bv);
      s = fmac(s, av, bv);
    }
    C[i * sCm + j * sCn] = s;
  }
  ex.sync();
}


// Householder reflector for column (alpha; x) with |x|^2 = xn2, in the
// scalar's own precision: H = I - tau v v^H, v = (1; x * scal),
// H^H (alpha; x) = (beta; 0), beta real.
template <class T>
__device__ inline void householder(T alpha, typename Traits<T>::R xn2, T& tau, T& scal, T& beta) {
  using R = typename Traits<T>::R;
  const R ar = re(alpha), ai = im(alpha);
  if (xn2 == R(0) && ai == R(0)) {
    tau = zero<T>(); scal = zero<T>(); beta = alpha;
    return;
  }
  R b = sqrt(ar * ar + ai * ai + xn2);
  if (ar >= R(0)) b = -b;
  tau = make_scalar<T>((b - ar) / b, -ai / b);
  const R dr = ar - b, di = ai;
  const R d2 = dr * dr + di * di;
  scal = make_scalar<T>(dr / d2, -di / d2);
  beta = make_scalar<T>(b, R(0));
}

// Sum of v over the L consecutive lanes (L a power of two <= 32, aligned)
// that share a column pair; every lane of the warp must call it.
template <class R>
__device__ __forceinline__ R lanes_sum(R v, int L) {
#pragma unroll 1
  for (int o = L >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Reciprocal and reciprocal square root of the Jacobi rotation parameters:
// the hardware approximations in FP32 (a rotation need only be orthogonal to
// rounding, and the accumulated J is re-orthogonalised after the sweeps),
// exact in FP64.
__device__ __forceinline__ float jrcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double jrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float jrsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double jrsqrt(double x) { return 1.0 / sqrt(x); }

// Lanes per column for `cols` independent column operations on the
// executor: the largest power of two <= 32 whose groups of lanes cover every
// column at once (1 if the columns outnumber the threads).
template <class X>
__device__ __forceinline__ int lanes_per_column(const X ex, int cols) {
  int L = 32;
  while (L > 1 && L * cols > ex.size()) L >>= 1;
  return L;
}

template <class T>
__device__ __forceinline__ T lanes_sum_scalar(T v, int L);
template <>
__device__ __forceinline__ float lanes_sum_scalar<float>(float v, int L) { return lanes_sum(v, L); }
template <>
__device__ __forceinline__ double lanes_sum_scalar<double>(double v, int L) { return lanes_sum(v, L); }
template <>
__device__ __forceinline__ cfloat lanes_sum_scalar<cfloat>(cfloat v, int L) {
  return {lanes_sum(v.x, L), lanes_sum(v.y, L)};
}
template <>
__device__ __forceinline__ cdouble lanes_sum_scalar<cdouble>(cdouble v, int L) {
  return {lanes_sum(v.x, L), lanes_sum(v.y, L)};
}

// Apply the reflector H = I - f v v^H (v = (1; A[j+1.., j])) from the left
// to columns c0 .. c1-1 of M (rows j..m-1): w_c = v^H M_c, M_c -= v (f w_c).
// Each column is served by a group of L lanes that split its rows and sum
// their parts by shuffles, so that all columns proceed at once.
template <class T, class X>
__device__ __forceinline__ void apply_reflector(const X ex, int m, int j, const T* A, int sm, int sn, T f,
                                                T* Mt, int sMm, int sMn, int c0, int c1) {
  const int nc = c1 - c0;
  if (nc <= 0) return;
  const int L = lanes_per_column(ex, nc);
  const int slots = ex.size() / L;
  const int sub = ex.tid() / L, li = ex.tid() - (ex.tid() / L) * L;
  const T* vcol = A + j * sn;  // v_i = A[i][j] below the diagonal, v_j = 1
#pragma unroll 1
  for (int base = 0; base < nc; base += slots) {
    const int c = c0 + base + sub;
    const bool act = c < c1;
    T* mc = Mt + c * sMn;
    T w = zero<T>();
    if (act) {
#pragma unroll 2
      for (int i = j + li; i < m; i += L) {
        const T v = (i == j) ? one<T>() : vcol[i * sm];
        w = fmac(w, conjg(v), mc[i * sMm]);
      }
    }
    w = lanes_sum_scalar(w, L);
    if (act) {
      const T g = f * w;
#pragma unroll 2
      for (int i = j + li; i < m; i += L) {
        const T v = (i == j) ? one<T>() : vcol[i * sm];
        mc[i * sMm] -= v * g;
      }
    }
  }
}

// In-place Householder QR of A (m x n): on return the upper triangle of the
// leading k = min(m,n) rows holds R, the part below the diagonal holds the
// reflector vectors, tau[0..k) their factors.
template <class T, class X>
__device__ __noinline__ void cta_qr(const X ex, int m, int n, T* A, int sm, int sn, T* tau) {
  using R = typename Traits<T>::R;
  const int k = min(m, n);
  for (int j = 0; j < k; ++j) {
    R part = R(0);
#pragma unroll 1
    for (int i = j + 1 + ex.tid(); i < m; i += ex.size()) part += abs2(A[i * sm + j * sn]);
    const R xn2 = ex.template sum<R>(part);
    const T alpha = A[j * sm + j * sn];
    T t, sc, beta;
    householder(alpha, xn2, t, sc, beta);
    ex.sync();
#pragma unroll 1
    for (int i = j + 1 + ex.tid(); i < m; i += ex.size()) A[i * sm + j * sn] = A[i * sm + j * sn] * sc;
    if (ex.tid() == 0) { A[j * sm + j * sn] = beta; tau[j] = t; }
    ex.sync();
    apply_reflector(ex, m, j, A, sm, sn, conjg(t), A, sm, sn, j + 1, n);
    ex.sync();
  }
}

// Q = H_0 H_1 ... H_{k-1} restricted to its first k columns (m x k), from
// the reflectors stored by cta_qr in A.
template <class T, class X>
__device__ __noinline__ void cta_form_q(const X ex, int m, int k, const T* A, int sm, int sn, const T* tau, T* Q, int sQm,
                           int sQn) {
#pragma unroll 1
  for (int idx = ex.tid(); idx < m * k; idx += ex.size()) {
    const int i = idx / k, c = idx - (idx / k) * k;
    Q[i * sQm + c * sQn] = (i == c) ? one<T>() : zero<T>();
  }
  ex.sync();
  for (int j = k - 1; j >= 0; --j) {
    apply_reflector(ex, m, j, A, sm, sn, tau[j], Q, sQm, sQn, j, k);
    ex.sync();
  }
}

// Column length of the column-major FP32 workspaces below: rows rounded up
// to whole 16-byte chunks of four floats.
__host__ __device__ inline int jac_ld(int rows) { return (rows + 3) & ~3; }

// Chunk kk (rows 4kk .. 4kk+3) of the reflector v of column j of a
// column-major A: 0 above row j, 1 at row j, sc A[i][j] below (the stored
// column before its scaling).
__device__ __forceinline__ float4 reflector_chunk(const float4* aj, int kk, int j, float sc) {
  float4 x = aj[kk];
  if (kk == (j >> 2)) {
    const int r0 = kk << 2;
    x.x = (r0 < j) ? 0.f : (r0 == j ? 1.f : sc * x.x);
    x.y = (r0 + 1 < j) ? 0.f : (r0 + 1 == j ? 1.f : sc * x.y);
    x.z = (r0 + 2 < j) ? 0.f : (r0 + 2 == j ? 1.f : sc * x.z);
    x.w = (r0 + 3 < j) ? 0.f : (r0 + 3 == j ? 1.f : sc * x.w);
  } else {
    x.x *= sc; x.y *= sc; x.z *= sc; x.w *= sc;
  }
  return x;
}

__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, acc))));
}

// cta_qr for real FP32 on a column-major shared-memory A (m x n, column c at
// A + c lda, lda = jac_ld(m), 16-byte aligned, padding rows zero): the same
// Householder reflectors (householder()), stored the same way (R on and
// above the diagonal, the scaled v below it, tau[0..min(m,n))).  Per
// column one barrier: the lanes that apply H_j to column j+1 also reduce
// that column's next norm and diagonal entry and publish them, and the
// scaling of column j's v is done in the next step, when nothing reads it.
template <class X>
__device__ __noinline__ void qr_cm(const X ex, int m, int n, float* A, int lda, float* tau) {
  const int k = min(m, n);
  const int cw = lda >> 2;
  // two (alpha, |x|^2) slots, alternating between steps
  float* pub = reinterpret_cast<float*>(g_exec_red[ex.slot()]) + 120;
  float part = 0.f;
#pragma unroll 1
  for (int i = 1 + ex.tid(); i < m; i += ex.size()) part = fmaf(A[i], A[i], part);
  float xn2 = ex.template sum<float>(part);
  float alpha = A[0];
  float sc_p = 0.f, t_p = 0.f, beta_p = 0.f;
  for (int j = 0; j < k; ++j) {
    if (j > 0) {
      alpha = pub[2 * (j & 1)];
      xn2 = pub[2 * (j & 1) + 1];
    }
    float t, sc, beta;
    householder(alpha, xn2, t, sc, beta);
    if (j > 0) {
      // column j-1: scaled v below the diagonal, beta on it
      float* ap = A + (j - 1) * lda;
#pragma unroll 1
      for (int i = j + ex.tid(); i < m; i += ex.size()) ap[i] *= sc_p;
      if (ex.tid() == 0) { ap[j - 1] = beta_p; tau[j - 1] = t_p; }
    }
    const int c0 = j + 1, nc = n - c0;
    if (nc > 0) {
      const int L = lanes_per_column(ex, nc);
      const int slots = ex.size() / L;
      const int sub = ex.tid() / L, li = ex.tid() - (ex.tid() / L) * L;
      const float4* aj = reinterpret_cast<const float4*>(A + j * lda);
      const int kb = j >> 2;
#pragma unroll 1
      for (int base = 0; base < nc; base += slots) {
        const int c = c0 + base + sub;
        const bool act = c < n;
        float4* mc = reinterpret_cast<float4*>(A + c * lda);
        float w = 0.f;
        if (act) {
#pragma unroll 2
          for (int kk = kb + li; kk < cw; kk += L) w = dot4(reflector_chunk(aj, kk, j, sc), mc[kk], w);
        }
        w = lanes_sum(w, L);
        const bool next = act && c == j + 1 && c < k;
        float nn = 0.f, al = 0.f;
        if (act) {
          const float g = t * w;
#pragma unroll 2
          for (int kk = kb + li; kk < cw; kk += L) {
            const float4 x = reflector_chunk(aj, kk, j, sc);
            float4 y = mc[kk];
            y.x = fmaf(-g, x.x, y.x); y.y = fmaf(-g, x.y, y.y); y.z = fmaf(-g, x.z, y.z); y.w = fmaf(-g, x.w, y.w);
            mc[kk] = y;
            if (next) {
              const int r0 = kk << 2;
              const float e[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                if (r0 + q > c) nn = fmaf(e[q], e[q], nn);
                if (r0 + q == c) al = e[q];
              }
            }
          }
        }
        // every lane of the warp joins the shuffles; only the pivot's lanes
        // hold non-zero parts
#pragma unroll 1
        for (int o = L >> 1; o > 0; o >>= 1) {
          nn += __shfl_xor_sync(0xffffffffu, nn, o);
          al += __shfl_xor_sync(0xffffffffu, al, o);
        }
        if (next && li == 0) {
          pub[2 * ((j + 1) & 1)] = al;
          pub[2 * ((j + 1) & 1) + 1] = nn;
        }
      }
    }
    sc_p = sc; t_p = t; beta_p = beta;
    ex.sync();
  }
  if (k > 0) {
    float* ap = A + (k - 1) * lda;
#pragma unroll 1
    for (int i = k + ex.tid(); i < m; i += ex.size()) ap[i] *= sc_p;
    if (ex.tid() == 0) { ap[k - 1] = beta_p; tau[k - 1] = t_p; }
  }
  ex.sync();
}

// cta_form_q for the column-major A of qr_cm: Q (m x kq, column c at
// Q + c ldq, ldq = jac_ld(m), 16-byte aligned) = H_0 ... H_{kq-1} applied to
// the first kq columns of the identity, the reflectors applied last to
// first.
template <class X>
__device__ __noinline__ void form_q_cm(const X ex, int m, int kq, const float* A, int lda, const float* tau, float* Q,
                                       int ldq) {
#pragma unroll 1
  for (int idx = ex.tid(); idx < kq * ldq; idx += ex.size()) {
    const int c = idx / ldq, i = idx - (idx / ldq) * ldq;
    Q[idx] = (i == c) ? 1.f : 0.f;
  }
  ex.sync();
  const int cw = ldq >> 2;
  for (int j = kq - 1; j >= 0; --j) {
    const float t = tau[j];
    const int nc = kq - j;
    const int L = lanes_per_column(ex, nc);
    const int slots = ex.size() / L;
    const int sub = ex.tid() / L, li = ex.tid() - (ex.tid() / L) * L;
    const float4* aj = reinterpret_cast<const float4*>(A + j * lda);
    const int kb = j >> 2;
#pragma unroll 1
    for (int base = 0; base < nc; base += slots) {
      const int c = j + base + sub;
      const bool act = c < kq;
      float4* qc = reinterpret_cast<float4*>(Q + c * ldq);
      float w = 0.f;
      if (act) {
#pragma unroll 2
        for (int kk = kb + li; kk < cw; kk += L) w = dot4(reflector_chunk(aj, kk, j, 1.f), qc[kk], w);
      }
      w = lanes_sum(w, L);
      if (act) {
        const float g = t * w;
#pragma unroll 2
        for (int kk = kb + li; kk < cw; kk += L) {
          const float4 x = reflector_chunk(aj, kk, j, 1.f);
          float4 y = qc[kk];
          y.x = fmaf(-g, x.x, y.x); y.y = fmaf(-g, x.y, y.y); y.z = fmaf(-g, x.z, y.z); y.w = fmaf(-g, x.w, y.w);
          qc[kk] = y;
        }
      }
    }
    ex.sync();
  }
}

// Shared-memory factorisation workspace of each chain group: the QR / Q
// formation and the Jacobi sweeps run on shared-memory copies of their
// matrices when they fit (every step of these factorisations depends on the
// previous one, so each access would otherwise wait on L2).  Set at kernel
// entry; null when the launch has none.
__shared__ void* g_fz[4];
__shared__ long long g_fz_elems;  // scalars of each workspace

template <class T, class X>
__device__ inline void cta_copy(const X ex, int rows, int cols, const T* src, int lds, T* dst, int ldd) {
#pragma unroll 1
  for (int idx = ex.tid(); idx < rows * cols; idx += ex.size()) {
    const int i = idx / cols, j = idx - (idx / cols) * cols;
    dst[i * ldd + j] = src[i * lds + j];
  }
  ex.sync();
}

// A (m x n, row stride lda) <- its Householder QR in place (cta_qr) and
// Q (m x kq, row stride ldq) <- the first kq columns of the orthogonal factor
// (cta_form_q), in the chain's shared-memory workspace when both fit.
template <class T, class X>
__device__ __noinline__ void qr_with_q(const X ex, int m, int n, T* A, int lda, T* tau, int kq, T* Q, int ldq) {
  T* fz = (T*)g_fz[ex.slot()];
  if constexpr (std::is_same<T, float>::value) {
    // FP32: column-major copies in 16-byte chunks (qr_cm, form_q_cm)
    const int ld = jac_ld(m);
    if (fz && (long long)ld * (n + kq) <= g_fz_elems) {
      float* a = fz;
      float* q = fz + ld * n;
#pragma unroll 1
      for (int idx = ex.tid(); idx < n * ld; idx += ex.size()) {
        const int c = idx / ld, i = idx - (idx / ld) * ld;
        a[idx] = (i < m) ? A[i * lda + c] : 0.f;
      }
      ex.sync();
      qr_cm(ex, m, n, a, ld, tau);
      form_q_cm(ex, m, kq, a, ld, tau, q, ld);
#pragma unroll 1
      for (int idx = ex.tid(); idx < n * m; idx += ex.size()) {
        const int c = idx / m, i = idx - (idx / m) * m;
        A[i * lda + c] = a[c * ld + i];
      }
#pragma unroll 1
      for (int idx = ex.tid(); idx < kq * m; idx += ex.size()) {
        const int c = idx / m, i = idx - (idx / m) * m;
        Q[i * ldq + c] = q[c * ld + i];
      }
      ex.sync();
      return;
    }
  }
  if (fz && (long long)m * n + (long long)m * kq <= g_fz_elems) {
    T* a = fz;
    T* q = fz + m * n;
    cta_copy(ex, m, n, A, lda, a, n);
    cta_qr<T>(ex, m, n, a, n, 1, tau);
    cta_form_q<T>(ex, m, kq, a, n, 1, tau, q, kq, 1);
    cta_copy(ex, m, n, a, n, A, lda);
    cta_copy(ex, m, kq, q, kq, Q, ldq);
  } else {
    cta_qr<T>(ex, m, n, A, lda, 1, tau);
    cta_form_q<T>(ex, m, kq, A, lda, 1, tau, Q, ldq, 1);
  }
}

// Copy with optional conjugate-transpose: dst(i,j) = src(j,i)^* for i<rows, j<cols.
template <class T, class X>
__device__ __noinline__ void cta_adjoint(const X ex, int rows, int cols, const T* src, int sSm, int sSn, T* dst, int sDm,
                            int sDn) {
#pragma unroll 1
  for (int idx = ex.tid(); idx < rows * cols; idx += ex.size()) {
    const int i = idx / cols, j = idx - (idx / cols) * cols;
    dst[i * sDm + j * sDn] = conjg(src[j * sSm + i * sSn]);
  }
  ex.sync();
}

// One-sided Jacobi on the columns of W (p x q), accumulating J (q x q, reset
// to the identity here) so that on return W = W_in J has mutually orthogonal
// columns.  Returns the number of sweeps used; *converged set to 0 if the
// sweep limit was hit.  sflag: shared int scratch.
// Each sweep visits every column pair once in the round-robin order (n - 1
// rounds of n/2 disjoint pairs, n = q rounded up to even).  A pair is served
// by L consecutive lanes (the largest power of two <= 32 with L x n/2 within
// the executor), which split its rows and combine their partial sums by
// shuffles, so that all pairs of a round proceed at once.
template <class T, class X>
__device__ __noinline__ int cta_jacobi_svd(const X ex, int p, int q, T* W, int sWm, int sWn, T* J, int sJm, int sJn,
                              int* sflag, int max_sweeps, int* converged) {
  using R = typename Traits<T>::R;
#pragma unroll 1
  for (int idx = ex.tid(); idx < q * q; idx += ex.size()) {
    const int i = idx / q, c = idx - (idx / q) * q;
    J[i * sJm + c * sJn] = (i == c) ? one<T>() : zero<T>();
  }
  const int n = q + (q & 1);
  const int npair = n / 2;
  int L = 32;
  while (L > 1 && L * npair > ex.size()) L >>= 1;
  const int slots = ex.size() / L;
  const int sub = ex.tid() / L, li = ex.tid() - (ex.tid() / L) * L;
  // convergence threshold on |w_a^H w_b| / (|w_a| |w_b|): the rounding of a
  // length-p dot product is about sqrt(p) eps, below which rotations only
  // stir noise (the threshold of LAPACK's one-sided Jacobi, xGESVJ, scaled
  // by 4)
  const R tol = R(4) * sqrt(R(p > 4 ? p : 4)) * Traits<T>::eps();
  // a column whose norm is below eps ||W||_F (rotations keep ||W||_F) is
  // rounding noise of the matrix: pairs with one are left as they are
  R f2 = R(0);
#pragma unroll 1
  for (int idx = ex.tid(); idx < p * q; idx += ex.size()) {
    const int i = idx / q, c = idx - (idx / q) * q;
    f2 += abs2(W[i * sWm + c * sWn]);
  }
  f2 = ex.template sum<R>(f2);
  const R negl = Traits<T>::eps() * Traits<T>::eps() * f2;
  int sweep = 0;
  if (converged) *converged = 1;
  for (; sweep < max_sweeps; ++sweep) {
    if (ex.tid() == 0) *sflag = 0;
    ex.sync();
#pragma unroll 1
    for (int r = 0; r < n - 1; ++r) {
#pragma unroll 1
      for (int base = 0; base < npair; base += slots) {
        const int kp = base + sub;
        // round-robin pair kp of round r: (r + kp, r - kp) mod (n - 1), and
        // (r, n - 1) for kp = 0; kp < n/2 keeps each sum within one period
        int a = r, b = n - 1;
        if (kp > 0) {
          a = r + kp;
          if (a >= n - 1) a -= n - 1;
          b = r - kp;
          if (b < 0) b += n - 1;
        }
        if (a > b) { const int t = a; a = b; b = t; }
        const bool act = kp < npair && b < q;
        const int rstep = L * sWm;
        T* pa = W + li * sWm + a * sWn;
        T* pb = W + li * sWm + b * sWn;
        R al = R(0), be = R(0), gr = R(0), gi = R(0);
        if (act) {
          T g = zero<T>();
#pragma unroll 2
          for (int i = li, o = 0; i < p; i += L, o += rstep) {
            const T wa = pa[o], wb = pb[o];
            al += abs2(wa);
            be += abs2(wb);
            g = fmac(g, conjg(wa), wb);
          }
          gr = re(g);
          gi = im(g);
        }
        al = lanes_sum(al, L);
        be = lanes_sum(be, L);
        gr = lanes_sum(gr, L);
        gi = lanes_sum(gi, L);
        const R ga = sqrt(gr * gr + gi * gi);
        // sqrt(al) sqrt(be), not sqrt(al be): the product of two small squared
        // norms can underflow, and a zero threshold would rotate rounding
        // noise forever
        if (!act || ga == R(0) || !(al > negl) || !(be > negl) || !(ga > tol * (sqrt(al) * sqrt(be)))) continue;
        const R iga = jrcp(ga);
        const R zeta = (be - al) * (R(0.5) * iga);
        // tan of the rotation angle; for |zeta| beyond 1e15, zeta^2 would
        // overflow in FP32, and t = 1 / (2 zeta) to rounding
        const R az = fabs(zeta);
        const R t = (zeta >= R(0) ? R(1) : R(-1)) * jrcp(az > R(1e15) ? R(2) * az : az + sqrt(R(1) + zeta * zeta));
        if (t == R(0)) continue;  // a rotation below rounding leaves the pair as it is
        const R c = jrsqrt(R(1) + t * t), s = c * t;
        // G = [[c, s e^{i phi}], [-s e^{-i phi}, c]], e^{i phi} = g / |g|
        const T eph = make_scalar<T>(gr * iga, gi * iga);
        const T s_e = scale(eph, (R)s);                 // s e^{i phi}
        const T s_ec = scale(conjg(eph), (R)s);         // s e^{-i phi}
#pragma unroll 2
        for (int i = li, o = 0; i < p; i += L, o += rstep) {
          const T wa = pa[o], wb = pb[o];
          pa[o] = scale(wa, (R)c) - wb * s_ec;
          pb[o] = wa * s_e + scale(wb, (R)c);
        }
        T* ja_p = J + li * sJm + a * sJn;
        T* jb_p = J + li * sJm + b * sJn;
        const int jstep = L * sJm;
#pragma unroll 2
        for (int i = li, o = 0; i < q; i += L, o += jstep) {
          const T ja = ja_p[o], jb = jb_p[o];
          ja_p[o] = scale(ja, (R)c) - jb * s_ec;
          jb_p[o] = ja * s_e + scale(jb, (R)c);
        }
        if (li == 0) *sflag = 1;
      }
      ex.sync();
    }
    const int any = *sflag;
    ex.sync();
    if (!any) break;
  }
  if (sweep >= max_sweeps && converged) *converged = 0;
  ex.sync();
  return sweep;
}

// cta_jacobi_svd for real FP32 on a column-major shared-memory workspace:
// W (p x q, column c at W + c ldw) and J (q x q, column c at J + c ldj), with
// ldw = jac_ld(p), ldj = jac_ld(q), 16-byte aligned, the padding rows of W
// zero (rotations keep them zero).  The same rotations in the same round-
// robin order; a pair's L lanes split its columns into chunks of four rows
// (chunk k to lane k mod L) and move each chunk with one 16-byte access, so a
// round costs a quarter of the shared-memory instructions and address
// arithmetic of the strided form.
template <class X>
__device__ __noinline__ int jacobi_svd_cm(const X ex, int p, int q, float* W, int ldw, float* J, int ldj, int* sflag,
                                          int max_sweeps, int* converged) {
#pragma unroll 1
  for (int idx = ex.tid(); idx < q * ldj; idx += ex.size()) {
    const int c = idx / ldj, i = idx - (idx / ldj) * ldj;
    J[idx] = (i == c) ? 1.f : 0.f;
  }
  const int n = q + (q & 1);
  const int npair = n / 2;
  int L = 32;
  while (L > 1 && L * npair > ex.size()) L >>= 1;
  const int slots = ex.size() / L;
  const int sub = ex.tid() / L, li = ex.tid() - (ex.tid() / L) * L;
  const int cw = ldw >> 2, cj = ldj >> 2;  // chunks per column
  const float tol = 4.f * sqrtf((float)(p > 4 ? p : 4)) * Traits<float>::eps();
  float f2 = 0.f;
#pragma unroll 1
  for (int idx = ex.tid(); idx < q * ldw; idx += ex.size()) f2 += W[idx] * W[idx];
  f2 = ex.template sum<float>(f2);
  const float negl = Traits<float>::eps() * Traits<float>::eps() * f2;
  int sweep = 0;
  if (converged) *converged = 1;
  for (; sweep < max_sweeps; ++sweep) {
    if (ex.tid() == 0) *sflag = 0;
    ex.sync();
#pragma unroll 1
    for (int r = 0; r < n - 1; ++r) {
#pragma unroll 1
      for (int base = 0; base < npair; base += slots) {
        const int kp = base + sub;
        int a = r, b = n - 1;
        if (kp > 0) {
          a = r + kp;
          if (a >= n - 1) a -= n - 1;
          b = r - kp;
          if (b < 0) b += n - 1;
        }
        if (a > b) { const int t = a; a = b; b = t; }
        const bool act = kp < npair && b < q;
        float4* pa = reinterpret_cast<float4*>(W + a * ldw);
        float4* pb = reinterpret_cast<float4*>(W + b * ldw);
        float al = 0.f, be = 0.f, g = 0.f;
        if (act) {
#pragma unroll 3
          for (int k = li; k < cw; k += L) {
            const float4 x = pa[k], y = pb[k];
            al = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, al))));
            be = fmaf(y.x, y.x, fmaf(y.y, y.y, fmaf(y.z, y.z, fmaf(y.w, y.w, be))));
            g = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, g))));
          }
        }
        // the three sums together, offsets L/2 .. 1 as in lanes_sum
#pragma unroll 1
        for (int o = L >> 1; o > 0; o >>= 1) {
          al += __shfl_xor_sync(0xffffffffu, al, o);
          be += __shfl_xor_sync(0xffffffffu, be, o);
          g += __shfl_xor_sync(0xffffffffu, g, o);
        }
        const float ga = fabsf(g);
        if (!act || ga == 0.f || !(al > negl) || !(be > negl) || !(ga > tol * (sqrtf(al) * sqrtf(be)))) continue;
        const float iga = jrcp(ga);
        const float zeta = (be - al) * (0.5f * iga);
        const float az = fabsf(zeta);
        const float t = (zeta >= 0.f ? 1.f : -1.f) * jrcp(az > 1e15f ? 2.f * az : az + sqrtf(1.f + zeta * zeta));
        if (t == 0.f) continue;
        const float c = jrsqrt(1.f + t * t);
        const float s = (g >= 0.f ? c : -c) * t;  // s e^{i phi}, e^{i phi} = sign(g)
#pragma unroll 3
        for (int k = li; k < cw; k += L) {
          const float4 x = pa[k], y = pb[k];
          pa[k] = make_float4(fmaf(c, x.x, -s * y.x), fmaf(c, x.y, -s * y.y), fmaf(c, x.z, -s * y.z),
                              fmaf(c, x.w, -s * y.w));
          pb[k] = make_float4(fmaf(s, x.x, c * y.x), fmaf(s, x.y, c * y.y), fmaf(s, x.z, c * y.z),
                              fmaf(s, x.w, c * y.w));
        }
        float4* ja = reinterpret_cast<float4*>(J + a * ldj);
        float4* jb = reinterpret_cast<float4*>(J + b * ldj);
#pragma unroll 3
        for (int k = li; k < cj; k += L) {
          const float4 x = ja[k], y = jb[k];
          ja[k] = make_float4(fmaf(c, x.x, -s * y.x), fmaf(c, x.y, -s * y.y), fmaf(c, x.z, -s * y.z),
                              fmaf(c, x.w, -s * y.w));
          jb[k] = make_float4(fmaf(s, x.x, c * y.x), fmaf(s, x.y, c * y.y), fmaf(s, x.z, c * y.z),
                              fmaf(s, x.w, c * y.w));
        }
        if (li == 0) *sflag = 1;
      }
      ex.sync();
    }
    const int any = *sflag;
    ex.sync();
    if (!any) break;
  }
  if (sweep >= max_sweeps && converged) *converged = 0;
  ex.sync();
  return sweep;
}

}  // namespace gcf
