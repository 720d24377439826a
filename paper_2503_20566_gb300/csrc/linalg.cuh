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

}  // namespace gcf
