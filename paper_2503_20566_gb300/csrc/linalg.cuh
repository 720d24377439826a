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
template <class T, bool CA = false, bool CB = false, class X>
__device__ __noinline__ void cta_gemm(const X ex, int M, int N, int K, const T* A, int sAm, int sAk, const T* B,
                         int sBk, int sBn, T* C, int sCm, int sCn, bool accumulate) {
  if constexpr (!CA && !CB && MmaOk<T>::value) {
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

// In-place Householder QR of A (m x n): on return the upper triangle of the
// leading k = min(m,n) rows holds R, the part below the diagonal holds the
// reflector vectors, tau[0..k) their factors.  `red` is shared scratch (64 doubles).
template <class T, class X>
__device__ __noinline__ void cta_qr(const X ex, int m, int n, T* A, int sm, int sn, T* tau) {
  using R = typename Traits<T>::R;
  const int k = min(m, n);
  const int lane = ex.lane(), wid = ex.warp(), nw = ex.nwarps();
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
    const T ct = conjg(t);
    for (int c = j + 1 + wid; c < n; c += nw) {
      T w = zero<T>();
      for (int i = j + lane; i < m; i += 32) {
        const T v = (i == j) ? one<T>() : A[i * sm + j * sn];
        w = fmac(w, conjg(v), A[i * sm + c * sn]);
      }
      w = warp_sum_scalar(w);
      const T f = ct * w;
      for (int i = j + lane; i < m; i += 32) {
        const T v = (i == j) ? one<T>() : A[i * sm + j * sn];
        A[i * sm + c * sn] -= v * f;
      }
    }
    ex.sync();
  }
}

// Q = H_0 H_1 ... H_{k-1} restricted to its first k columns (m x k), from
// the reflectors stored by cta_qr in A.
template <class T, class X>
__device__ __noinline__ void cta_form_q(const X ex, int m, int k, const T* A, int sm, int sn, const T* tau, T* Q, int sQm,
                           int sQn) {
  const int lane = ex.lane(), wid = ex.warp(), nw = ex.nwarps();
#pragma unroll 1
  for (int idx = ex.tid(); idx < m * k; idx += ex.size()) {
    const int i = idx / k, c = idx - (idx / k) * k;
    Q[i * sQm + c * sQn] = (i == c) ? one<T>() : zero<T>();
  }
  ex.sync();
  for (int j = k - 1; j >= 0; --j) {
    const T t = tau[j];
    for (int c = j + wid; c < k; c += nw) {
      T w = zero<T>();
      for (int i = j + lane; i < m; i += 32) {
        const T v = (i == j) ? one<T>() : A[i * sm + j * sn];
        w = fmac(w, conjg(v), Q[i * sQm + c * sQn]);
      }
      w = warp_sum_scalar(w);
      const T f = t * w;
      for (int i = j + lane; i < m; i += 32) {
        const T v = (i == j) ? one<T>() : A[i * sm + j * sn];
        Q[i * sQm + c * sQn] -= v * f;
      }
    }
    ex.sync();
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
template <class T, class X>
__device__ __noinline__ int cta_jacobi_svd(const X ex, int p, int q, T* W, int sWm, int sWn, T* J, int sJm, int sJn,
                              int* sflag, int max_sweeps, int* converged) {
  using R = typename Traits<T>::R;
  const int lane = ex.lane(), wid = ex.warp(), nw = ex.nwarps();
#pragma unroll 1
  for (int idx = ex.tid(); idx < q * q; idx += ex.size()) {
    const int i = idx / q, c = idx - (idx / q) * q;
    J[i * sJm + c * sJn] = (i == c) ? one<T>() : zero<T>();
  }
  const int n = q + (q & 1);
  const R tol = R(8) * Traits<T>::eps();
  int sweep = 0;
  if (converged) *converged = 1;
  for (; sweep < max_sweeps; ++sweep) {
    if (ex.tid() == 0) *sflag = 0;
    ex.sync();
    for (int r = 0; r < n - 1; ++r) {
      for (int kp = wid; kp < n / 2; kp += nw) {
        int a, b;
        if (kp == 0) { a = r % (n - 1); b = n - 1; }
        else { a = (r + kp) % (n - 1); b = (r - kp + n - 1) % (n - 1); }
        if (a >= q || b >= q) continue;
        if (a > b) { int t = a; a = b; b = t; }
        R al = R(0), be = R(0);
        T g = zero<T>();
        for (int i = lane; i < p; i += 32) {
          const T wa = W[i * sWm + a * sWn], wb = W[i * sWm + b * sWn];
          al += abs2(wa);
          be += abs2(wb);
          g = fmac(g, conjg(wa), wb);
        }
        al = warp_sum(al); be = warp_sum(be); g = warp_sum_scalar(g);
        const R gr = re(g), gi = im(g);
        const R ga = sqrt(gr * gr + gi * gi);
        if (ga == R(0) || !(ga > tol * sqrt(al * be))) continue;
        const R zeta = (be - al) / (R(2) * ga);
        const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
        const R c = R(1) / sqrt(R(1) + t * t), s = c * t;
        // G = [[c, s e^{i phi}], [-s e^{-i phi}, c]], e^{i phi} = g / |g|
        const T eph = make_scalar<T>(gr / ga, gi / ga);
        const T s_e = scale(eph, (R)s);                 // s e^{i phi}
        const T s_ec = scale(conjg(eph), (R)s);         // s e^{-i phi}
        for (int i = lane; i < p; i += 32) {
          const T wa = W[i * sWm + a * sWn], wb = W[i * sWm + b * sWn];
          W[i * sWm + a * sWn] = scale(wa, (R)c) - wb * s_ec;
          W[i * sWm + b * sWn] = wa * s_e + scale(wb, (R)c);
        }
        for (int i = lane; i < q; i += 32) {
          const T ja = J[i * sJm + a * sJn], jb = J[i * sJm + b * sJn];
          J[i * sJm + a * sJn] = scale(ja, (R)c) - jb * s_ec;
          J[i * sJm + b * sJn] = ja * s_e + scale(jb, (R)c);
        }
        if (lane == 0) *sflag = 1;
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
