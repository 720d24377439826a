// Device layer of the GCF-PEPS contraction: sector gather (Sec. S-2, Eq. S5),
// boundary-MPS row absorption with QR / LQ / truncated-SVD compression, and
// the environment steps of the 4-layer strip (plaquette and vertical-hop
// ratios) and of the 3-layer row (gradient and horizontal-hop ratios).
//
// One CTA owns one Markov chain at a time; all tensors of that chain live in
// the CTA's slice of a global scratch arena (L2-resident for the active CTAs).
//
// Tensor layouts (row-major):
//   PEPS tensor at a vertex, "box" of D_k^4: W[l][r][d][u]; missing legs of
//     the open boundary use index 0 only (dimension 1).
//   boundary-MPS site: M[a][i][b] (left bond, physical, right bond); the
//     bond dimensions of every MPS come from host-computed tables bd[0..Lx]
//     with bd[0] = bd[Lx] = 1 and bd[c] = left bond of site c.
//   strip environment: E[a][i][j][b] (B bond, row-r bond, row-(r+1) bond,
//     T bond); row environment: E[a][l][b].
#pragma once

#include "common.cuh"
#include "linalg.cuh"

namespace gcf {

enum { MAX_L = 64 };

// Everything a VMC kernel needs; plain pointers into device memory.
template <class T>
struct KParams {
  // model
  int N, Lx, Ly, Dk, chi, matter, P;
  int n_h, n_v, n_s, cfg_len, n_plaq, n_slots;
  double h, g, J, m;
  const int* Q;            // [Ly*Lx]
  const long long* voff;   // [Lx*Ly] parameter offset of each vertex
  const int* vbs;          // [Lx*Ly] block size of each vertex
  const T* params;
  // MPS tables (see host planner): bond dims of stored MPS and per-step
  // QR dims / SVD flags, each row of Lx+1 ints.
  const int* bondB;  // slot j = B[j-1], j = 0..Ly-1
  const int* bondT;  // slot r = T[r], r = 1..Ly (index 0 unused)
  const int* qrB;    // B-step r (absorbing row r), r = 0..Ly-2
  const int* svdB;
  const int* qrT;    // T-step r, r = 1..Ly-1
  const int* svdT;
  // scratch
  T* scratch;
  long long ws_stride;     // elements per CTA
  long long o_net, o_prop, o_B, o_T, o_Q, o_M1, o_M2, o_M3, o_tau, o_J, o_envR, o_envL,
      o_envX, o_envY, o_t1, o_t2, o_t3, o_env3R, o_env3L, o_env3X, o_env3Y, o_G;
  long long mps_stride, qsite_stride;
  int env_stride, env3_stride;
  int max_sweeps_svd;
  // per-run
  int n_chains, n_sweeps, mode, want;  // mode 0: measure given configs, 1: sample
  unsigned long long seed;
  int8_t* configs;
  double* log_abs;
  double* phase;
  double* e_loc;
  int* block_ids;
  T* O;
  int* accepted;
  int* proposed;
  int* status;       // [4] error flags (gauss, numeric, svd not converged)
};

enum { WANT_AMP = 1, WANT_ELOC = 2, WANT_GRAD = 4 };
enum { ST_GAUSS = 0, ST_NUMERIC = 1, ST_SVD = 2 };

struct Shared {
  double red[64];
  int iflag[4];
  int bd_off[MAX_L + 1];
  int bd_off2[MAX_L + 1];
  int sel[4 * MAX_L * 4];
  double sigma[4 * MAX_L * 4];
};

__device__ inline int hl_dim(int c, int Dk) { return c == 0 ? 1 : Dk; }
__device__ inline int hr_dim(int c, int Lx, int Dk) { return c == Lx - 1 ? 1 : Dk; }
__device__ inline int dn_dim(int r, int Dk) { return r == 0 ? 1 : Dk; }
__device__ inline int up_dim(int r, int Ly, int Dk) { return r == Ly - 1 ? 1 : Dk; }

// ---------------------------------------------------------------------------
// Configuration helpers (int8 layout documented in the public header)
// ---------------------------------------------------------------------------
template <class T>
__device__ inline void leg_values(const KParams<T>& k, const int8_t* cfg, int x, int y, int& nl,
                                  int& nr, int& nd, int& nu, int& p) {
  nl = x > 0 ? cfg[y * (k.Lx - 1) + x - 1] : 0;
  nr = x < k.Lx - 1 ? cfg[y * (k.Lx - 1) + x] : 0;
  nd = y > 0 ? cfg[k.n_h + (y - 1) * k.Lx + x] : 0;
  nu = y < k.Ly - 1 ? cfg[k.n_h + y * k.Lx + x] : 0;
  p = cfg[k.n_h + k.n_v + y * k.Lx + x];
}

// Block id selected at (x, y) by cfg, or -1 if the Gauss law (Eq. 1) fails.
template <class T>
__device__ inline int block_of(const KParams<T>& k, const int8_t* cfg, int x, int y) {
  int nl, nr, nd, nu, p;
  leg_values(k, cfg, x, y, nl, nr, nd, nu, p);
  if (p < 0 || p >= k.P) return -1;
  int tot = p + nl + nd - nr - nu - k.Q[y * k.Lx + x];
  tot %= k.N;
  if (tot != 0) return -1;
  const int n[4] = {nl, nr, nd, nu};
  const bool has[4] = {x > 0, x < k.Lx - 1, y > 0, y < k.Ly - 1};
  int last = 3;
  while (!has[last]) --last;
  int bid = p;
  for (int i = 0; i < last; ++i)
    if (has[i]) bid = bid * k.N + n[i];
  return bid;
}

// Copy the selected block of (x, y) into a D_k^4 box (thread-parallel).
template <class T>
__device__ inline void gather_box(const KParams<T>& k, int x, int y, int bid, T* box) {
  const int Dk = k.Dk;
  const int dl = hl_dim(x, Dk), dr = hr_dim(x, k.Lx, Dk), dd = dn_dim(y, Dk),
            du = up_dim(y, k.Ly, Dk);
  const int v = y * k.Lx + x;
  const T* src = k.params + k.voff[v] + (long long)bid * k.vbs[v];
  const int bs = dl * dr * dd * du;
  for (int e = threadIdx.x; e < bs; e += blockDim.x) {
    int t = e;
    const int iu = t % du; t /= du;
    const int id = t % dd; t /= dd;
    const int ir = t % dr; t /= dr;
    const int il = t;
    box[((il * Dk + ir) * Dk + id) * Dk + iu] = src[e];
  }
}

template <class T>
__device__ inline T* ws_of(const KParams<T>& k) {
  return k.scratch + (long long)blockIdx.x * k.ws_stride;
}

template <class T>
__device__ inline T* net_box(const KParams<T>& k, T* ws, int x, int y) {
  return ws + k.o_net + (long long)(y * k.Lx + x) * (k.Dk * k.Dk * k.Dk * k.Dk);
}

// site offsets of a packed MPS with bond table bd and physical dim phys
__device__ inline void mps_offsets(const int* bd, int phys, int Lx, int* off) {
  if (threadIdx.x == 0) {
    int o = 0;
    for (int c = 0; c < Lx; ++c) { off[c] = o; o += bd[c] * phys * bd[c + 1]; }
    off[Lx] = o;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// Rescaling: divide a tensor by its largest |component|, return log(scale).
// ---------------------------------------------------------------------------
template <class T>
__device__ __noinline__ double rescale(T* a, int n, double* red) {
  using R = typename Traits<T>::R;
  double mx = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) mx = fmax(mx, (double)absmax1(a[i]));
  mx = block_max(mx, red);
  if (!(mx > 0.0) || !isfinite(mx)) return 0.0;
  const R s = (R)(1.0 / mx);
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = scale(a[i], s);
  __syncthreads();
  return log(mx);
}

template <class T>
__device__ __noinline__ double frob_rescale(T* a, int n, double* red) {
  using R = typename Traits<T>::R;
  double s2 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s2 += (double)abs2(a[i]);
  s2 = block_sum(s2, red);
  if (!(s2 > 0.0) || !isfinite(s2)) return 0.0;
  const double nr = sqrt(s2);
  const R s = (R)(1.0 / nr);
  for (int i = threadIdx.x; i < n; i += blockDim.x) a[i] = scale(a[i], s);
  __syncthreads();
  return log(nr);
}

// ---------------------------------------------------------------------------
// Row absorption + compression.
//   in : MPS `mps_in` (bond table bdi, physical dim pin) and row `row` whose
//        tensors are boxes net_box(x=c, y=row); flip=1 swaps the d and u legs
//        (absorption from above).
//   out: MPS `mout` with bond table bdo, physical dim pout; qr/svd: the
//        step's QR left dims and SVD flags.  Returns log of the scale factor
//        (output state = exp(ret) * mout, up to the discarded weight).
// Algorithm: QR left to right on the absorbed MPS (left-canonical form),
// then right to left: LQ where no truncation is needed, one-sided Jacobi SVD
// keeping the chi largest singular values otherwise.
// ---------------------------------------------------------------------------
template <class T>
__device__ __noinline__ double absorb_compress(const KParams<T>& k, T* ws, Shared& sh, const T* mps_in,
                                  const int* bdi, int pin, int row, int flip, T* mout,
                                  const int* bdo, int pout, const int* qr, const int* svd) {
  const int Lx = k.Lx, Dk = k.Dk;
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  const int sd = flip ? 1 : Dk, su = flip ? Dk : 1;
  T* M1 = ws + k.o_M1;
  T* M2 = ws + k.o_M2;
  T* M3 = ws + k.o_M3;
  T* tau = ws + k.o_tau;
  T* Jm = ws + k.o_J;
  T* Qs = ws + k.o_Q;
  double logs = 0.0;
  mps_offsets(bdi, pin, Lx, sh.bd_off);
  mps_offsets(bdo, pout, Lx, sh.bd_off2);

  // R carry (rows qr[c], cols ab[c]); starts as [1]
  if (threadIdx.x == 0) M3[0] = one<T>();
  __syncthreads();
  int Rrows = 1, Rcols = 1;
  for (int c = 0; c < Lx; ++c) {
    const int a = bdi[c], b = bdi[c + 1];
    const int l = hl_dim(c, Dk), r = hr_dim(c, Lx, Dk);
    const int abl = a * l, abr = b * r;
    const T* M = mps_in + sh.bd_off[c];
    const T* W = net_box(k, ws, c, row);
    // Z[(a,l)][u][(b,r)] = sum_d M[a][d][b] W[l][r][d][u]   -> M2
    const int nZ = abl * pout * abr;
    for (int idx = threadIdx.x; idx < nZ; idx += blockDim.x) {
      int t = idx;
      const int ir = t % r; t /= r;
      const int ib = t % b; t /= b;
      const int iu = t % pout; t /= pout;
      const int il = t % l; t /= l;
      const int ia = t;
      T s = zero<T>();
      for (int d = 0; d < pin; ++d)
        s = fmac(s, M[(ia * pin + d) * b + ib], W[il * D3 + ir * D2 + d * sd + iu * su]);
      M2[idx] = s;
    }
    __syncthreads();
    // X = R (Rrows x abl) * Z (abl x pout*abr)  -> M1 (rows Rrows*pout, cols abr)
    cta_gemm<T>(Rrows, pout * abr, abl, M3, Rcols, 1, M2, pout * abr, 1, M1, pout * abr, 1, false);
    const int rows = Rrows * pout, cols = abr;
    if (c < Lx - 1) {
      cta_qr<T>(rows, cols, M1, cols, 1, tau, sh.red);
      const int kq = min(rows, cols);
      // Q -> Qs site c (rows x kq)
      T* Qc = Qs + (long long)c * k.qsite_stride;
      cta_form_q<T>(rows, kq, M1, cols, 1, tau, Qc, kq, 1);
      // R (kq x cols) -> M3
      for (int idx = threadIdx.x; idx < kq * cols; idx += blockDim.x) {
        const int i = idx / cols, j = idx - (idx / cols) * cols;
        M3[idx] = (j >= i) ? M1[i * cols + j] : zero<T>();
      }
      __syncthreads();
      logs += frob_rescale(M3, kq * cols, sh.red);
      Rrows = kq; Rcols = cols;
    } else {
      // last site: keep X (rows x 1) in M3 as the right-to-left carry start
      for (int idx = threadIdx.x; idx < rows; idx += blockDim.x) M3[idx] = M1[idx];
      __syncthreads();
      Rrows = rows; Rcols = 1;
    }
  }
  (void)qr;
  // Right to left.  Y = M3 viewed as (qr[c]) x (pout * fin[c+1]).
  for (int c = Lx - 1; c >= 1; --c) {
    const int yr = qr[c], yc = pout * bdo[c + 1];
    const int kk = bdo[c];
    T* site = mout + sh.bd_off2[c];
    // LQ: Y^H (yc x yr) -> M1, QR, L = R^H, Q = Q'^H
    cta_adjoint<T>(yc, yr, M3, yc, 1, M1, yr, 1);
    cta_qr<T>(yc, yr, M1, yr, 1, tau, sh.red);
    const int k0 = min(yr, yc);
    // Q' (yc x k0) -> M2
    cta_form_q<T>(yc, k0, M1, yr, 1, tau, M2, k0, 1);
    // L (yr x k0) = R'^H -> Jm region used as L buffer (M3 free now)
    for (int idx = threadIdx.x; idx < yr * k0; idx += blockDim.x) {
      const int i = idx / k0, j = idx - (idx / k0) * k0;
      M3[idx] = (i >= j) ? conjg(M1[j * yr + i]) : zero<T>();
    }
    __syncthreads();
    if (!svd[c]) {
      // site = Q'^H (k0 x yc); carry L (yr x k0)
      cta_adjoint<T>(k0, yc, M2, k0, 1, site, yc, 1);
    } else {
      // one-sided Jacobi on L (yr x k0): L J = W, keep the kk largest columns
      int conv = 1;
      cta_jacobi_svd<T>(yr, k0, M3, k0, 1, Jm, k0, 1, &sh.iflag[0], k.max_sweeps_svd, &conv);
      if (!conv && threadIdx.x == 0) atomicAdd(&k.status[ST_SVD], 1);
      for (int j = threadIdx.x; j < k0; j += blockDim.x) {
        double s2 = 0.0;
        for (int i = 0; i < yr; ++i) s2 += (double)abs2(M3[i * k0 + j]);
        sh.sigma[j] = s2;
      }
      __syncthreads();
      for (int j = threadIdx.x; j < k0; j += blockDim.x) {
        int rank = 0;
        const double sj = sh.sigma[j];
        for (int i = 0; i < k0; ++i) {
          const double si = sh.sigma[i];
          rank += (si > sj) || (si == sj && i < j);
        }
        if (rank < kk) sh.sel[rank] = j;
      }
      __syncthreads();
      // site[n][x] = sum_j conj(J[j][sel n]) Q'^H[j][x] = sum_j conj(J[j][sel]) conj(Q'[x][j])
      for (int idx = threadIdx.x; idx < kk * yc; idx += blockDim.x) {
        const int n = idx / yc, x = idx - (idx / yc) * yc;
        const int jn = sh.sel[n];
        T s = zero<T>();
        for (int j = 0; j < k0; ++j) s = fmac(s, conjg(Jm[j * k0 + jn]), conjg(M2[x * k0 + j]));
        site[idx] = s;
      }
      // carry U S = W[:, sel] (yr x kk) -> M1 then back to M3
      for (int idx = threadIdx.x; idx < yr * kk; idx += blockDim.x) {
        const int i = idx / kk, n = idx - (idx / kk) * kk;
        M1[idx] = M3[i * k0 + sh.sel[n]];
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < yr * kk; idx += blockDim.x) M3[idx] = M1[idx];
      __syncthreads();
    }
    logs += frob_rescale(M3, yr * kk, sh.red);
    // next Y = Q_{c-1} (qr[c-1]*pout x qr[c]) * carry (qr[c] x kk)
    const T* Qp = Qs + (long long)(c - 1) * k.qsite_stride;
    const int prow = qr[c - 1] * pout;
    cta_gemm<T>(prow, kk, yr, Qp, yr, 1, M3, kk, 1, M1, kk, 1, false);
    for (int idx = threadIdx.x; idx < prow * kk; idx += blockDim.x) M3[idx] = M1[idx];
    __syncthreads();
  }
  // site 0: Y (1 x pout*fin[1]) normalised
  {
    const int n0 = pout * bdo[1];
    logs += frob_rescale(M3, n0, sh.red);
    T* site = mout + sh.bd_off2[0];
    for (int idx = threadIdx.x; idx < n0; idx += blockDim.x) site[idx] = M3[idx];
    __syncthreads();
  }
  return logs;
}

// ---------------------------------------------------------------------------
// Strip (4-layer) environment steps.  Dims: E[a][i][j][b] = (nA, nI, nJ, nB).
// Column tensors: Bs (nA x pB x nA'), W1 box (row r), W2 box (row r+1),
// Ts (nB x pT x nB'); nI' = nJ' = hr, pM = vertical bond between the rows.
// ---------------------------------------------------------------------------
struct StripDims {
  int nA, nI, nJ, nB;     // left cut
  int nA2, nI2, nJ2, nB2; // right cut
  int pB, pM, pT;         // physical dims: B-phys (= d of row r), middle, T-phys
};

template <class T>
__device__ __noinline__ void strip_left_step(int Dk, const StripDims& d, const T* L, const T* Bs, const T* W1,
                                const T* W2, const T* Ts, T* out, T* t1, T* t2, T* t3) {
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  // S1: X1[i][j][b][dd][a2] = sum_a L[a][i][j][b] Bs[a][dd][a2]
  {
    const int n = d.nI * d.nJ * d.nB * d.pB * d.nA2;
    const int sLa = d.nI * d.nJ * d.nB, sBa = d.pB * d.nA2;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int a2 = t % d.nA2; t /= d.nA2;
      const int dd = t % d.pB; t /= d.pB;
      const int ijb = t;  // (i*nJ + j)*nB + b
      T s = zero<T>();
      const T* lp = L + ijb;
      const T* bp = Bs + dd * d.nA2 + a2;
      for (int a = 0; a < d.nA; ++a) s = fmac(s, lp[a * sLa], bp[a * sBa]);
      t1[idx] = s;
    }
    __syncthreads();
  }
  // S2: X2[j][b][a2][i2][m] = sum_{i,dd} X1[i][j][b][dd][a2] W1[i][i2][dd][m]
  {
    const int n = d.nJ * d.nB * d.nA2 * d.nI2 * d.pM;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int m = t % d.pM; t /= d.pM;
      const int i2 = t % d.nI2; t /= d.nI2;
      const int a2 = t % d.nA2; t /= d.nA2;
      const int b = t % d.nB; t /= d.nB;
      const int j = t;
      T s = zero<T>();
      for (int i = 0; i < d.nI; ++i)
        for (int dd = 0; dd < d.pB; ++dd)
          s = fmac(s, t1[(((i * d.nJ + j) * d.nB + b) * d.pB + dd) * d.nA2 + a2],
                   W1[i * D3 + i2 * D2 + dd * Dk + m]);
      t2[idx] = s;
    }
    __syncthreads();
  }
  // S3: X3[a2][i2][j2][b][u] = sum_{j,m} X2[j][b][a2][i2][m] W2[j][j2][m][u]
  {
    const int n = d.nA2 * d.nI2 * d.nJ2 * d.nB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int u = t % d.pT; t /= d.pT;
      const int b = t % d.nB; t /= d.nB;
      const int j2 = t % d.nJ2; t /= d.nJ2;
      const int i2 = t % d.nI2; t /= d.nI2;
      const int a2 = t;
      T s = zero<T>();
      for (int j = 0; j < d.nJ; ++j)
        for (int m = 0; m < d.pM; ++m)
          s = fmac(s, t2[(((j * d.nB + b) * d.nA2 + a2) * d.nI2 + i2) * d.pM + m],
                   W2[j * D3 + j2 * D2 + m * Dk + u]);
      t3[idx] = s;
    }
    __syncthreads();
  }
  // S4: out[a2][i2][j2][b2] = sum_{b,u} X3[a2][i2][j2][b][u] Ts[b][u][b2]
  {
    const int n = d.nA2 * d.nI2 * d.nJ2 * d.nB2;
    const int K = d.nB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int b2 = idx % d.nB2;
      const int aij = idx / d.nB2;
      T s = zero<T>();
      const T* xp = t3 + aij * K;
      for (int bu = 0; bu < K; ++bu) s = fmac(s, xp[bu], Ts[bu * d.nB2 + b2]);
      out[idx] = s;
    }
    __syncthreads();
  }
}

// R[a][i][j][b] = sum Bs[a][dd][a2] W1[i][i2][dd][m] W2[j][j2][m][u] Ts[b][u][b2] R2[a2][i2][j2][b2]
template <class T>
__device__ __noinline__ void strip_right_step(int Dk, const StripDims& d, const T* R2, const T* Bs, const T* W1,
                                 const T* W2, const T* Ts, T* out, T* t1, T* t2, T* t3) {
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  // S1: Y1[a2][i2][j2][b][u] = sum_b2 R2[a2][i2][j2][b2] Ts[b][u][b2]
  {
    const int n = d.nA2 * d.nI2 * d.nJ2 * d.nB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int bu = idx % (d.nB * d.pT);
      const int aij = idx / (d.nB * d.pT);
      T s = zero<T>();
      const T* rp = R2 + aij * d.nB2;
      const T* tp = Ts + bu * d.nB2;
      for (int b2 = 0; b2 < d.nB2; ++b2) s = fmac(s, rp[b2], tp[b2]);
      t1[idx] = s;
    }
    __syncthreads();
  }
  // S2: Y2[a2][i2][j][m][b] = sum_{j2,u} Y1[a2][i2][j2][b][u] W2[j][j2][m][u]
  {
    const int n = d.nA2 * d.nI2 * d.nJ * d.pM * d.nB;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int b = t % d.nB; t /= d.nB;
      const int m = t % d.pM; t /= d.pM;
      const int j = t % d.nJ; t /= d.nJ;
      const int i2 = t % d.nI2; t /= d.nI2;
      const int a2 = t;
      T s = zero<T>();
      for (int j2 = 0; j2 < d.nJ2; ++j2)
        for (int u = 0; u < d.pT; ++u)
          s = fmac(s, t1[(((a2 * d.nI2 + i2) * d.nJ2 + j2) * d.nB + b) * d.pT + u],
                   W2[j * D3 + j2 * D2 + m * Dk + u]);
      t2[idx] = s;
    }
    __syncthreads();
  }
  // S3: Y3[a2][i][j][dd][b] = sum_{i2,m} Y2[a2][i2][j][m][b] W1[i][i2][dd][m]
  {
    const int n = d.nA2 * d.nI * d.nJ * d.pB * d.nB;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int b = t % d.nB; t /= d.nB;
      const int dd = t % d.pB; t /= d.pB;
      const int j = t % d.nJ; t /= d.nJ;
      const int i = t % d.nI; t /= d.nI;
      const int a2 = t;
      T s = zero<T>();
      for (int i2 = 0; i2 < d.nI2; ++i2)
        for (int m = 0; m < d.pM; ++m)
          s = fmac(s, t2[(((a2 * d.nI2 + i2) * d.nJ + j) * d.pM + m) * d.nB + b],
                   W1[i * D3 + i2 * D2 + dd * Dk + m]);
      t3[idx] = s;
    }
    __syncthreads();
  }
  // S4: R[a][i][j][b] = sum_{a2,dd} Bs[a][dd][a2] Y3[a2][i][j][dd][b]
  {
    const int n = d.nA * d.nI * d.nJ * d.nB;
    const int sY = d.nI * d.nJ * d.pB * d.nB;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int b = t % d.nB; t /= d.nB;
      const int j = t % d.nJ; t /= d.nJ;
      const int i = t % d.nI; t /= d.nI;
      const int a = t;
      T s = zero<T>();
      for (int a2 = 0; a2 < d.nA2; ++a2)
        for (int dd = 0; dd < d.pB; ++dd)
          s = fmac(s, Bs[(a * d.pB + dd) * d.nA2 + a2],
                   t3[a2 * sY + ((i * d.nJ + j) * d.pB + dd) * d.nB + b]);
      out[idx] = s;
    }
    __syncthreads();
  }
}

// sum_k A[k] B[k] (no conjugation), broadcast; returns (re, im) in doubles
template <class T>
__device__ inline void cta_dot(const T* A, const T* B, int n, double* red, double& r, double& i) {
  T s = zero<T>();
  for (int k = threadIdx.x; k < n; k += blockDim.x) s = fmac(s, A[k], B[k]);
  r = (double)re(s);
  i = (double)im(s);
  block_sum2(r, i, red);
}

// ---------------------------------------------------------------------------
// Row (3-layer) environment steps.  E[a][l][b] = (nA, nH, nB).
// ---------------------------------------------------------------------------
struct RowDims {
  int nA, nH, nB;     // left cut
  int nA2, nH2, nB2;  // right cut
  int pB, pT;
};

template <class T>
__device__ __noinline__ void row_left_step(int Dk, const RowDims& d, const T* L, const T* Bs, const T* W,
                              const T* Ts, T* out, T* t1, T* t2) {
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  // S1: X1[l][b][dd][a2] = sum_a L[a][l][b] Bs[a][dd][a2]
  {
    const int n = d.nH * d.nB * d.pB * d.nA2;
    const int sLa = d.nH * d.nB, sBa = d.pB * d.nA2;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int da = idx % (d.pB * d.nA2);
      const int lb = idx / (d.pB * d.nA2);
      T s = zero<T>();
      for (int a = 0; a < d.nA; ++a) s = fmac(s, L[a * sLa + lb], Bs[a * sBa + da]);
      t1[idx] = s;
    }
    __syncthreads();
  }
  // S2: X2[b][a2][r][u] = sum_{l,dd} X1[l][b][dd][a2] W[l][r][dd][u]
  {
    const int n = d.nB * d.nA2 * d.nH2 * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int u = t % d.pT; t /= d.pT;
      const int r = t % d.nH2; t /= d.nH2;
      const int a2 = t % d.nA2; t /= d.nA2;
      const int b = t;
      T s = zero<T>();
      for (int l = 0; l < d.nH; ++l)
        for (int dd = 0; dd < d.pB; ++dd)
          s = fmac(s, t1[((l * d.nB + b) * d.pB + dd) * d.nA2 + a2], W[l * D3 + r * D2 + dd * Dk + u]);
      t2[idx] = s;
    }
    __syncthreads();
  }
  // S3: out[a2][r][b2] = sum_{b,u} X2[b][a2][r][u] Ts[b][u][b2]
  {
    const int n = d.nA2 * d.nH2 * d.nB2;
    const int sXb = d.nA2 * d.nH2 * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int b2 = idx % d.nB2;
      const int ar = idx / d.nB2;
      T s = zero<T>();
      for (int b = 0; b < d.nB; ++b)
        for (int u = 0; u < d.pT; ++u)
          s = fmac(s, t2[b * sXb + ar * d.pT + u], Ts[(b * d.pT + u) * d.nB2 + b2]);
      out[idx] = s;
    }
    __syncthreads();
  }
}

template <class T>
__device__ __noinline__ void row_right_step(int Dk, const RowDims& d, const T* R2, const T* Bs, const T* W,
                               const T* Ts, T* out, T* t1, T* t2) {
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  // S1: Y1[a2][r][b][u] = sum_b2 R2[a2][r][b2] Ts[b][u][b2]
  {
    const int n = d.nA2 * d.nH2 * d.nB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int bu = idx % (d.nB * d.pT);
      const int ar = idx / (d.nB * d.pT);
      T s = zero<T>();
      for (int b2 = 0; b2 < d.nB2; ++b2) s = fmac(s, R2[ar * d.nB2 + b2], Ts[bu * d.nB2 + b2]);
      t1[idx] = s;
    }
    __syncthreads();
  }
  // S2: Y2[a2][l][dd][b] = sum_{r,u} Y1[a2][r][b][u] W[l][r][dd][u]
  {
    const int n = d.nA2 * d.nH * d.pB * d.nB;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int b = t % d.nB; t /= d.nB;
      const int dd = t % d.pB; t /= d.pB;
      const int l = t % d.nH; t /= d.nH;
      const int a2 = t;
      T s = zero<T>();
      for (int r = 0; r < d.nH2; ++r)
        for (int u = 0; u < d.pT; ++u)
          s = fmac(s, t1[((a2 * d.nH2 + r) * d.nB + b) * d.pT + u], W[l * D3 + r * D2 + dd * Dk + u]);
      t2[idx] = s;
    }
    __syncthreads();
  }
  // S3: out[a][l][b] = sum_{a2,dd} Bs[a][dd][a2] Y2[a2][l][dd][b]
  {
    const int n = d.nA * d.nH * d.nB;
    const int sY = d.nH * d.pB * d.nB;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int b = t % d.nB; t /= d.nB;
      const int l = t % d.nH; t /= d.nH;
      const int a = t;
      T s = zero<T>();
      for (int a2 = 0; a2 < d.nA2; ++a2)
        for (int dd = 0; dd < d.pB; ++dd)
          s = fmac(s, Bs[(a * d.pB + dd) * d.nA2 + a2], t2[a2 * sY + (l * d.pB + dd) * d.nB + b]);
      out[idx] = s;
    }
    __syncthreads();
  }
}

// G[l][r][dd][u] = sum L[a][l][b] Bs[a][dd][a2] Ts[b][u][b2] R2[a2][r][b2]
// (open tensor of one vertex of the row, written over actual dims)
template <class T>
__device__ __noinline__ void row_site_open(int Dk, const RowDims& d, const T* L, const T* Bs, const T* Ts,
                              const T* R2, T* G, T* t1, T* t2) {
  // X1[l][b][dd][a2] (left S1)
  {
    const int n = d.nH * d.nB * d.pB * d.nA2;
    const int sLa = d.nH * d.nB, sBa = d.pB * d.nA2;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int da = idx % (d.pB * d.nA2);
      const int lb = idx / (d.pB * d.nA2);
      T s = zero<T>();
      for (int a = 0; a < d.nA; ++a) s = fmac(s, L[a * sLa + lb], Bs[a * sBa + da]);
      t1[idx] = s;
    }
  }
  // Y1[a2][r][b][u] (right S1)
  {
    const int n = d.nA2 * d.nH2 * d.nB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      const int bu = idx % (d.nB * d.pT);
      const int ar = idx / (d.nB * d.pT);
      T s = zero<T>();
      for (int b2 = 0; b2 < d.nB2; ++b2) s = fmac(s, R2[ar * d.nB2 + b2], Ts[bu * d.nB2 + b2]);
      t2[idx] = s;
    }
  }
  __syncthreads();
  {
    const int n = d.nH * d.nH2 * d.pB * d.pT;
    for (int idx = threadIdx.x; idx < n; idx += blockDim.x) {
      int t = idx;
      const int u = t % d.pT; t /= d.pT;
      const int dd = t % d.pB; t /= d.pB;
      const int r = t % d.nH2; t /= d.nH2;
      const int l = t;
      T s = zero<T>();
      for (int b = 0; b < d.nB; ++b)
        for (int a2 = 0; a2 < d.nA2; ++a2)
          s = fmac(s, t1[((l * d.nB + b) * d.pB + dd) * d.nA2 + a2],
                   t2[((a2 * d.nH2 + r) * d.nB + b) * d.pT + u]);
      G[idx] = s;
    }
    __syncthreads();
  }
  (void)Dk;
}

}  // namespace gcf
