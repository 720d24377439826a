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
#include "envsteps.cuh"

namespace gcf {

enum { MAX_L = 64 };

// Everything a VMC kernel needs; plain pointers into device memory.
template <class T>
struct KParams {
  // model
  int N, Lx, Ly, Dk, chi, matter, P;
  int n_h, n_v, n_s, cfg_len, n_plaq, n_slots;
  double h, g, J, m;
  double elink[8];         // g (2 - 2 cos(2 pi n / N)) for n = 0..N-1
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
  // all tables in one block: the six above, then the derived offB, offT
  // (site offsets per B / T slot, rows of Lx+1) and denseB, denseT (Ly+1
  // flags each: the step takes the identity + core form)
  const int* tab;
  int tab_ints;
  // scratch
  T* scratch;
  long long ws_stride;     // elements per CTA
  long long o_net, o_prop, o_B, o_T, o_Q, o_M1, o_M2, o_M3, o_tau, o_J, o_envR, o_envL,
      o_envX, o_envY, o_t1, o_t2, o_t3, o_env3R, o_env3L, o_env3X, o_env3Y, o_G;
  long long mps_stride, qsite_stride;
  // Boundary-MPS store.  ck_every = 0: every B[r] / T[r] of the chain is kept
  // (B slot j at o_B + j mps_stride, T slot r at o_T + r mps_stride).
  // ck_every = K >= 2: only every K-th is kept (B slot j with j % K == 0 at
  // o_B + (j / K) mps_stride; T slot r with (Ly - r) % K == 0 at
  // o_T + ((Ly - r) / K) mps_stride) and the slots of one segment between
  // two kept ones live in a segment buffer (o_Bseg / o_Tseg + position
  // mps_stride), recomputed from the segment's kept slot when a pass needs
  // them.
  int ck_every;
  long long o_Bseg, o_Tseg;
  int env_stride, env3_stride;
  int max_sweeps_svd;
  // hot buffers: in dynamic shared memory when hot_in_smem, else in scratch
  int hot_in_smem;
  long long o_sigma, o_sel, dense_max, o_Z, z_size, q_pack, o_X, o_W1, o_W2, o_W3, o_W4;
  long long so_net, so_prop, so_cop, so_envL, so_envX, so_envY, so_env3L, so_env3X, so_env3Y,
      so_t1, so_t2, smem_cfg_bytes;
  long long group_smem_bytes;  // grouped kernel: shared bytes per chain group
  int group_threads;          // grouped kernel: threads per chain (128)
  int lockstep;               // grouped kernels: keep a CTA's chains at the same row
  int lock_fault;             // test hook: group 0 never counts in, so the others' waits run out
  int gemm_mode;              // GemmMode of the contraction GEMMs
  int row_gemm_mode;          // GemmMode of the row environments (O, amplitude, hops)
  int absorb_gemm_mode;       // GemmMode of the boundary-MPS absorption (B[r], T[r])
  // BF16 GEMMs of real chains on the fifth-generation tensor cores
  // (tcgen05.cuh): 1 if used, the bytes of a chain's operand staging area and
  // its byte offset from the start of the chain's dynamic shared memory
  int tc_bf16;
  long long tc_bytes, tc_off;
  // shared-memory factorisation workspace of a chain (linalg.cuh): scalars
  // (0: none) and byte offset from the start of the chain's dynamic shared
  // memory
  long long fz_elems, fz_off;
  // right environments and the staged B / T rows of the current pass
  int mps_in_smem, renv_in_smem;
  long long so_envR, so_env3R, so_sB, so_sT;
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
  int* status;       // [4] counters: Gauss violations, tensor-core waits run out, SVDs not converged, lockstep waits run out
};

enum { WANT_AMP = 1, WANT_ELOC = 2, WANT_GRAD = 4 };
enum { ST_GAUSS = 0, ST_TC_TIMEOUT = 1, ST_SVD = 2, ST_PHASE_TIMEOUT = 3 };

struct Shared {
  double red[64];
  double bcast;
  int iflag[4];
  int ab[MAX_L + 1];
  int zoff[MAX_L + 1];
  int qoff[MAX_L + 1];
  int bd_off[MAX_L + 1];
  int bd_off2[MAX_L + 1];
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
template <class T, class X>
__device__ inline void gather_box(const X ex, const KParams<T>& k, int x, int y, int bid, T* box) {
  const int Dk = k.Dk;
  const int dl = hl_dim(x, Dk), dr = hr_dim(x, k.Lx, Dk), dd = dn_dim(y, Dk),
            du = up_dim(y, k.Ly, Dk);
  const int v = y * k.Lx + x;
  const T* src = k.params + k.voff[v] + (long long)bid * k.vbs[v];
  const int bs = dl * dr * dd * du;
#pragma unroll 1
  for (int e = ex.tid(); e < bs; e += ex.size()) {
    int t = e;
    const int iu = t % du; t /= du;
    const int id = t % dd; t /= dd;
    const int ir = t % dr; t /= dr;
    const int il = t;
    box[((il * Dk + ir) * Dk + id) * Dk + iu] = src[e];
  }
}

// Address of B slot j (B[j-1]) and of T slot r (T[r]) in a chain's scratch.
template <class T>
__device__ inline T* bslot_ptr(const KParams<T>& k, T* ws, int j) {
  const int K = k.ck_every;
  if (!K) return ws + k.o_B + (long long)j * k.mps_stride;
  if (j % K == 0) return ws + k.o_B + (long long)(j / K) * k.mps_stride;
  return ws + k.o_Bseg + (long long)(j % K) * k.mps_stride;
}
template <class T>
__device__ inline T* tslot_ptr(const KParams<T>& k, T* ws, int r) {
  const int K = k.ck_every;
  if (!K) return ws + k.o_T + (long long)r * k.mps_stride;
  const int d = k.Ly - r;
  if (d % K == 0) return ws + k.o_T + (long long)(d / K) * k.mps_stride;
  return ws + k.o_Tseg + (long long)(d % K) * k.mps_stride;
}

template <class T>
__device__ inline T* net_box(const KParams<T>& k, T* ws, int x, int y) {
  return ws + k.o_net + (long long)(y * k.Lx + x) * (k.Dk * k.Dk * k.Dk * k.Dk);
}

// ---------------------------------------------------------------------------
// Rescaling by exact powers of two; the returned integer e means
// "tensor_in = 2^e * tensor_out".
// ---------------------------------------------------------------------------
template <class T, class X>
__device__ __noinline__ int rescale(const X ex, T* a, int n) {
  using R = typename Traits<T>::R;
  float mx = 0.f;
#pragma unroll 1
  for (int i = ex.tid(); i < n; i += ex.size()) mx = fmaxf(mx, (float)absmax1(a[i]));
  mx = ex.maxf(mx);
  if (!(mx > 0.f) || !isfinite(mx)) return 0;
  const int e = exp2_of(mx);
  const R s = pow2r<R>(-e);
#pragma unroll 1
  for (int i = ex.tid(); i < n; i += ex.size()) a[i] = scale(a[i], s);
  ex.sync();
  return e;
}

// the same with the scale chosen from the Frobenius norm (|a| -> [0.5, 1))
template <class T, class X>
__device__ __noinline__ int frob_rescale(const X ex, T* a, int n) {
  using R = typename Traits<T>::R;
  R s2 = R(0);
#pragma unroll 1
  for (int i = ex.tid(); i < n; i += ex.size()) s2 += abs2(a[i]);
  s2 = ex.template sum<R>(s2);
  if (!(s2 > R(0)) || !isfinite((float)s2)) return 0;
  const int e = exp2_of((float)sqrt(s2));
  const R s = pow2r<R>(-e);
#pragma unroll 1
  for (int i = ex.tid(); i < n; i += ex.size()) a[i] = scale(a[i], s);
  ex.sync();
  return e;
}

// sum_k A[k] B[k] (no conjugation), broadcast to all threads as (re, im)
template <class T, class X>
__device__ __noinline__ void cta_dot(const X ex, const T* A, const T* B, int n, typename Traits<T>::R& r,
                               typename Traits<T>::R& i) {
  using R = typename Traits<T>::R;
  T s = zero<T>();
#pragma unroll 1
  for (int k = ex.tid(); k < n; k += ex.size()) s = fmac(s, A[k], B[k]);
  r = re(s);
  i = im(s);
  ex.template sum2<R>(r, i);
}

// ---------------------------------------------------------------------------
// Exact compression in identity + core form.
// When every output bond of a step is at full rank, bd[c] = min(p^c, p^(L-c))
// (p = D_k, L = Lx; no truncation), the compressed boundary state is an
// exact MPS whose sites left of m = floor(L/2) are identity isometries
// M[a][i][a*p + i], whose sites right of m are identity isometries
// M[i*p^(L-1-c) + b][i][b], and whose site m holds the normalised dense state
// v[(u_0..u_{m-1})][u_m][(u_{m+1}..u_{L-1})].  It is the same state the QR /
// LQ sweep produces, in a different gauge.  The dense state is obtained by
// contracting the input MPS to a vector and applying the row MPO site by site.
// Returns the binary exponent e of the scale (state = 2^e * output).
// ---------------------------------------------------------------------------
template <class T, class X>
__device__ __noinline__ int dense_absorb(const X ex, const KParams<T>& k, Shared& sh, const T* net, const T* mps_in,
                                            const int* bdi, int pin, int row, int flip, T* mout,
                                            const int* bdo, int pout, T* bufA, T* bufB) {
  const int Lx = k.Lx, Dk = k.Dk;
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  const int sd = flip ? 1 : Dk, su = flip ? Dk : 1;
  // 1. input vector v[(i_0..i_{L-1})], i_0 most significant
  if (ex.tid() == 0) bufA[0] = one<T>();
  ex.sync();
  int rows = 1;
  for (int c = 0; c < Lx; ++c) {
    const T* M = mps_in + sh.bd_off[c];
    // bufB[(p, i)][b] = sum_a bufA[p][a] M[a][(i b)]
    cta_gemm<T>(ex, rows, pin * bdi[c + 1], bdi[c], bufA, bdi[c], 1, M, pin * bdi[c + 1], 1, bufB,
                pin * bdi[c + 1], 1, false);
    rows *= pin;
    T* t = bufA; bufA = bufB; bufB = t;
  }
  // 2. MPO sweep: t_c[h][U][u][Dr] = sum_{h', d} W_c[h'][h][d][u] t_{c-1}[h'][U][d][Dr]
  int NU = 1, ND = rows / pin;  // ND = pin^(L-1) before position 0
  for (int c = 0; c < Lx; ++c) {
    const int hl = hl_dim(c, Dk), hr = hr_dim(c, Lx, Dk);
    const T* W = net + (long long)(row * Lx + c) * (Dk * Dk * Dk * Dk);
    const int nout = hr * NU * pout * ND;
#pragma unroll 1
    for (int idx = ex.tid(); idx < nout; idx += ex.size()) {
      int t = idx;
      const int Dr = t % ND; t /= ND;
      const int u = t % pout; t /= pout;
      const int U = t % NU; t /= NU;
      const int h = t;
      T s = zero<T>();
      for (int hp = 0; hp < hl; ++hp)
        for (int d = 0; d < pin; ++d)
          s = fmac(s, W[hp * D3 + h * D2 + d * sd + u * su], bufA[((hp * NU + U) * pin + d) * ND + Dr]);
      bufB[idx] = s;
    }
    ex.sync();
    T* tt = bufA; bufA = bufB; bufB = tt;
    NU *= pout;
    if (c < Lx - 1) ND /= pin;
  }
  // 3. scale v' (length pout^L, bufA) by a power of two near its norm
  using R = typename Traits<T>::R;
  const int nv = NU;
  R s2 = R(0);
#pragma unroll 1
  for (int i = ex.tid(); i < nv; i += ex.size()) s2 += abs2(bufA[i]);
  s2 = ex.template sum<R>(s2);
  const int e = (s2 > R(0) && isfinite((float)s2)) ? exp2_of((float)sqrt(s2)) : 0;
  const R inv = pow2r<R>(-e);
  // 4. identity sites and the core
  const int m = Lx / 2;
  for (int c = 0; c < Lx; ++c) {
    const int a = bdo[c], b = bdo[c + 1];
    T* site = mout + sh.bd_off2[c];
    const int n = a * pout * b;
    if (c == m) {
#pragma unroll 1
      for (int i = ex.tid(); i < n; i += ex.size()) site[i] = scale(bufA[i], inv);
    } else {
#pragma unroll 1
      for (int i = ex.tid(); i < n; i += ex.size()) {
        const int ib = i % b, ii = (i / b) % pout, ia = i / (b * pout);
        const bool on = (c < m) ? (ib == ia * pout + ii) : (ia == ii * b + ib);
        site[i] = on ? one<T>() : zero<T>();
      }
    }
  }
  ex.sync();
  return e;
}

// sel[0..kk) <- the indices of the kk largest of sigma[0..k0), largest first
// (ties: lower index first).
template <class R, class X>
__device__ inline void select_largest(const X ex, int k0, int kk, const R* sigma, int* sel) {
#pragma unroll 1
  for (int j = ex.tid(); j < k0; j += ex.size()) {
    int rank = 0;
    const R sj = sigma[j];
    for (int i = 0; i < k0; ++i) {
      const R si = sigma[i];
      rank += (si > sj) || (si == sj && i < j);
    }
    if (rank < kk) sel[rank] = j;
  }
  ex.sync();
}

// Truncated SVD step of a bond in FP32, in the chain's shared-memory
// workspace: L (yr x k0, row-major) = W J^T by one-sided Jacobi
// (jacobi_svd_cm), the kk columns of W with the largest norms kept, one
// Newton-Schulz step on the kept columns of J only,
//   Jn = J_s (3 I - J_s^T J_s) / 2,
// then carry = L Jn (yr x kk, row-major) and site = Jn^T Q'^T (kk x yc,
// row-major), Q' = Qp (yc x k0, row-major).  The squared column norms of W
// go to sigma.  Returns false, having done nothing, when the workspace is
// too small.
template <class X>
__device__ __noinline__ bool truncate_f32_smem(const X ex, int yr, int yc, int k0, int kk, const float* L,
                                               const float* Qp, float* carry, float* site, float* sigma, int* sel,
                                               int* sflag, int max_sweeps, int* conv) {
  float* fz = (float*)g_fz[ex.slot()];
  const int ldw = jac_ld(yr), ldj = jac_ld(k0);
  if (!fz || (long long)(ldw + ldj) * k0 + 2LL * ldj * kk + (long long)kk * kk > g_fz_elems) return false;
  float* w = fz;                // W, column-major (ldw)
  float* jj = w + ldw * k0;     // J, column-major (ldj)
  float* js = jj + ldj * k0;    // kept columns of J
  float* jn = js + ldj * kk;    // after the Newton-Schulz step
  float* gg = jn + ldj * kk;    // kk x kk, row-major
#pragma unroll 1
  for (int idx = ex.tid(); idx < k0 * ldw; idx += ex.size()) {
    const int c = idx / ldw, i = idx - (idx / ldw) * ldw;
    w[idx] = (i < yr) ? L[i * k0 + c] : 0.f;
  }
  ex.sync();
  jacobi_svd_cm(ex, yr, k0, w, ldw, jj, ldj, sflag, max_sweeps, conv);
#pragma unroll 1
  for (int j = ex.tid(); j < k0; j += ex.size()) {
    const float4* col = reinterpret_cast<const float4*>(w + j * ldw);
    float s2 = 0.f;
    for (int q = 0; q < (ldw >> 2); ++q) s2 = dot4(col[q], col[q], s2);
    sigma[j] = s2;
  }
  ex.sync();
  select_largest(ex, k0, kk, sigma, sel);
#pragma unroll 1
  for (int idx = ex.tid(); idx < kk * ldj; idx += ex.size()) {
    const int n = idx / ldj, i = idx - (idx / ldj) * ldj;
    js[idx] = jj[sel[n] * ldj + i];
  }
  ex.sync();
  // gg = J_s^T J_s, then (3 I - gg) / 2
  tile_gemm_f32(ex, kk, kk, k0, js, ldj, 1, js, 1, ldj, gg, kk, 1);
#pragma unroll 1
  for (int idx = ex.tid(); idx < kk * kk; idx += ex.size()) {
    const int i = idx / kk, j = idx - (idx / kk) * kk;
    gg[idx] = fmaf(-0.5f, gg[idx], i == j ? 1.5f : 0.f);
  }
  ex.sync();
  tile_gemm_f32(ex, k0, kk, kk, js, 1, ldj, gg, kk, 1, jn, 1, ldj);
  tile_gemm_f32(ex, yr, kk, k0, L, k0, 1, jn, 1, ldj, carry, kk, 1);
  tile_gemm_f32(ex, kk, yc, k0, jn, ldj, 1, Qp, 1, k0, site, yc, 1);
  return true;
}

// ---------------------------------------------------------------------------
// Row absorption + compression.
//   in : MPS `mps_in` (bond table bdi, physical dim pin) and row `row` whose
//        tensors are boxes net_box(x=c, y=row); flip=1 swaps the d and u legs
//        (absorption from above).
//   out: MPS `mout` with bond table bdo, physical dim pout; qr/svd: the
//        step's QR left dims and SVD flags.  Returns the binary exponent e of
//        the scale (output state = 2^e * mout, up to the discarded weight).
// Algorithm: QR left to right on the absorbed MPS (left-canonical form),
// then right to left: LQ where no truncation is needed, one-sided Jacobi SVD
// keeping the chi largest singular values otherwise.
// ---------------------------------------------------------------------------
template <class T, class X>
__device__ __noinline__ int absorb_compress(const X ex, const KParams<T>& k, T* ws, T* hot_base, Shared& sh, const T* net,
                                  const T* mps_in, const int* bdi, int pin, int row, int flip, T* mout,
                                  const int* bdo, int pout, const int* qr, const int* svd, const int* offi,
                                  const int* offo, int dense) {
  const int Lx = k.Lx, Dk = k.Dk;
  const int D3 = Dk * Dk * Dk, D2 = Dk * Dk;
  const int sd = flip ? 1 : Dk, su = flip ? Dk : 1;
  T* M1 = ws + k.o_M1;
  T* M2 = ws + k.o_M2;
  T* M3 = ws + k.o_M3;
  T* tau = ws + k.o_tau;
  T* Jm = ws + k.o_J;
  T* Qs = ws + k.o_Q;
  int logs = 0;
#pragma unroll 1
  for (int c = ex.tid(); c <= Lx; c += ex.size()) {
    sh.bd_off[c] = offi[c];
    sh.bd_off2[c] = offo[c];
  }
  ex.sync();
  // Dense (identity + core) path: every output bond at full rank and the
  // dense state small enough (flag planned on the host).
  if (dense) {
    T* bufA = k.hot_in_smem ? hot_base + k.so_t1 : ws + k.o_t1;
    T* bufB = k.hot_in_smem ? hot_base + k.so_t2 : ws + k.o_t2;
    return dense_absorb<T>(ex, k, sh, net, mps_in, bdi, pin, row, flip, mout, bdo, pout, bufA, bufB);
  }

  // General path.  Z_c (absorbed sites) for all c; then a QR sweep from the
  // left over the bonds that must shrink (all bonds if the step truncates),
  // then an LQ / truncated-SVD sweep from the right over the bonds that must
  // shrink; sites in between are the absorbed tensors with the carries
  // multiplied in.  Without truncation this reaches the exact state with the
  // step's bond dimensions; with truncation it is the full canonical sweep.
  if (ex.tid() == 0) {
    int any_svd = 0;
    for (int c = 1; c < Lx; ++c) any_svd |= svd[c];
    int zo = 0, qo = 0;
    for (int c = 0; c <= Lx; ++c) sh.ab[c] = (c == 0 || c == Lx) ? 1 : bdi[c] * Dk;
    for (int c = 0; c < Lx; ++c) {
      sh.zoff[c] = zo;
      zo += sh.ab[c] * pout * sh.ab[c + 1];
      sh.qoff[c] = qo;
      qo += qr[c] * pout * qr[c + 1];
    }
    int cl = 0;
    while (cl < Lx - 1 && (any_svd || qr[cl] * pout < sh.ab[cl + 1])) ++cl;
    sh.iflag[1] = cl;
  }
  ex.sync();
  const int cL = sh.iflag[1];
  T* Z = ws + k.o_Z;
  T* Xb = ws + k.o_X;
  T* Y = ws + k.o_W1;
  T* Yh = ws + k.o_W2;
  T* Qp = ws + k.o_W3;
  T* Lc = ws + k.o_W4;
  for (int c = 0; c < Lx; ++c) {
    const int a = bdi[c], b = bdi[c + 1];
    const int l = hl_dim(c, Dk), r = hr_dim(c, Lx, Dk);
    const T* M = mps_in + sh.bd_off[c];
    const T* W = net + (long long)(row * Lx + c) * (Dk * Dk * Dk * Dk);
    const int nZ = a * l * pout * b * r;
    T* Zc = Z + sh.zoff[c];
#pragma unroll 1
    for (int idx = ex.tid(); idx < nZ; idx += ex.size()) {
      int t = idx;
      const int ir = t % r; t /= r;
      const int ib = t % b; t /= b;
      const int iu = t % pout; t /= pout;
      const int il = t % l; t /= l;
      const int ia = t;
      T s = zero<T>();
      for (int d = 0; d < pin; ++d)
        s = fmac(s, M[(ia * pin + d) * b + ib], W[il * D3 + ir * D2 + d * sd + iu * su]);
      Zc[idx] = s;
    }
  }
  // ---- left QR sweep over sites 0..cL-1; R carry in M3 (Rrows x ab[c])
  if (ex.tid() == 0) M3[0] = one<T>();
  ex.sync();
  int Rrows = 1;
  for (int c = 0; c <= cL; ++c) {
    const int abl = sh.ab[c], abr = sh.ab[c + 1];
    const int rows = Rrows * pout, cols = abr;
    // X = R (Rrows x abl) * Z_c (abl x pout*abr) -> (Rrows*pout) x abr
    T* X = (c == cL) ? Xb : M1;
    cta_gemm<T>(ex, Rrows, pout * abr, abl, M3, abl, 1, Z + sh.zoff[c], pout * abr, 1, X, pout * abr, 1, false);
    if (c == cL) break;
    const int kq = min(rows, cols);
    qr_with_q<T>(ex, rows, cols, M1, cols, tau, kq, Qs + sh.qoff[c], kq);
#pragma unroll 1
    for (int idx = ex.tid(); idx < kq * cols; idx += ex.size()) {
      const int i = idx / cols, j = idx - (idx / cols) * cols;
      M3[idx] = (j >= i) ? M1[i * cols + j] : zero<T>();
    }
    ex.sync();
    logs += frob_rescale(ex, M3, kq * cols);
    Rrows = kq;
  }
  // ---- right sweep over every site.  The carry Lc (rdim x kc) is the
  // identity while no bond to the right has been reduced.
  bool ident = true;
  int kc = 1, rdim = 1;
  for (int c = Lx - 1; c >= 0; --c) {
    const int cur = (c < cL) ? qr[c] : (c == cL ? Rrows : sh.ab[c]);
    const int rd = (c < cL) ? qr[c + 1] : sh.ab[c + 1];
    const T* S = (c < cL) ? Qs + sh.qoff[c] : (c == cL ? Xb : Z + sh.zoff[c]);
    const T* Yp;
    int yc;
    if (ident) {
      Yp = S;
      yc = pout * rd;
    } else {
      // Y = S ((cur*pout) x rdim) * Lc (rdim x kc), viewed cur x (pout*kc)
      cta_gemm<T>(ex, cur * pout, kc, rdim, S, rdim, 1, Lc, kc, 1, Y, kc, 1, false);
      Yp = Y;
      yc = pout * kc;
    }
    const int yr = cur;
    T* site = mout + sh.bd_off2[c];
    if (c >= 1 && (svd[c] || bdo[c] < cur)) {
      const int kk = bdo[c];
      cta_adjoint<T>(ex, yc, yr, Yp, yc, 1, Yh, yr, 1);
      const int k0 = min(yr, yc);
      qr_with_q<T>(ex, yc, yr, Yh, yr, tau, k0, Qp, k0);
      // L = R'^H (yr x k0)
#pragma unroll 1
      for (int idx = ex.tid(); idx < yr * k0; idx += ex.size()) {
        const int i = idx / k0, j = idx - (idx / k0) * k0;
        Lc[idx] = (i >= j) ? conjg(Yh[j * yr + i]) : zero<T>();
      }
      ex.sync();
      if (!svd[c]) {
        cta_adjoint<T>(ex, k0, yc, Qp, k0, 1, site, yc, 1);
      } else {
        // L J = W with orthogonal columns W (one-sided Jacobi).  J is a
        // product of many rotations, and in FP32 it drifts from orthogonal by
        // ~1e-5, which enters the kept subspace at every cut; one
        // Newton-Schulz step J <- J (3 I - J^H J) / 2 restores orthogonality
        // to rounding, and the kept W = L J is recomputed so that both
        // factors agree.
        using RR = typename Traits<T>::R;
        RR* sigma = (RR*)(ws + k.o_sigma);
        int* sel = (int*)(ws + k.o_sel);
        int conv = 1;
        bool done = false;
        if constexpr (std::is_same<T, float>::value)
          done = truncate_f32_smem(ex, yr, yc, k0, kk, Lc, Qp, Yh, site, sigma, sel, &sh.iflag[0],
                                   k.max_sweeps_svd, &conv);
        if (!done) {
          T* L0 = ws + k.o_M2;
          T* Gm = ws + k.o_M1;
          T* Jn = ws + k.o_M3;
#pragma unroll 1
          for (int idx = ex.tid(); idx < yr * k0; idx += ex.size()) L0[idx] = Lc[idx];
          ex.sync();
          T* fz = (T*)g_fz[ex.slot()];
          if (fz && (long long)yr * k0 + (long long)k0 * k0 <= g_fz_elems) {
            // sweeps on shared-memory copies; only J is needed afterwards
            // (W is recomputed as L J below)
            T* w = fz;
            T* jj = fz + yr * k0;
            cta_copy(ex, yr, k0, Lc, k0, w, k0);
            cta_jacobi_svd<T>(ex, yr, k0, w, k0, 1, jj, k0, 1, &sh.iflag[0], k.max_sweeps_svd, &conv);
            cta_copy(ex, k0, k0, jj, k0, Jm, k0);
          } else {
            cta_jacobi_svd<T>(ex, yr, k0, Lc, k0, 1, Jm, k0, 1, &sh.iflag[0], k.max_sweeps_svd, &conv);
          }
          cta_gemm<T, true, false, false>(ex, k0, k0, k0, Jm, 1, k0, Jm, k0, 1, Gm, k0, 1, false);
#pragma unroll 1
          for (int idx = ex.tid(); idx < k0 * k0; idx += ex.size()) {
            const int i = idx / k0, j = idx - (idx / k0) * k0;
            Gm[idx] = scale(Gm[idx], RR(-0.5));
            if (i == j) Gm[idx] += make_scalar<T>(RR(1.5), RR(0));
          }
          ex.sync();
          cta_gemm<T, false, false, false>(ex, k0, k0, k0, Jm, k0, 1, Gm, k0, 1, Jn, k0, 1, false);
          cta_gemm<T, false, false, false>(ex, yr, k0, k0, L0, k0, 1, Jn, k0, 1, Lc, k0, 1, false);
          // squared column norms -> sigma, selected columns -> sel (scratch)
#pragma unroll 1
          for (int j = ex.tid(); j < k0; j += ex.size()) {
            RR s2 = RR(0);
            for (int i = 0; i < yr; ++i) s2 += abs2(Lc[i * k0 + j]);
            sigma[j] = s2;
          }
          ex.sync();
          select_largest(ex, k0, kk, sigma, sel);
          // site[n][x] = sum_j conj(J[j][sel n]) Q'^H[j][x]
#pragma unroll 1
          for (int idx = ex.tid(); idx < kk * yc; idx += ex.size()) {
            const int n = idx / yc, x = idx - (idx / yc) * yc;
            const int jn = sel[n];
            T s = zero<T>();
            for (int j = 0; j < k0; ++j) s = fmac(s, conjg(Jn[j * k0 + jn]), conjg(Qp[x * k0 + j]));
            site[idx] = s;
          }
          // carry U S = W[:, sel] (yr x kk)
#pragma unroll 1
          for (int idx = ex.tid(); idx < yr * kk; idx += ex.size()) {
            const int i = idx / kk, n = idx - (idx / kk) * kk;
            Yh[idx] = Lc[i * k0 + sel[n]];
          }
          ex.sync();
        }
        if (!conv && ex.tid() == 0) atomicAdd(&k.status[ST_SVD], 1);
#pragma unroll 1
        for (int idx = ex.tid(); idx < yr * kk; idx += ex.size()) Lc[idx] = Yh[idx];
        ex.sync();
      }
      logs += frob_rescale(ex, Lc, yr * kk);
      kc = kk;
      rdim = yr;
      ident = false;
    } else {
      // no reduction at this site's left bond (cur == bdo[c]): keep Y
#pragma unroll 1
      for (int idx = ex.tid(); idx < yr * yc; idx += ex.size()) site[idx] = Yp[idx];
      ex.sync();
      logs += rescale(ex, site, yr * yc);
      ident = true;
    }
  }
  return logs;
}

}  // namespace gcf
