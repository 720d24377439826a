// The persistent VMC kernel: one CTA per Markov chain at a time.
//
// mode 0 (measure): for each given configuration, absorb rows bottom-up into
//   B[r], then run the measurement pass.
// mode 1 (sample): for each chain, build T[r] top-down once, then per sweep
//   the plaquette pass (bottom-up, Metropolis, Sec. S-1/S-2), with matter the
//   horizontal-hop pass (top-down) and vertical-hop pass (bottom-up), then the
//   measurement pass, whose T[r] serve the next sweep.
// Measurement pass (top-down over rows r): 3-layer row environments of row r
//   give O (Eq. S3), horizontal-hop ratios and, for r = Ly-1, the amplitude;
//   the 4-layer strip (r, r+1) gives plaquette and vertical-hop ratios for
//   E_loc (Eq. S2); then T[r] = absorb(T[r+1], row r).
#pragma once

#include "peps_dev.cuh"

namespace gcf {

struct SharedV;
__host__ __device__ constexpr unsigned long sizeof_sharedv_aligned();
struct SharedV {
  Shared base;
  int offB[MAX_L + 1];
  int offT[MAX_L + 1];
  int logB[MAX_L + 2];   // binary exponents of the stored MPS scales
  int logT[MAX_L + 2];
  int logR[MAX_L + 2];   // of the right environments of the current pass
  double eacc[2];
  int flag, ok, bad;
  int lock, phase;   // lockstep with the CTA's other chain groups; phases passed
  int segB, segT;    // segment of B / T slots the segment buffers hold (-1: none)
  float redf[32];
  int n_acc, n_prop;
  long long next;    // multi-context launches: the chain this group takes next
};

// Lockstep of the chain groups of one CTA: before each row of a pass every
// group's leader counts in on g_phase_arrive and waits (bounded) until all
// locked groups have; the groups then work on the same rows at the same time,
// so the SM fetches one region of code instead of one per chain.  No data is
// exchanged: the rendezvous only aligns timing.  g_lock_ok[g]: group g has a
// physical chain this round.
__shared__ int g_phase_arrive;
__shared__ int g_lock_ok[4];
constexpr int kPhaseSpinLimit = 1 << 22;

__host__ __device__ constexpr unsigned long sizeof_sharedv_aligned() {
  return (sizeof(SharedV) + 15) / 16 * 16;
}

template <class T, class X>
struct Chain {
  using R = typename Traits<T>::R;
  X ex;
  const KParams<T>& k;
  T* ws;
  SharedV& sv;
  int8_t* cfg;  // shared copy of the configuration
  int chain;
  unsigned long long key;
  // hot buffers (shared memory when they fit, else scratch)
  T *net, *props, *cop, *envL, *envX, *envY, *env3L, *env3X, *env3Y, *t1, *t2;
  T* hot;
  T *eR, *e3R, *sB, *sT;  // right environments; staged MPS rows (or the slots)
  const int* tab;         // the context's tables (shared-memory copy when it fits)

  __device__ Chain(const X ex_, const KParams<T>& kk, T* w, SharedV& s, int8_t* c, int ch, T* hot_, const int* tab_)
      : ex(ex_), k(kk), ws(w), sv(s), cfg(c), chain(ch), hot(hot_), tab(tab_) {
    key = stream_key(k.seed, (unsigned long long)ch);
    if (k.hot_in_smem) {
      net = hot_ + k.so_net; props = hot_ + k.so_prop; cop = hot_ + k.so_cop;
      envL = hot_ + k.so_envL; envX = hot_ + k.so_envX; envY = hot_ + k.so_envY;
      env3L = hot_ + k.so_env3L; env3X = hot_ + k.so_env3X; env3Y = hot_ + k.so_env3Y;
      t1 = hot_ + k.so_t1; t2 = hot_ + k.so_t2;
    }
    if (k.hot_in_smem && k.mps_in_smem) {
      sB = hot_ + k.so_sB; sT = hot_ + k.so_sT;
    } else {
      sB = nullptr; sT = nullptr;
    }
    if (k.hot_in_smem && k.mps_in_smem && k.renv_in_smem) {
      eR = hot_ + k.so_envR; e3R = hot_ + k.so_env3R;
    } else {
      eR = ws + k.o_envR; e3R = ws + k.o_env3R;
    }
    if (!k.hot_in_smem) {
      net = ws + k.o_net; props = ws + k.o_prop; cop = ws + k.o_t3;
      envL = ws + k.o_envL; envX = ws + k.o_envX; envY = ws + k.o_envY;
      env3L = ws + k.o_env3L; env3X = ws + k.o_env3X; env3Y = ws + k.o_env3Y;
      t1 = ws + k.o_t1; t2 = ws + k.o_t2;
    }
  }

  // rendezvous with the other locked groups of the CTA (no-op unless locked);
  // a wait that runs out of iterations drops this group out of lockstep and
  // records ST_PHASE_TIMEOUT
  __device__ void phase_sync() {
    if (!sv.lock) return;
    const int n_groups = blockDim.x / ex.size();
    ex.sync();
    if (ex.leader()) {
      sv.phase += 1;
      const int target = sv.phase * n_groups;
      if (!(k.lock_fault && ex.slot() == 0)) atomicAdd(&g_phase_arrive, 1);
      int it = 0;
      while (*(volatile int*)&g_phase_arrive < target && it < kPhaseSpinLimit) {
        __nanosleep(64);
        ++it;
      }
      if (it >= kPhaseSpinLimit) {
        sv.lock = 0;
        atomicAdd(&k.status[ST_PHASE_TIMEOUT], 1);
      }
    }
    ex.sync();
  }
  // arithmetic of this chain's contraction GEMMs from here on
  __device__ void set_gemm_mode(int m) {
    ex.sync();
    if (ex.leader()) g_gemm_mode[ex.slot()] = m;
    ex.sync();
  }

  __device__ T* Bslot(int j) const { return bslot_ptr(k, ws, j); }
  __device__ T* Tslot(int r) const { return tslot_ptr(k, ws, r); }

  // Checkpointed store: make B slot j (T slot r) readable.  A kept slot
  // always is; a slot of another segment than the buffer holds is rebuilt
  // by absorbing the rows above the segment's kept slot, with the network
  // as it stands (the rows a pass has not reached yet, so the same tensors
  // the slot was first built from).  Both run on every thread of the chain.
  __device__ void ensure_B(int j) {
    const int K = k.ck_every;
    if (!K || j % K == 0 || sv.segB == j / K) return;
    const int s0 = (j / K) * K;
    const int top = min(s0 + K - 1, k.Ly - 1);
    for (int r = s0; r < top; ++r) absorb_B(r);
  }
  __device__ void ensure_T(int r) {
    const int K = k.ck_every;
    if (!K || (k.Ly - r) % K == 0 || sv.segT == (k.Ly - r) / K) return;
    const int r0 = k.Ly - ((k.Ly - r) / K) * K;  // the segment's kept slot
    const int bottom = max(r0 - K + 1, 1);
    for (int rr = r0 - 1; rr >= bottom; --rr) absorb_T(rr);
  }
  __device__ int tW() const { return k.Lx + 1; }
  __device__ int tR() const { return k.Ly + 1; }
  __device__ const int* bdB(int j) const { return tab + j * tW(); }
  __device__ const int* bdT(int r) const { return tab + (tR() + r) * tW(); }
  __device__ const int* qrBt(int r) const { return tab + (2 * tR() + r) * tW(); }
  __device__ const int* svdBt(int r) const { return tab + (3 * tR() + r) * tW(); }
  __device__ const int* qrTt(int r) const { return tab + (4 * tR() + r) * tW(); }
  __device__ const int* svdTt(int r) const { return tab + (5 * tR() + r) * tW(); }
  __device__ const int* offBt(int j) const { return tab + (6 * tR() + j) * tW(); }
  __device__ const int* offTt(int r) const { return tab + (7 * tR() + r) * tW(); }
  __device__ int denseB(int r) const { return tab[8 * tR() * tW() + r]; }
  __device__ int denseT(int r) const { return tab[8 * tR() * tW() + tR() + r]; }
  // site offsets of the MPS rows of the current pass into shared memory
  __device__ void load_offsets(const int* src, int* dst) {
#pragma unroll 1
    for (int c = ex.tid(); c <= k.Lx; c += ex.size()) dst[c] = src[c];
    ex.sync();
  }
  __device__ int physB(int j) const { return j == 0 ? 1 : k.Dk; }   // B[j-1] phys = up dim of row j-1
  __device__ int physT(int r) const { return r == k.Ly ? 1 : k.Dk; } // T[r] phys = down dim of row r
  __device__ T* box(int x, int y) const {
    return net + (long long)(y * k.Lx + x) * (k.Dk * k.Dk * k.Dk * k.Dk);
  }
  __device__ T* prop(int i) const { return props + i * (k.Dk * k.Dk * k.Dk * k.Dk); }

  // ---- configuration moves on the shared copy (thread 0 writes) ---------
  __device__ __noinline__ void plaq_apply(int x, int y, int t) {
    if (ex.tid() == 0) {
      // link values and t are in [0, N): one conditional add / subtract
      // replaces the modulo
      const int N = k.N;
      int8_t* h = cfg;
      int8_t* v = cfg + k.n_h;
      auto up = [N, t](int8_t& a) { const int s = a + t; a = (int8_t)(s >= N ? s - N : s); };
      auto dn = [N, t](int8_t& a) { const int s = a - t; a = (int8_t)(s < 0 ? s + N : s); };
      up(h[y * (k.Lx - 1) + x]);
      up(v[y * k.Lx + x + 1]);
      dn(h[(y + 1) * (k.Lx - 1) + x]);
      dn(v[y * k.Lx + x]);
    }
    ex.sync();
  }
  // Hop across link (x,a): returns 1 if a move exists (and applies it).
  // On a hard-core lattice the hop available after a hop is its inverse, so
  // calling this again reverts the move.
  __device__ __noinline__ int hop_apply(int x, int y, int a) {
    int& ok = sv.ok;
    if (ex.tid() == 0) {
      const int N = k.N;
      const int x2 = a == 1 ? x + 1 : x, y2 = a == 1 ? y : y + 1;
      int8_t* p = cfg + k.n_h + k.n_v;
      int8_t* lk = a == 1 ? &cfg[y * (k.Lx - 1) + x] : &cfg[k.n_h + y * k.Lx + x];
      const int s1 = y * k.Lx + x, s2 = y2 * k.Lx + x2;
      ok = 0;
      // forward: boson from x+e to x raises the link; conjugate lowers it
      int dir = 0;
      if (p[s1] == 0 && p[s2] == 1) dir = +1;
      else if (p[s1] == 1 && p[s2] == 0) dir = -1;
      if (dir != 0) {
        p[s1] = (int8_t)(1 - p[s1]);
        p[s2] = (int8_t)(1 - p[s2]);
        *lk = (int8_t)(((int)*lk + dir + N) % N);
        ok = 1;
      }
    }
    ex.sync();
    const int r = ok;
    ex.sync();
    return r;
  }

  __device__ __noinline__ void gather_into(int x, int y, T* dst) {
    const int bid = block_of(k, cfg, x, y);
    if (bid < 0) {
      if (ex.tid() == 0) atomicAdd(&k.status[ST_GAUSS], 1);
      return;
    }
    gather_box(ex, k, x, y, bid, dst);
  }

  // gather the selected blocks of n vertices (x[i], y[i]) into dst[i] in
  // parallel (thread groups per vertex); caller synchronises
  __device__ __noinline__ void gather_n(int n, const int* xs, const int* ys, T* const* dst) {
    const int D4 = k.Dk * k.Dk * k.Dk * k.Dk;
    const int per = ex.size() / n;
    const int g = ex.tid() / per, tl = ex.tid() - g * per;
    if (g < n) {
      const int x = xs[g], y = ys[g];
      const int bid = block_of(k, cfg, x, y);
      if (bid < 0) {
        if (tl == 0) atomicAdd(&k.status[ST_GAUSS], 1);
      } else {
        const int Dk = k.Dk;
        const int dl = hl_dim(x, Dk), dr = hr_dim(x, k.Lx, Dk), dd = dn_dim(y, Dk),
                  du = up_dim(y, k.Ly, Dk);
        const int v = y * k.Lx + x;
        const T* src = k.params + k.voff[v] + (long long)bid * k.vbs[v];
        const int bs = dl * dr * dd * du;
        T* box = dst[g];
#pragma unroll 1
        for (int e = tl; e < bs; e += per) {
          int t = e;
          const int iu = t % du; t /= du;
          const int id = t % dd; t /= dd;
          const int ir = t % dr; t /= dr;
          const int il = t;
          box[((il * Dk + ir) * Dk + id) * Dk + iu] = src[e];
        }
      }
    }
    (void)D4;
  }
  __device__ __noinline__ void gather_plaq(int c, int r) {
    const int xs[4] = {c, c + 1, c, c + 1};
    const int ys[4] = {r, r, r + 1, r + 1};
    T* const dst[4] = {prop(0), prop(1), prop(2), prop(3)};
    gather_n(4, xs, ys, dst);
  }
  __device__ __noinline__ void gather_pair(int x0, int y0, T* d0, int x1, int y1, T* d1) {
    const int xs[2] = {x0, x1};
    const int ys[2] = {y0, y1};
    T* const dst[2] = {d0, d1};
    gather_n(2, xs, ys, dst);
  }

  __device__ __noinline__ bool check_and_gather_all() {
    int& bad = sv.bad;
    if (ex.tid() == 0) bad = 0;
    ex.sync();
#pragma unroll 1
    for (int v = ex.tid(); v < k.n_s; v += ex.size()) {
      if (block_of(k, cfg, v % k.Lx, v / k.Lx) < 0) bad = 1;
    }
    ex.sync();
    const bool ok = bad == 0;
    ex.sync();
    if (!ok) return false;
    for (int y = 0; y < k.Ly; ++y)
      for (int x = 0; x < k.Lx; ++x) gather_box(ex, k, x, y, block_of(k, cfg, x, y), box(x, y));
    ex.sync();
    return true;
  }

  // ---- boundary MPS --------------------------------------------------------
  __device__ __noinline__ void absorb_B(int r) {  // B[r] = absorb(B[r-1], row r)
    const bool own_mode = k.absorb_gemm_mode != k.gemm_mode;
    if (own_mode) set_gemm_mode(k.absorb_gemm_mode);
    const int ls = absorb_compress(ex, k, ws, hot, sv.base, net, Bslot(r), bdB(r), physB(r), r, 0, Bslot(r + 1),
                                      bdB(r + 1), physB(r + 1), qrBt(r), svdBt(r), offBt(r), offBt(r + 1),
                                      denseB(r));
    if (ex.tid() == 0) {
      sv.logB[r + 1] = sv.logB[r] + ls;
      if (k.ck_every && (r + 1) % k.ck_every) sv.segB = (r + 1) / k.ck_every;
    }
    ex.sync();
    if (own_mode) set_gemm_mode(k.gemm_mode);
  }
  __device__ __noinline__ void absorb_T(int r) {  // T[r] = absorb(T[r+1], row r flipped)
    const bool own_mode = k.absorb_gemm_mode != k.gemm_mode;
    if (own_mode) set_gemm_mode(k.absorb_gemm_mode);
    const int ls = absorb_compress(ex, k, ws, hot, sv.base, net, Tslot(r + 1), bdT(r + 1), physT(r + 1), r, 1,
                                      Tslot(r), bdT(r), physT(r), qrTt(r), svdTt(r), offTt(r + 1), offTt(r),
                                      denseT(r));
    if (ex.tid() == 0) {
      sv.logT[r] = sv.logT[r + 1] + ls;
      if (k.ck_every && (k.Ly - r) % k.ck_every) sv.segT = (k.Ly - r) / k.ck_every;
    }
    ex.sync();
    if (own_mode) set_gemm_mode(k.gemm_mode);
  }

  // ---- strip (rows r, r+1) between B[r-1] (slot r) and T[r+2] -------------
  __device__ SDims sdims(int r, int c) const {
    SDims d;
    const int* bb = bdB(r);
    const int* bt = bdT(r + 2);
    d.nA = bb[c]; d.nB = bt[c];
    d.nI = d.nJ = hl_dim(c, k.Dk);
    d.nA2 = bb[c + 1]; d.nB2 = bt[c + 1];
    d.nI2 = d.nJ2 = hr_dim(c, k.Lx, k.Dk);
    d.pB = physB(r); d.pM = k.Dk; d.pT = physT(r + 2);
    return d;
  }
  __device__ int env_size(const SDims& d, bool right) const {
    return right ? d.nA2 * d.nI2 * d.nJ2 * d.nB2 : d.nA * d.nI * d.nJ * d.nB;
  }
  __device__ T* envR(int c) const { return eR + (long long)c * k.env_stride; }
  // B / T rows used by the current strip or row pass: staged copies in shared
  // memory when available, else the scratch slots
  const T* curB;
  const T* curT;
  // The staged rows are copied by the tensor memory accelerator (one bulk
  // copy per row, rounded up to 16 bytes within the slot's padding), or by
  // the threads if a bulk wait ran out.
  __device__ __noinline__ void stage(int jb, int jt, int physb, int physt) {
    const T* b = Bslot(jb);
    const T* t = Tslot(jt);
    if (sB) {
      const int nb = sv.offB[k.Lx], nt = sv.offT[k.Lx];
      const unsigned bb = (unsigned)((nb * sizeof(T) + 15) / 16 * 16), bt = (unsigned)((nt * sizeof(T) + 15) / 16 * 16);
      bool bulk = false;
      if (bb + bt < (1u << 20)) bulk = bulk_copy2(ex, sB, b, bb, sT, t, bt, k.status + ST_TC_TIMEOUT);
      if (!bulk) {
#pragma unroll 1
        for (int i = ex.tid(); i < nb; i += ex.size()) sB[i] = b[i];
#pragma unroll 1
        for (int i = ex.tid(); i < nt; i += ex.size()) sT[i] = t[i];
      }
      ex.sync();
      curB = sB;
      curT = sT;
    } else {
      curB = b;
      curT = t;
    }
    (void)physb; (void)physt;
  }

  // builds R_c for c = Lx..0 (exponents in sv.logR), returns the strip value
  // as mantissa (vr, vi) and binary exponent ve
  __device__ __noinline__ void strip_right_envs(int r, R& vr, R& vi, int& ve) {
    const int Lx = k.Lx;
    load_offsets(offBt(r), sv.offB);
    load_offsets(offTt(r + 2), sv.offT);
    stage(r, r + 2, physB(r), physT(r + 2));
    if (ex.tid() == 0) { envR(Lx)[0] = one<T>(); sv.logR[Lx] = 0; }
    ex.sync();
    for (int c = Lx - 1; c >= 0; --c) {
      const SDims d = sdims(r, c);
      const int ls = sright(d, envR(c + 1), curB + sv.offB[c], box(c, r), box(c, r + 1),
                           curT + sv.offT[c], envR(c));
      if (ex.tid() == 0) sv.logR[c] = sv.logR[c + 1] + ls;
      ex.sync();
    }
    vr = re(envR(0)[0]);
    vi = im(envR(0)[0]);
    ve = sv.logR[0];
    ex.sync();
  }

  __device__ __noinline__ int strip_step_left(int r, int c, const T* Lin, const T* W1, const T* W2, T* out) {
    const SDims d = sdims(r, c);
    return sleft(d, Lin, curB + sv.offB[c], W1, W2, curT + sv.offT[c], out);
  }

  __device__ int sleft(const SDims& d, const T* L, const T* Bs, const T* W1, const T* W2, const T* Ts,
                         T* out) {
    switch (k.Dk) {
      case 1: return strip_left<T, 1>(ex, d, L, Bs, W1, W2, Ts, out, t1, t2, cop);
      case 2: return strip_left<T, 2>(ex, d, L, Bs, W1, W2, Ts, out, t1, t2, cop);
      default: return strip_left<T, 3>(ex, d, L, Bs, W1, W2, Ts, out, t1, t2, cop);
    }
  }
  __device__ int sright(const SDims& d, const T* R2, const T* Bs, const T* W1, const T* W2, const T* Ts,
                          T* out) {
    switch (k.Dk) {
      case 1: return strip_right<T, 1>(ex, d, R2, Bs, W1, W2, Ts, out, t1, t2, cop);
      case 2: return strip_right<T, 2>(ex, d, R2, Bs, W1, W2, Ts, out, t1, t2, cop);
      default: return strip_right<T, 3>(ex, d, R2, Bs, W1, W2, Ts, out, t1, t2, cop);
    }
  }
  __device__ int rleft(const RDims& d, const T* L, const T* Bs, const T* W, const T* Ts, T* out) {
    switch (k.Dk) {
      case 1: return row_left<T, 1>(ex, d, L, Bs, W, Ts, out, t1, t2);
      case 2: return row_left<T, 2>(ex, d, L, Bs, W, Ts, out, t1, t2);
      default: return row_left<T, 3>(ex, d, L, Bs, W, Ts, out, t1, t2);
    }
  }
  __device__ int rright(const RDims& d, const T* R2, const T* Bs, const T* W, const T* Ts, T* out) {
    switch (k.Dk) {
      case 1: return row_right<T, 1>(ex, d, R2, Bs, W, Ts, out, t1, t2);
      case 2: return row_right<T, 2>(ex, d, R2, Bs, W, Ts, out, t1, t2);
      default: return row_right<T, 3>(ex, d, R2, Bs, W, Ts, out, t1, t2);
    }
  }
  __device__ void ropen(const RDims& d, const T* L, const T* Bs, const T* Ts, const T* R2, T* G) {
    switch (k.Dk) {
      case 1: row_open<T, 1>(ex, d, L, Bs, Ts, R2, G, t1, t2); break;
      case 2: row_open<T, 2>(ex, d, L, Bs, Ts, R2, G, t1, t2); break;
      default: row_open<T, 3>(ex, d, L, Bs, Ts, R2, G, t1, t2); break;
    }
  }

  // ---- row r between B[r-1] (slot r) and T[r+1] ---------------------------
  __device__ RDims rdims(int r, int c) const {
    RDims d;
    const int* bb = bdB(r);
    const int* bt = bdT(r + 1);
    d.nA = bb[c]; d.nB = bt[c]; d.nH = hl_dim(c, k.Dk);
    d.nA2 = bb[c + 1]; d.nB2 = bt[c + 1]; d.nH2 = hr_dim(c, k.Lx, k.Dk);
    d.pB = physB(r); d.pT = physT(r + 1);
    return d;
  }
  __device__ T* env3R(int c) const { return e3R + (long long)c * k.env3_stride; }

  __device__ __noinline__ void row_right_envs(int r, R& vr, R& vi, int& ve) {
    const int Lx = k.Lx;
    load_offsets(offBt(r), sv.offB);
    load_offsets(offTt(r + 1), sv.offT);
    stage(r, r + 1, physB(r), physT(r + 1));
    if (ex.tid() == 0) { env3R(Lx)[0] = one<T>(); sv.logR[Lx] = 0; }
    ex.sync();
    for (int c = Lx - 1; c >= 0; --c) {
      const RDims d = rdims(r, c);
      const int ls = rright(d, env3R(c + 1), curB + sv.offB[c], box(c, r), curT + sv.offT[c], env3R(c));
      if (ex.tid() == 0) sv.logR[c] = sv.logR[c + 1] + ls;
      ex.sync();
    }
    vr = re(env3R(0)[0]);
    vi = im(env3R(0)[0]);
    ve = sv.logR[0];
    ex.sync();
  }

  __device__ __noinline__ int row_step_left(int r, int c, const T* Lin, const T* W, T* out) {
    const RDims d = rdims(r, c);
    return rleft(d, Lin, curB + sv.offB[c], W, curT + sv.offT[c], out);
  }

  // Metropolis decision (Sec. S-1): accept iff u |den|^2 < |num|^2, with
  // den = (dr + i di) 2^de and num = (nr + i ni) 2^ne; evaluated once on
  // thread 0 (exact powers of two, no logarithms) and broadcast.
  __device__ __noinline__ bool metro_accept(double u, R dr, R di, int de, R nr, R ni, int ne) {
    if (ex.tid() == 0) {
      const double d2 = (double)dr * dr + (double)di * di;
      const double n2 = (double)nr * nr + (double)ni * ni;
      bool acc;
      if (!(n2 > 0.0)) acc = false;
      else if (!(d2 > 0.0)) acc = true;
      else acc = u * d2 < n2 * pow2d_exact(2 * (ne - de));
      sv.flag = acc ? 1 : 0;
    }
    ex.sync();
    const bool a = sv.flag != 0;
    ex.sync();
    return a;
  }
  // eacc += coef * num / den (thread 0)
  __device__ __noinline__ void add_ratio(double coef, R nr, R ni, int ne, R dr, R di, int de) {
    if (ex.tid() == 0) {
      // (nr + i ni) / (dr + i di) in the chain's precision, after scaling
      // both by the same exact power of two (|d| in [0.5, 1), so d2 cannot
      // underflow), then the exact power-of-two scale and FP64 accumulation
      const float m = fmaxf(fabsf((float)dr), fabsf((float)di));
      const R sc = m > 0.f ? pow2r<R>(-exp2_of(m)) : R(1);
      dr *= sc; di *= sc; nr *= sc; ni *= sc;
      const R d2 = dr * dr + di * di;
      const R qr = (nr * dr + ni * di) / d2;
      const R qi = (ni * dr - nr * di) / d2;
      const double f = pow2d_exact(ne - de);
      sv.eacc[0] += coef * ((double)qr * f);
      sv.eacc[1] += coef * ((double)qi * f);
    }
  }

  // ---- RNG -------------------------------------------------------------------
  __device__ double uniform_at(unsigned long long ctr) const {
    return word_to_uniform(stream_word(key, ctr));
  }
  // E_loc term of the hop across horizontal link (c, r) -> (c+1, r), from the
  // row environments of the measurement pass (left env Lc at column c)
  __device__ __noinline__ void hhop_ratio(int r, int c, const T* Lc, T* X1, T* X2, int eL, R dr, R di, int de) {
    if (!hop_apply(c, r, 1)) return;
    gather_pair(c, r, prop(0), c + 1, r, prop(1));
    ex.sync();
    const int l1 = row_step_left(r, c, Lc, prop(0), X1);
    const int l2 = row_step_left(r, c + 1, X1, prop(1), X2);
    R nr, ni;
    const RDims d2 = rdims(r, c + 1);
    cta_dot(ex, X2, env3R(c + 2), d2.nA2 * d2.nH2 * d2.nB2, nr, ni);
    add_ratio(k.J, nr, ni, eL + l1 + l2 + sv.logR[c + 2], dr, di, de);
    hop_apply(c, r, 1);
  }
  // E_loc term of the hop across vertical link (c, r) -> (c, r+1), from the
  // strip environments of the measurement pass (left env Lc at column c)
  __device__ __noinline__ void vhop_ratio(int r, int c, const T* Lc, T* X1, int eL, R dr, R di, int de) {
    if (!hop_apply(c, r, 2)) return;
    gather_pair(c, r, prop(0), c, r + 1, prop(2));
    ex.sync();
    const int l1 = strip_step_left(r, c, Lc, prop(0), prop(2), X1);
    R nr, ni;
    const SDims d1 = sdims(r, c);
    cta_dot(ex, X1, envR(c + 1), env_size(d1, true), nr, ni);
    add_ratio(k.J, nr, ni, eL + l1 + sv.logR[c + 1], dr, di, de);
    hop_apply(c, r, 2);
  }

  __device__ int power_at(unsigned long long ctr) const {
    if (k.N == 2) return 1;
    return 1 + (int)(stream_word(key, ctr) % (unsigned long long)(k.N - 1));
  }
};

template <class T, class X>
__device__ void copy_box(const X ex, T* dst, const T* src, int n) {
#pragma unroll 1
  for (int i = ex.tid(); i < n; i += ex.size()) dst[i] = src[i];
}

// ---------------------------------------------------------------------------
// Passes
// ---------------------------------------------------------------------------

// plaquette pass, bottom-up, Metropolis (Sec. S-1 rule, Sec. S-2 moves)
template <class T, class X>
__device__ __noinline__ void plaquette_pass(Chain<T, X>& ch, int w) {
  const X ex = ch.ex;
  using R = typename Traits<T>::R;
  const KParams<T>& k = ch.k;
  const int Lx = k.Lx, Ly = k.Ly, D4 = k.Dk * k.Dk * k.Dk * k.Dk;
  T* Lc = ch.envL;
  T* X1 = ch.envX;
  T* X2 = ch.envY;
  for (int r = 0; r < Ly - 1; ++r) {
    ch.phase_sync();
    ch.ensure_T(r + 2);
    R dr, di;
    int de;
    ch.strip_right_envs(r, dr, di, de);
    if (ex.tid() == 0) Lc[0] = one<T>();
    ex.sync();
    int eL = 0;
    for (int c = 0; c < Lx - 1; ++c) {
      const int j = r * (Lx - 1) + c;
      const unsigned long long base = (unsigned long long)w * k.n_slots;
      const int t = ch.power_at(base + 2 * j);
      const double u = ch.uniform_at(base + 2 * j + 1);
      ch.plaq_apply(c, r, t);
      ch.gather_plaq(c, r);
      ex.sync();
      const int l1 = ch.strip_step_left(r, c, Lc, ch.prop(0), ch.prop(2), X1);
      const int l2 = ch.strip_step_left(r, c + 1, X1, ch.prop(1), ch.prop(3), X2);
      R nr, ni;
      const SDims d2 = ch.sdims(r, c + 1);
      cta_dot(ex, X2, ch.envR(c + 2), ch.env_size(d2, true), nr, ni);
      const int ne = eL + l1 + l2 + ch.sv.logR[c + 2];
      const bool acc = ch.metro_accept(u, dr, di, de, nr, ni, ne);
      if (ex.tid() == 0) { ch.sv.n_prop += 1; if (acc) ch.sv.n_acc += 1; }
      const SDims d1 = ch.sdims(r, c);
      const int n1 = ch.env_size(d1, true);
      if (acc) {
        copy_box(ex, ch.box(c, r), ch.prop(0), D4);
        copy_box(ex, ch.box(c + 1, r), ch.prop(1), D4);
        copy_box(ex, ch.box(c, r + 1), ch.prop(2), D4);
        copy_box(ex, ch.box(c + 1, r + 1), ch.prop(3), D4);
        dr = nr; di = ni; de = ne;
        // L_{c+1} is X1 (built from the accepted column c)
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
        eL += l1;
      } else {
        ch.plaq_apply(c, r, k.N - t);  // revert
        eL += ch.strip_step_left(r, c, Lc, ch.box(c, r), ch.box(c, r + 1), X1);
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
      }
      ex.sync();
    }
    ch.absorb_B(r);
  }
}

// horizontal-hop pass (matter), top-down with row environments
template <class T, class X>
__device__ __noinline__ void hhop_pass(Chain<T, X>& ch, int w) {
  const X ex = ch.ex;
  using R = typename Traits<T>::R;
  const KParams<T>& k = ch.k;
  const int Lx = k.Lx, Ly = k.Ly, D4 = k.Dk * k.Dk * k.Dk * k.Dk;
  T* Lc = ch.env3L;
  T* X1 = ch.env3X;
  T* X2 = ch.env3Y;
  for (int r = Ly - 1; r >= 0; --r) {
    ch.phase_sync();
    ch.ensure_B(r);
    R dr, di;
    int de;
    ch.row_right_envs(r, dr, di, de);
    if (ex.tid() == 0) Lc[0] = one<T>();
    ex.sync();
    int eL = 0;
    for (int c = 0; c < Lx - 1; ++c) {
      const unsigned long long ctr =
          (unsigned long long)w * k.n_slots + 2 * k.n_plaq + r * (Lx - 1) + c;
      const double u = ch.uniform_at(ctr);
      bool acc = false;
      int l1 = 0;
      if (ch.hop_apply(c, r, 1)) {
        ch.gather_pair(c, r, ch.prop(0), c + 1, r, ch.prop(1));
        ex.sync();
        l1 = ch.row_step_left(r, c, Lc, ch.prop(0), X1);
        const int l2 = ch.row_step_left(r, c + 1, X1, ch.prop(1), X2);
        R nr, ni;
        const RDims d2 = ch.rdims(r, c + 1);
        cta_dot(ex, X2, ch.env3R(c + 2), d2.nA2 * d2.nH2 * d2.nB2, nr, ni);
        const int ne = eL + l1 + l2 + ch.sv.logR[c + 2];
        acc = ch.metro_accept(u, dr, di, de, nr, ni, ne);
        if (ex.tid() == 0) { ch.sv.n_prop += 1; if (acc) ch.sv.n_acc += 1; }
        if (acc) {
          copy_box(ex, ch.box(c, r), ch.prop(0), D4);
          copy_box(ex, ch.box(c + 1, r), ch.prop(1), D4);
          dr = nr; di = ni; de = ne;
        } else {
          ch.hop_apply(c, r, 1);
        }
      }
      ex.sync();
      const RDims d1 = ch.rdims(r, c);
      const int n1 = d1.nA2 * d1.nH2 * d1.nB2;
      if (acc) {
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
        eL += l1;
      } else {
        eL += ch.row_step_left(r, c, Lc, ch.box(c, r), X1);
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
      }
      ex.sync();
    }
    if (r >= 1) ch.absorb_T(r);
  }
}

// vertical-hop pass (matter), bottom-up with strip environments
template <class T, class X>
__device__ __noinline__ void vhop_pass(Chain<T, X>& ch, int w) {
  const X ex = ch.ex;
  using R = typename Traits<T>::R;
  const KParams<T>& k = ch.k;
  const int Lx = k.Lx, Ly = k.Ly, D4 = k.Dk * k.Dk * k.Dk * k.Dk;
  T* Lc = ch.envL;
  T* X1 = ch.envX;
  T* Lnext = ch.envY;
  for (int r = 0; r < Ly - 1; ++r) {
    ch.phase_sync();
    ch.ensure_T(r + 2);
    R dr, di;
    int de;
    ch.strip_right_envs(r, dr, di, de);
    if (ex.tid() == 0) Lc[0] = one<T>();
    ex.sync();
    int eL = 0;
    for (int c = 0; c < Lx; ++c) {
      const unsigned long long ctr =
          (unsigned long long)w * k.n_slots + 2 * k.n_plaq + k.n_h + r * Lx + c;
      const double u = ch.uniform_at(ctr);
      bool acc = false;
      int l1 = 0;
      if (ch.hop_apply(c, r, 2)) {
        ch.gather_pair(c, r, ch.prop(0), c, r + 1, ch.prop(2));
        ex.sync();
        l1 = ch.strip_step_left(r, c, Lc, ch.prop(0), ch.prop(2), X1);
        R nr, ni;
        const SDims d1 = ch.sdims(r, c);
        cta_dot(ex, X1, ch.envR(c + 1), ch.env_size(d1, true), nr, ni);
        const int ne = eL + l1 + ch.sv.logR[c + 1];
        acc = ch.metro_accept(u, dr, di, de, nr, ni, ne);
        if (ex.tid() == 0) { ch.sv.n_prop += 1; if (acc) ch.sv.n_acc += 1; }
        if (acc) {
          copy_box(ex, ch.box(c, r), ch.prop(0), D4);
          copy_box(ex, ch.box(c, r + 1), ch.prop(2), D4);
          dr = nr; di = ni; de = ne;
        } else {
          ch.hop_apply(c, r, 2);
        }
      }
      ex.sync();
      const SDims d1 = ch.sdims(r, c);
      const int n1 = ch.env_size(d1, true);
      if (acc) {
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
        eL += l1;
      } else {
        eL += ch.strip_step_left(r, c, Lc, ch.box(c, r), ch.box(c, r + 1), Lnext);
#pragma unroll 1
        for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = Lnext[i];
      }
      ex.sync();
    }
    ch.absorb_B(r);
  }
}

// measurement pass, top-down; writes sample s
template <class T, class X>
__device__ __noinline__ void measure_pass(Chain<T, X>& ch, long long s) {
  const X ex = ch.ex;
  using R = typename Traits<T>::R;
  const KParams<T>& k = ch.k;
  const int Lx = k.Lx, Ly = k.Ly, Dk = k.Dk, D4 = Dk * Dk * Dk * Dk;
  const bool want_e = (k.want & WANT_ELOC) && k.e_loc;
  const bool want_g = (k.want & WANT_GRAD) && (k.O || k.block_ids);
  const bool want_a = (k.want & WANT_AMP) && (k.log_abs || k.phase);
  if (ex.tid() == 0) { ch.sv.eacc[0] = 0.0; ch.sv.eacc[1] = 0.0; }
  ex.sync();
  for (int r = Ly - 1; r >= 0; --r) {
    ch.phase_sync();
    ch.ensure_B(r);
    // ---- row r: gradient, horizontal hops, amplitude
    const bool need_row = want_g || (r == Ly - 1 && want_a) || (want_e && k.matter && k.J != 0.0);
    if (need_row) {
      ch.set_gemm_mode(k.row_gemm_mode);
      R dr, di;
      int de;
      ch.row_right_envs(r, dr, di, de);
      if (r == Ly - 1 && want_a && ex.tid() == 0) {
        // psi = <B[Ly-2] | row Ly-1> = (dr + i di) 2^(de + e_B)
        const double a2 = (double)dr * dr + (double)di * di;
        const double ln2 = 0.69314718055994530942;
        const double la = (a2 > 0.0) ? (double)(ch.sv.logB[Ly - 1] + de) * ln2 + 0.5 * log(a2) : -INFINITY;
        if (k.log_abs) k.log_abs[s] = la;
        if (k.phase) k.phase[s] = (a2 > 0.0) ? atan2((double)di, (double)dr) : 0.0;
      }
      T* Lc = ch.env3L;
      T* X1 = ch.env3X;
      T* X2 = ch.env3Y;
      if (ex.tid() == 0) Lc[0] = one<T>();
      ex.sync();
      int eL = 0;
      const R den2 = dr * dr + di * di;
      for (int c = 0; c < Lx; ++c) {
        const RDims d = ch.rdims(r, c);
        if (want_g) {
          T* G = ch.ws + k.o_G;
          ch.ropen(d, Lc, ch.curB + ch.sv.offB[c], ch.curT + ch.sv.offT[c], ch.env3R(c + 1), G);
          // O = G 2^(eL + eR[c+1] - de) / (dr + i di)
          const R f = pow2r<R>(eL + ch.sv.logR[c + 1] - de) / den2;
          const T fac = make_scalar<T>(dr * f, -di * f);
          const int v = r * Lx + c;
          const int n = d.nH * d.nH2 * d.pB * d.pT;
          if (k.O) {
            T* dst = k.O + (s * k.n_s + v) * (long long)D4;
#pragma unroll 1
            for (int i = ex.tid(); i < n; i += ex.size()) store_stream(dst + i, G[i] * fac);
          }
          if (k.block_ids && ex.tid() == 0) store_stream(k.block_ids + s * k.n_s + v, block_of(k, ch.cfg, c, r));
        }
        if (want_e && k.matter && k.J != 0.0 && c < Lx - 1) ch.hhop_ratio(r, c, Lc, X1, X2, eL, dr, di, de);
        if (c < Lx - 1) {
          eL += ch.row_step_left(r, c, Lc, ch.box(c, r), X1);
          const int n1 = d.nA2 * d.nH2 * d.nB2;
#pragma unroll 1
          for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
          ex.sync();
        }
      }
    }
    ch.set_gemm_mode(k.gemm_mode);
    // ---- strip (r, r+1): plaquettes and vertical hops
    if (want_e && r <= Ly - 2) {
      R dr, di;
      int de;
      ch.strip_right_envs(r, dr, di, de);
      T* Lc = ch.envL;
      T* X1 = ch.envX;
      T* X2 = ch.envY;
      if (ex.tid() == 0) Lc[0] = one<T>();
      ex.sync();
      int eL = 0;
      const int npow = k.N == 2 ? 1 : 2;
      const double amp = k.N == 2 ? -2.0 * k.h : -k.h;
      for (int c = 0; c < Lx; ++c) {
        if (c < Lx - 1 && k.h != 0.0) {
          for (int q = 0; q < npow; ++q) {
            const int t = q == 0 ? 1 : k.N - 1;
            ch.plaq_apply(c, r, t);
            ch.gather_plaq(c, r);
            ex.sync();
            const int l1 = ch.strip_step_left(r, c, Lc, ch.prop(0), ch.prop(2), X1);
            const int l2 = ch.strip_step_left(r, c + 1, X1, ch.prop(1), ch.prop(3), X2);
            R nr, ni;
            const SDims d2 = ch.sdims(r, c + 1);
            cta_dot(ex, X2, ch.envR(c + 2), ch.env_size(d2, true), nr, ni);
            ch.add_ratio(amp, nr, ni, eL + l1 + l2 + ch.sv.logR[c + 2], dr, di, de);
            ch.plaq_apply(c, r, k.N - t);
          }
        }
        if (k.matter && k.J != 0.0) ch.vhop_ratio(r, c, Lc, X1, eL, dr, di, de);
        if (c < Lx - 1) {
          const SDims d1 = ch.sdims(r, c);
          eL += ch.strip_step_left(r, c, Lc, ch.box(c, r), ch.box(c, r + 1), X1);
          const int n1 = ch.env_size(d1, true);
#pragma unroll 1
          for (int i = ex.tid(); i < n1; i += ex.size()) Lc[i] = X1[i];
          ex.sync();
        }
      }
    }
    // ---- T[r]
    if (r >= 1 && (k.mode == 1 || want_e || want_g)) ch.absorb_T(r);
  }
  if (want_e && ex.tid() == 0) {
    // diagonal part: g sum_links (2 - 2 cos(2 pi n / N)) (table) + m sum_x p_x
    double e = 0.0;
    for (int i = 0; i < k.n_h + k.n_v; ++i) e += k.elink[ch.cfg[i]];
    if (k.matter)
      for (int i = 0; i < k.n_s; ++i) e += k.m * ch.cfg[k.n_h + k.n_v + i];
    k.e_loc[2 * s] = e + ch.sv.eacc[0];
    k.e_loc[2 * s + 1] = ch.sv.eacc[1];
  }
  ex.sync();
}

template <class T, class X>
__device__ void init_trivial_slots(const X ex, const KParams<T>& k, T* ws) {
#pragma unroll 1
  for (int c = ex.tid(); c < k.Lx; c += ex.size()) {
    bslot_ptr(k, ws, 0)[c] = one<T>();      // B[-1]
    tslot_ptr(k, ws, k.Ly)[c] = one<T>();   // T[Ly]
  }
  ex.sync();
}

// The context's integer tables (bond dimensions, QR / SVD plans, MPS site
// offsets, dense-step flags) are read in every environment step and by the
// serial bookkeeping of each absorption; a shared-memory copy per CTA turns
// those dependent global loads into shared-memory loads.  Lattices whose
// tables exceed the copy (above about 16 x 16) read them from global memory.
constexpr int kTabCap = 2560;
__shared__ int g_tab[kTabCap];

template <class T>
__device__ const int* stage_tables(const KParams<T>& k) {
  const bool fits = k.tab_ints <= kTabCap;
  if (fits) {
#pragma unroll 1
    for (int i = threadIdx.x; i < k.tab_ints; i += blockDim.x) g_tab[i] = k.tab[i];
  }
  __syncthreads();
  return fits ? g_tab : k.tab;
}

// Lockstep decision of one chain round, taken by every group of the CTA (with
// or without a chain): lock only if all groups have a physical chain.
template <class X>
__device__ void lock_exchange(const X ex, SharedV* sv, int grp, int n_groups, bool ok) {
  if (ex.leader()) g_lock_ok[grp] = ok ? 1 : 0;
  if (threadIdx.x == 0) g_phase_arrive = 0;  // the previous round's arrivals are complete
  __syncthreads();
  if (sv && ex.leader()) {
    int all = 1;
    for (int i = 0; i < n_groups; ++i) all &= g_lock_ok[i];
    sv->lock = all;
    sv->phase = 0;
  }
  __syncthreads();
}

// Per-chain body shared by the kernels.
template <class T, class X>
__device__ void run_chain(const X ex, const KParams<T>& k, T* ws, SharedV& sv, int8_t* cfg, T* hot, const int* tab,
                          int chain, int lock_group = -1, int n_groups = 1) {
  int8_t* gcfg = k.configs + (long long)chain * k.cfg_len;
#pragma unroll 1
  for (int i = ex.tid(); i < k.cfg_len; i += ex.size()) cfg[i] = gcfg[i];
  if (ex.leader()) {
    sv.logB[0] = 0; sv.logT[k.Ly] = 0; sv.n_acc = 0; sv.n_prop = 0;
    sv.lock = 0; sv.phase = 0;
    sv.segB = -1; sv.segT = -1;
  }
  ex.sync();
  Chain<T, X> ch(ex, k, ws, sv, cfg, chain, hot, tab);
  const bool ok = ch.check_and_gather_all();
  if (lock_group >= 0) lock_exchange(ex, &sv, lock_group, n_groups, ok);
  if (!ok) {
    if (ex.leader()) {
      atomicAdd(&k.status[ST_GAUSS], 1);
      const int ns = k.mode == 1 ? k.n_sweeps : 1;
      for (int w = 0; w < ns; ++w) {
        const long long s = (long long)chain * ns + w;
        if (k.log_abs) k.log_abs[s] = -INFINITY;
        if (k.phase) k.phase[s] = 0.0;
        if (k.e_loc) { k.e_loc[2 * s] = NAN; k.e_loc[2 * s + 1] = NAN; }
      }
    }
    ex.sync();
    return;
  }
  if (k.mode == 0) {
    for (int r = 0; r < k.Ly - 1; ++r) {
      ch.phase_sync();
      ch.absorb_B(r);
    }
    measure_pass(ch, (long long)chain);
  } else {
    for (int r = k.Ly - 1; r >= 2; --r) {
      ch.phase_sync();
      ch.absorb_T(r);
    }
    for (int w = 0; w < k.n_sweeps; ++w) {
      plaquette_pass(ch, w);
      if (k.matter) {
        hhop_pass(ch, w);
        vhop_pass(ch, w);
      }
      measure_pass(ch, (long long)chain * k.n_sweeps + w);
    }
#pragma unroll 1
    for (int i = ex.tid(); i < k.cfg_len; i += ex.size()) gcfg[i] = cfg[i];
    if (ex.leader()) {
      if (k.accepted) k.accepted[chain] = sv.n_acc;
      if (k.proposed) k.proposed[chain] = sv.n_prop;
    }
  }
  ex.sync();
}

// Tensor-core set-up of a launch (tcgen05.cuh): TMEM columns and a
// completion barrier per chain group, and each group's operand staging area
// at byte `tc_off` of the group's dynamic shared memory (group g's region
// starts at g * group_bytes).  Every thread of the CTA calls it.
template <class T>
__device__ void tc_begin(const KParams<T>& k, int n_groups, int8_t* dyn_base, long long group_bytes) {
  if (threadIdx.x < 4)
    g_tc_stage[threadIdx.x] = (k.tc_bf16 && threadIdx.x < n_groups)
                                  ? (unsigned char*)(dyn_base + threadIdx.x * group_bytes + k.tc_off)
                                  : nullptr;
  if (threadIdx.x < 4)
    g_fz[threadIdx.x] = (k.fz_elems > 0 && threadIdx.x < n_groups)
                            ? (void*)(dyn_base + threadIdx.x * group_bytes + k.fz_off)
                            : nullptr;
  if (threadIdx.x == 0) {
    g_tc_cap = k.tc_bytes;
    g_tc_status = k.status + ST_TC_TIMEOUT;
    g_fz_elems = k.fz_elems;
  }
  if (k.tc_bf16) tc_setup(n_groups);
  bulk_setup(n_groups);
}
template <class T>
__device__ void tc_end(const KParams<T>& k, int n_groups) {
  __syncthreads();
  bulk_teardown(n_groups);
  if (k.tc_bf16) tc_teardown(n_groups);
}

// One CTA per chain (any size; the general form).
template <class T>
__global__ void __launch_bounds__(256, 2) vmc_kernel(const __grid_constant__ KParams<T> k) {
  extern __shared__ __align__(16) int8_t dyn_smem[];
  int8_t* dyn_cfg = dyn_smem;
  T* hot = (T*)(dyn_smem + k.smem_cfg_bytes);
  __shared__ SharedV sv;
  CtaExec ex;
  if (threadIdx.x < 4) g_gemm_mode[threadIdx.x] = k.gemm_mode;
  const int* tab = stage_tables(k);
  tc_begin(k, 1, dyn_smem, 0);
  T* ws = k.scratch + (long long)blockIdx.x * k.ws_stride;
  init_trivial_slots(ex, k, ws);
  for (int chain = blockIdx.x; chain < k.n_chains; chain += gridDim.x)
    run_chain(ex, k, ws, sv, dyn_cfg, hot, tab, chain);
  tc_end(k, 1);
}

// Several chains per CTA, one per group of G = 128 threads (GroupExec, a
// hardware barrier per group).  Groups never wait on one another.  Dynamic
// shared memory per group: [SharedV][configuration][hot buffers].
template <class T, class X, int G>
__device__ void grouped_body(const KParams<T>& k) {
  extern __shared__ __align__(16) int8_t dyn_smem[];
  if (threadIdx.x < 4) g_gemm_mode[threadIdx.x] = k.gemm_mode;
  const int* tab = stage_tables(k);
  const int g = threadIdx.x / G, NG = blockDim.x / G;
  tc_begin(k, NG, dyn_smem, k.group_smem_bytes);
  int8_t* base = dyn_smem + g * k.group_smem_bytes;
  SharedV& sv = *reinterpret_cast<SharedV*>(base);
  int8_t* cfg = base + sizeof_sharedv_aligned();
  T* hot = (T*)(cfg + k.smem_cfg_bytes);
  X ex;
  const long long slot = (long long)blockIdx.x * NG + g;
  T* ws = k.scratch + slot * k.ws_stride;
  init_trivial_slots(ex, k, ws);
  const long long stride = (long long)gridDim.x * NG;
  if (!k.lockstep) {
    for (long long chain = slot; chain < k.n_chains; chain += stride)
      run_chain(ex, k, ws, sv, cfg, hot, tab, (int)chain);
  } else {
    // lockstep: every group takes part in every round's exchange and barrier
    const long long rounds = (k.n_chains + stride - 1) / stride;
    for (long long rd = 0; rd < rounds; ++rd) {
      const long long chain = slot + rd * stride;
      if (chain < k.n_chains)
        run_chain(ex, k, ws, sv, cfg, hot, tab, (int)chain, g, NG);
      else
        lock_exchange(ex, (SharedV*)nullptr, g, NG, false);
      __syncthreads();
    }
  }
  tc_end(k, NG);
}

template <class T>
__global__ void __launch_bounds__(256, 2) vmc_kernel_grouped(const __grid_constant__ KParams<T> k) {
  grouped_body<T, GroupExec<128>, 128>(k);
}

// Four chains per CTA of 512 threads (one CTA per SM).
template <class T>
__global__ void __launch_bounds__(512, 1) vmc_kernel_grouped4(const __grid_constant__ KParams<T> k) {
  grouped_body<T, GroupExec<128>, 128>(k);
}

// Chains of several contexts (lattices of different sizes) in one persistent
// launch: global chain g belongs to context i with start[i] <= g <
// start[i+1] and is that context's chain g - start[i].  One chain per CTA;
// the scratch arena has a slot of ws_stride (the largest of the contexts)
// per CTA; dynamic shared memory is the largest of the contexts' needs.
template <class T>
__global__ void __launch_bounds__(256, 2)
    vmc_kernel_multi(const KParams<T>* __restrict__ ks, int n_ctx, const long long* __restrict__ start,
                     long long total, T* arena, long long ws_stride, unsigned long long* queue) {
  extern __shared__ __align__(16) int8_t dyn_smem[];
  __shared__ SharedV sv;
  CtaExec ex;
  T* ws = arena + (long long)blockIdx.x * ws_stride;
  const int* tab = nullptr;
  int cur = -1;
  tc_begin(ks[0], 1, dyn_smem, 0);
  for (;;) {
    // the next chain of the launch's queue (contexts in the host's order,
    // the costliest first), taken when this CTA is free
    if (threadIdx.x == 0) sv.next = (long long)atomicAdd(queue, 1ull);
    __syncthreads();
    const long long gidx = sv.next;
    __syncthreads();
    if (gidx >= total) break;
    int i = 0;
    while (i + 1 < n_ctx && gidx >= start[i + 1]) ++i;
    const KParams<T>& k = ks[i];
    if (i != cur) {
      __syncthreads();  // the previous context's chain is done with the tables
      if (threadIdx.x < 4) g_gemm_mode[threadIdx.x] = k.gemm_mode;
      tab = stage_tables(k);
      init_trivial_slots(ex, k, ws);
      cur = i;
    }
    run_chain(ex, k, ws, sv, dyn_smem, (T*)(dyn_smem + k.smem_cfg_bytes), tab, (int)(gidx - start[i]));
  }
  tc_end(ks[0], 1);
}

// The same with four chains per CTA of 512 threads (groups of 128, one CTA
// per SM): chain slot s = 4 blockIdx + group owns scratch s of the arena and
// takes the queue's next chain whenever it is free.
// The groups run chains of different contexts at once, so they read the
// contexts' tables from global memory, keep their hot buffers in scratch
// (placement level 0) and do not keep lockstep; dynamic shared memory per
// group: [SharedV][configuration of the largest context][tcgen05 staging]
// [factorisation workspace] (offsets in the KParams, common to all contexts).
template <class T>
__global__ void __launch_bounds__(512, 1)
    vmc_kernel_multi4(const KParams<T>* __restrict__ ks, int n_ctx, const long long* __restrict__ start,
                      long long total, T* arena, long long ws_stride, long long group_bytes,
                      unsigned long long* queue) {
  extern __shared__ __align__(16) int8_t dyn_smem[];
  constexpr int G = 128;
  const int g = threadIdx.x / G, NG = blockDim.x / G;
  if (threadIdx.x < 4) g_gemm_mode[threadIdx.x] = ks[0].gemm_mode;
  tc_begin(ks[0], NG, dyn_smem, group_bytes);
  int8_t* base = dyn_smem + g * group_bytes;
  SharedV& sv = *reinterpret_cast<SharedV*>(base);
  int8_t* cfg = base + sizeof_sharedv_aligned();
  GroupExec<G> ex;
  const long long slot = (long long)blockIdx.x * NG + g;
  T* ws = arena + slot * ws_stride;
  int cur = -1;
  for (;;) {
    if (ex.leader()) sv.next = (long long)atomicAdd(queue, 1ull);
    ex.sync();
    const long long gidx = sv.next;
    ex.sync();
    if (gidx >= total) break;
    int i = 0;
    while (i + 1 < n_ctx && gidx >= start[i + 1]) ++i;
    const KParams<T>& k = ks[i];
    if (i != cur) {
      init_trivial_slots(ex, k, ws);
      cur = i;
    }
    run_chain(ex, k, ws, sv, cfg, (T*)(cfg + k.smem_cfg_bytes), k.tab, (int)(gidx - start[i]));
  }
  tc_end(ks[0], NG);
}

}  // namespace gcf
