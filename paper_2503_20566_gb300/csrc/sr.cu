// FP64 reductions and the stochastic-reconfiguration / tVMC solve.
//
// Paper, Sec. S-1 (Eq. S3, read as F = <O^* E> - <O^*><E>) and Sec. S-3
// (Eqs. S6-S8): S_mn = <O_m^* O_n> - <O_m^*><O_n>; (S + lambda) x = F is
// solved by conjugate gradient without forming S, using the sparsity of O:
// sample s touches exactly one block per vertex.
//   S v = (1/Ns) sum_s O_s^* (t_s - tbar),  t_s = O_s . v,  tbar = mean_s t_s.
// Everything here runs in FP64 (complex FP64 for complex tensors).
#include <type_traits>

#include "sr.cuh"

namespace gcf {

__device__ inline void atomic_add_c(cdouble* a, double r, double i) {
  atomicAdd(&a->x, r);
  atomicAdd(&a->y, i);
}

template <class T>
__device__ inline cdouble to_cd(T v) {
  return {(double)re(v), (double)im(v)};
}

// t_s = sum_v sum_e O[s][v][e] * x[off(v, bid) + e]; one warp per sample.
template <class T>
__global__ void k_gather_dot(SrGeom g, const int* bids, const T* O, const cdouble* x, cdouble* t) {
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= g.Ns) return;
  double ar = 0.0, ai = 0.0;
  for (int v = 0; v < g.n_s; ++v) {
    const int bid = bids[s * g.n_s + v];
    const int bs = g.vbs[v];
    const long long base = g.voff[v] + (long long)bid * bs;
    const T* o = O + (s * g.n_s + v) * (long long)g.D4;
    for (int e = lane; e < bs; e += 32) {
      const cdouble a = to_cd(o[e]);
      const cdouble b = x[base + e];
      ar += a.x * b.x - a.y * b.y;
      ai += a.x * b.y + a.y * b.x;
    }
  }
  ar = warp_sum(ar);
  ai = warp_sum(ai);
  if (lane == 0) t[s] = {ar, ai};
}

// out[off(v,bid)+e] += sum_s coef_s * conj?(O[s][v][e]) for one vertex per
// blockIdx.y and a chunk of samples per blockIdx.x; block-local accumulation
// in shared memory (all blocks of the vertex), flushed with global atomics.
template <class T, bool CONJ>
__global__ void k_scatter(SrGeom g, const int* bids, const T* O, const cdouble* coef, cdouble* out,
                          int chunk) {
  extern __shared__ double acc[];  // 2 * nb_v * bs_v
  const int v = blockIdx.y;
  const int bs = g.vbs[v];
  const int nb = g.vnb[v];
  const int n = nb * bs;
  for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) acc[i] = 0.0;
  __syncthreads();
  const long long s0 = (long long)blockIdx.x * chunk;
  const long long s1 = min((long long)g.Ns, s0 + chunk);
  const long long tot = (s1 - s0) * bs;
  for (long long q = threadIdx.x; q < tot; q += blockDim.x) {
    const long long s = s0 + q / bs;
    const int e = (int)(q % bs);
    const int bid = bids[s * g.n_s + v];
    cdouble o = to_cd(O[(s * g.n_s + v) * (long long)g.D4 + e]);
    if (CONJ) o.y = -o.y;
    const cdouble c = coef[s];
    const double pr = c.x * o.x - c.y * o.y, pi = c.x * o.y + c.y * o.x;
    atomicAdd(&acc[2 * (bid * bs + e)], pr);
    atomicAdd(&acc[2 * (bid * bs + e) + 1], pi);
  }
  __syncthreads();
  cdouble* dst = out + g.voff[v];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double r = acc[2 * i], im_ = acc[2 * i + 1];
    if (r != 0.0 || im_ != 0.0) atomic_add_c(&dst[i], r, im_);
  }
}

// per-chain means of E_loc and the global mean (one block per chain)
__global__ void k_chain_means(const double* e, int n_per_chain, cdouble* chain_mean) {
  __shared__ double red[64];
  const int c = blockIdx.x;
  double r = 0.0, i = 0.0;
  for (int s = threadIdx.x; s < n_per_chain; s += blockDim.x) {
    r += e[2 * ((long long)c * n_per_chain + s)];
    i += e[2 * ((long long)c * n_per_chain + s) + 1];
  }
  block_sum2(r, i, red);
  if (threadIdx.x == 0) chain_mean[c] = {r / n_per_chain, i / n_per_chain};
}

// mean and std error over m values (single block); out[0..2] = Re, Im, err
__global__ void k_mean_err(const cdouble* v, int m, double* out) {
  __shared__ double red[64];
  double r = 0.0, i = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) { r += v[k].x; i += v[k].y; }
  block_sum2(r, i, red);
  const double mr = r / m, mi = i / m;
  double q = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) q += (v[k].x - mr) * (v[k].x - mr);
  q = block_sum(q, red);
  if (threadIdx.x == 0) {
    out[0] = mr;
    out[1] = mi;
    out[2] = m > 1 ? sqrt(q / (m - 1) / m) : 0.0;
  }
}

// E_loc as complex per sample; coefficient for F: (E_s - Ebar) / Ns
__global__ void k_f_coef(const double* e, long long Ns, const double* emean, cdouble* coef) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Ns) return;
  coef[s] = {(e[2 * s] - emean[0]) / (double)Ns, (e[2 * s + 1] - emean[1]) / (double)Ns};
}

// coef_s = (t_s - tbar) / Ns where tbar = mean t
__global__ void k_center(cdouble* t, long long Ns, const cdouble* tbar) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= Ns) return;
  t[s] = {(t[s].x - tbar->x) / (double)Ns, (t[s].y - tbar->y) / (double)Ns};
}

__global__ void k_sum_c(const cdouble* v, long long n, cdouble* out, double scale_) {
  __shared__ double red[64];
  double r = 0.0, i = 0.0;
  for (long long k = threadIdx.x; k < n; k += blockDim.x) { r += v[k].x; i += v[k].y; }
  block_sum2(r, i, red);
  if (threadIdx.x == 0) *out = {r * scale_, i * scale_};
}

// First stage of a deterministic sum over many blocks: block b writes the sum
// of its grid-stride share to part[b]; k_sum_c over part[] finishes it.
__global__ void k_sum_c_part(const cdouble* v, long long n, cdouble* part) {
  __shared__ double red[64];
  double r = 0.0, i = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    r += v[k].x;
    i += v[k].y;
  }
  block_sum2(r, i, red);
  if (threadIdx.x == 0) part[blockIdx.x] = {r, i};
}

// FP32 copy of the real parts of a vector.  The FP32-storage kernels form
// their products in FP32 from exactly these values, so reading the copy
// instead of the FP64 vector changes no result.
__global__ void k_real_to_f32(const cdouble* v, long long n, float* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = (float)v[k].x;
}

// dot products <a, b> = sum conj(a) b (single block, grid-stride)
__global__ void k_dot(const cdouble* a, const cdouble* b, long long n, double* out) {
  __shared__ double red[64];
  double r = 0.0, i = 0.0;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x) {
    r += a[k].x * b[k].x + a[k].y * b[k].y;
    i += a[k].x * b[k].y - a[k].y * b[k].x;
  }
  block_sum2(r, i, red);
  if (threadIdx.x == 0) { atomicAdd(&out[0], r); atomicAdd(&out[1], i); }
}

// y = y + lambda x (the diagonal shift)
__global__ void k_axpy_real(cdouble* y, const cdouble* x, double a, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) { y[k].x += a * x[k].x; y[k].y += a * x[k].y; }
}

// CG vector update: x += alpha p; r -= alpha Ap; alpha = rz / pAp (real)
__global__ void k_cg_xr(cdouble* x, cdouble* r, const cdouble* p, const cdouble* Ap,
                        const double* sc, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double alpha = sc[0] / sc[2];
  x[k].x += alpha * p[k].x; x[k].y += alpha * p[k].y;
  r[k].x -= alpha * Ap[k].x; r[k].y -= alpha * Ap[k].y;
}

// p = z + beta p, beta = rz_new / rz_old (z = M^-1 r; z = r without
// preconditioning)
__global__ void k_cg_p(cdouble* p, const cdouble* z, const double* sc, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double beta = sc[4] / sc[0];
  p[k].x = z[k].x + beta * p[k].x;
  p[k].y = z[k].y + beta * p[k].y;
}

// params += c * x  (c complex); real storage takes the real part
template <class T>
__global__ void k_update(T* params, const cdouble* x, double cr, double ci, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double dr = cr * x[k].x - ci * x[k].y;
  const double di = cr * x[k].y + ci * x[k].x;
  T v = params[k];
  params[k] = make_scalar<T>((double)re(v) + dr, (double)im(v) + di);
}

// ---------------------------------------------------------------------------
// Sample order grouped by (vertex, block): for every vertex a stable counting
// sort of the samples by the block they select.  seg[v * (maxnb + 1) + b] is
// the start of block b of vertex v inside perm[v * Ns ...]; built once per SR
// step (block ids do not change during the solve).  One CTA per vertex.
// ---------------------------------------------------------------------------
__global__ void k_sort_by_block(SrGeom g, const int* bids, int maxnb, int* perm, int* seg) {
  __shared__ int wsum[32];
  __shared__ int base_s;
  const int v = blockIdx.x;
  const int nb = g.vnb[v];
  const long long Ns = g.Ns;
  int* pv = perm + (long long)v * Ns;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  for (int b = 0; b < nb; ++b) {
    if (threadIdx.x == 0) seg[v * (maxnb + 1) + b] = base_s;
    __syncthreads();
    for (long long s0 = 0; s0 < Ns; s0 += blockDim.x) {
      const long long s = s0 + threadIdx.x;
      const int hit = (s < Ns && bids[s * g.n_s + v] == b) ? 1 : 0;
      // block-wide exclusive scan of hit (stable order)
      const unsigned m = __ballot_sync(0xffffffffu, hit);
      const int before = __popc(m & ((1u << lane) - 1u));
      if (lane == 0) wsum[wid] = __popc(m);
      __syncthreads();
      int off = 0, tot = 0;
      for (int w = 0; w < nw; ++w) {
        if (w < wid) off += wsum[w];
        tot += wsum[w];
      }
      if (hit) pv[base_s + off + before] = (int)s;
      __syncthreads();
      if (threadIdx.x == 0) base_s += tot;
      __syncthreads();
    }
  }
  if (threadIdx.x == 0) seg[v * (maxnb + 1) + nb] = base_s;
}

// storage-precision accumulator type: FP32 forms accumulate short partial
// sums in float before adding them into FP64
template <class T> struct PartialOf { using type = double; };
template <> struct PartialOf<float> { using type = float; };
template <> struct PartialOf<cfloat> { using type = float; };

// t_s = sum_v sum_e O[s][v][e] x[off(v, bid) + e]: one warp per sample, lanes
// over vertices; the per-vertex block dot in the storage precision, the sum
// over vertices in FP64.  CPLX selects complex arithmetic.
template <class T, bool CPLX>
__global__ void k_gather2(SrGeom g, const int* bids, const T* O, const cdouble* x, cdouble* t) {
  using P = typename PartialOf<T>::type;
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= g.Ns) return;
  double ar = 0.0, ai = 0.0;
  for (int v = lane; v < g.n_s; v += 32) {
    const int bid = bids[s * g.n_s + v];
    const int bs = g.vbs[v];
    const cdouble* xb = x + g.voff[v] + (long long)bid * bs;
    const T* o = O + (s * g.n_s + v) * (long long)g.D4;
    P pr = P(0), pi = P(0);
#pragma unroll 4
    for (int e = 0; e < bs; ++e) {
      const T ov = o[e];
      const cdouble xv = xb[e];
      if (CPLX) {
        pr += (P)re(ov) * (P)xv.x - (P)im(ov) * (P)xv.y;
        pi += (P)re(ov) * (P)xv.y + (P)im(ov) * (P)xv.x;
      } else {
        pr += (P)re(ov) * (P)xv.x;
      }
    }
    ar += (double)pr;
    if (CPLX) ai += (double)pi;
  }
  ar = warp_sum(ar);
  if (CPLX) ai = warp_sum(ai);
  if (lane == 0) t[s] = {ar, CPLX ? ai : 0.0};
}

// The same product with each sample's O row (n_s x D4 storage scalars,
// contiguous) read by the whole warp in 16-byte vectors; needs D4 a multiple
// of VE = 16 / sizeof(T).  Per-vector partials in the storage precision,
// then FP64.
template <class T, bool CPLX>
__global__ void k_gather_vec(SrGeom g, const int* bids, const T* O, const cdouble* x, cdouble* t) {
  using P = typename PartialOf<T>::type;
  constexpr int VE = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= g.Ns) return;
  const int nvec = g.n_s * g.D4 / VE;
  const float4* row = reinterpret_cast<const float4*>(O + s * g.n_s * (long long)g.D4);
  const int* brow = bids + s * g.n_s;
  double ar = 0.0, ai = 0.0;
#pragma unroll 2
  for (int j = lane; j < nvec; j += 32) {
    const int el = j * VE, v = el / g.D4, e0 = el - v * g.D4;
    const int bs = g.vbs[v];
    if (e0 >= bs) continue;
    const float4 raw = row[j];
    const T* ov = reinterpret_cast<const T*>(&raw);
    const cdouble* xb = x + g.voff[v] + (long long)brow[v] * bs + e0;
    P pr = P(0), pi = P(0);
#pragma unroll
    for (int i = 0; i < VE; ++i) {
      if (e0 + i < bs) {
        const cdouble xv = xb[i];
        if (CPLX) {
          pr += (P)re(ov[i]) * (P)xv.x - (P)im(ov[i]) * (P)xv.y;
          pi += (P)re(ov[i]) * (P)xv.y + (P)im(ov[i]) * (P)xv.x;
        } else {
          pr += (P)re(ov[i]) * (P)xv.x;
        }
      }
    }
    ar += (double)pr;
    if (CPLX) ai += (double)pi;
  }
  ar = warp_sum(ar);
  if (CPLX) ai = warp_sum(ai);
  if (lane == 0) t[s] = {ar, CPLX ? ai : 0.0};
}

// k_gather_vec for real FP32 storage whose block sizes (hence vertex offsets)
// are multiples of 4, with D4 = 2^d4_shift: the direction x comes as its FP32
// copy xf and is read in 16-byte quads like O.  Same products, same order.
__global__ void k_gather_f4(SrGeom g, const int* bids, const float* O, const float* xf, int d4_shift,
                            cdouble* t) {
  const int lane = threadIdx.x & 31;
  const long long s = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (s >= g.Ns) return;
  const int nvec = (g.n_s * g.D4) >> 2;
  const float4* row = reinterpret_cast<const float4*>(O + s * g.n_s * (long long)g.D4);
  const int* brow = bids + s * g.n_s;
  double ar = 0.0;
#pragma unroll 2
  for (int j = lane; j < nvec; j += 32) {
    const int el = j << 2, v = el >> d4_shift, e0 = el - (v << d4_shift);
    const int bs = g.vbs[v];
    if (e0 >= bs) continue;
    const float4 o = row[j];
    const float4 xq = *reinterpret_cast<const float4*>(xf + g.voff[v] + (long long)brow[v] * bs + e0);
    float pr = 0.f;
    pr += o.x * xq.x;
    pr += o.y * xq.y;
    pr += o.z * xq.z;
    pr += o.w * xq.w;
    ar += (double)pr;
  }
  ar = warp_sum(ar);
  if (lane == 0) t[s] = {ar, 0.0};
}

// O in segment order: osort[Ns * pbs[v] + q * bs_v + e] = O[perm_v[q]][v][e].
// Grid (row chunks, vertices); consecutive threads write consecutive entries.
template <class T>
__global__ void k_permute_O(SrGeom g, const int* perm, const long long* pbs, const T* O, T* osort) {
  const int v = blockIdx.y;
  const int bs = g.vbs[v];
  const long long n = g.Ns * bs;
  const int* pv = perm + (long long)v * g.Ns;
  T* dst = osort + g.Ns * pbs[v];
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long q = i / bs;
    const int e = (int)(i - q * bs);
    dst[i] = O[((long long)pv[q] * g.n_s + v) * g.D4 + e];
  }
}

// out[off(v, b) + e] += sum_{s in segment (v, b)} coef_s op(O[s][v][e]) on
// the segment-ordered copy of O.  Grid = segments x split: CTA (segment,
// part) streams one contiguous part of its segment's rows (thread t keeps
// entry e = t % bs of rows t / bs, t / bs + rows-per-step, ...), sums in the
// storage precision in chunks of 32 rows, then FP64, and combines parts
// with FP64 atomics; coef is gathered through perm (it stays in L2).
// op = conj if CONJ, |.|^2 if SQ.
template <class T, bool CONJ, bool CPLX, bool SQ>
__global__ void k_scatter_sorted(SrGeom g, const int* perm, const int* seg, int maxnb, int split, const T* osort,
                                 const long long* pbs, const cdouble* coef, cdouble* out, const int* seg_v,
                                 const int* seg_b) {
  using P = typename PartialOf<T>::type;
  __shared__ double red[2 * 256];
  const int sid = blockIdx.x / split, part = blockIdx.x - (blockIdx.x / split) * split;
  const int v = seg_v[sid], b = seg_b[sid];
  const int bs = g.vbs[v];
  const int seg0 = seg[v * (maxnb + 1) + b], seg1 = seg[v * (maxnb + 1) + b + 1];
  const int len = seg1 - seg0;
  const int per = (len + split - 1) / split;
  const int s_begin = seg0 + part * per, s_end = min(seg1, s_begin + per);
  if (s_begin >= s_end) return;
  const int* pv = perm + (long long)v * g.Ns;
  const T* rows = osort + g.Ns * pbs[v];
  const int rps = max(1, (int)blockDim.x / bs);  // rows per step
  const int e = threadIdx.x % bs, rr = threadIdx.x / bs;
  double ar = 0.0, ai = 0.0;
  if (rr < rps) {
    int cnt = 0;
    P pr = P(0), pi = P(0);
#pragma unroll 4
    for (int q = s_begin + rr; q < s_end; q += rps) {
      const T ov = rows[(long long)q * bs + e];
      const cdouble c = coef[pv[q]];
      P orr = (P)re(ov), oi = CONJ ? -(P)im(ov) : (P)im(ov);
      if (SQ) {
        orr = orr * orr + oi * oi;
        oi = P(0);
      }
      if (CPLX && !SQ) {
        pr += (P)c.x * orr - (P)c.y * oi;
        pi += (P)c.x * oi + (P)c.y * orr;
      } else {
        pr += (P)c.x * orr;
      }
      if (++cnt == 32) {
        ar += (double)pr;
        ai += (double)pi;
        pr = P(0);
        pi = P(0);
        cnt = 0;
      }
    }
    ar += (double)pr;
    ai += (double)pi;
  }
  red[threadIdx.x] = ar;
  red[256 + threadIdx.x] = ai;
  __syncthreads();
  if (threadIdx.x < bs) {
    double sr = 0.0, si = 0.0;
    for (int q = 0; q < rps; ++q) {
      sr += red[q * bs + threadIdx.x];
      si += red[256 + q * bs + threadIdx.x];
    }
    cdouble* dst = out + g.voff[v] + (long long)b * bs + threadIdx.x;
    atomicAdd(&dst->x, sr);
    if (CPLX) atomicAdd(&dst->y, si);
  }
}

// Real FP32 storage with bs a multiple of 4: each thread takes a 16-byte
// quad (4 entries) of a row, and the coefficients come as the FP32 copy of
// their real parts (the values the products use); otherwise as
// k_scatter_sorted.
template <bool SQ>
__global__ void k_scatter_sorted_f4(SrGeom g, const int* perm, const int* seg, int maxnb, int split,
                                    const float* osort, const long long* pbs, const float* coef, cdouble* out,
                                    const int* seg_v, const int* seg_b) {
  __shared__ double red[256 * 4];
  const int sid = blockIdx.x / split, part = blockIdx.x - (blockIdx.x / split) * split;
  const int v = seg_v[sid], b = seg_b[sid];
  const int bs = g.vbs[v], nq = bs >> 2;
  const int seg0 = seg[v * (maxnb + 1) + b], seg1 = seg[v * (maxnb + 1) + b + 1];
  const int len = seg1 - seg0;
  const int per = (len + split - 1) / split;
  const int s_begin = seg0 + part * per, s_end = min(seg1, s_begin + per);
  if (s_begin >= s_end) return;
  const int* pv = perm + (long long)v * g.Ns;
  const float* rows = osort + g.Ns * pbs[v];
  const int rps = max(1, (int)blockDim.x / nq);  // rows per step
  const int qi = threadIdx.x % nq, rr = threadIdx.x / nq;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  if (rr < rps) {
    int cnt = 0;
    float part4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int q = s_begin + rr; q < s_end; q += rps) {
      const float4 o = *reinterpret_cast<const float4*>(rows + (long long)q * bs + 4 * qi);
      const float c = coef[pv[q]];
      if (SQ) {
        part4[0] += c * o.x * o.x; part4[1] += c * o.y * o.y;
        part4[2] += c * o.z * o.z; part4[3] += c * o.w * o.w;
      } else {
        part4[0] += c * o.x; part4[1] += c * o.y; part4[2] += c * o.z; part4[3] += c * o.w;
      }
      if (++cnt == 32) {
#pragma unroll
        for (int i = 0; i < 4; ++i) { acc[i] += (double)part4[i]; part4[i] = 0.f; }
        cnt = 0;
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] += (double)part4[i];
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) red[4 * threadIdx.x + i] = acc[i];
  __syncthreads();
  if (threadIdx.x < bs) {
    const int q4 = threadIdx.x >> 2, i = threadIdx.x & 3;
    double sr = 0.0;
    for (int r = 0; r < rps; ++r) sr += red[4 * (r * nq + q4) + i];
    atomicAdd(&(out + g.voff[v] + (long long)b * bs + threadIdx.x)->x, sr);
  }
}

__global__ void k_fill_c(cdouble* v, long long n, double r, double i) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[k] = {r, i};
}

__global__ void k_e_to_c(const double* e, long long n, cdouble* v) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[k] = {e[2 * k], e[2 * k + 1]};
}

__global__ void k_copy_scalar(double* sc) { sc[0] = sc[4]; sc[1] = sc[5]; }

// Jacobi preconditioner of S + shift: diag(S)_m = <|O_m|^2> - |<O_m>|^2
// (clamped at 0 against rounding); dinv = 1 / (diag + shift).
__global__ void k_jacobi(const cdouble* sq_mean, const cdouble* obar, double shift, double* dinv, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const double d = sq_mean[k].x - (obar[k].x * obar[k].x + obar[k].y * obar[k].y);
  dinv[k] = 1.0 / (fmax(d, 0.0) + shift);
}
__global__ void k_fill_d(double* v, long long n, double a) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) v[k] = a;
}
__global__ void k_precond(cdouble* z, const cdouble* r, const double* dinv, long long n) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  z[k].x = dinv[k] * r[k].x;
  z[k].y = dinv[k] * r[k].y;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

template <class T>
static cudaError_t scatter(const SrGeom& g, const SrWork& w, const T* O, const cdouble* coef,
                           cdouble* out, bool conj, cudaStream_t st, long long* launches, bool sq = false) {
  constexpr bool C = Traits<T>::cplx;
  // about 2048 samples per CTA: the average segment holds Ns * n_s / n_seg
  const long long per_seg = g.Ns * g.n_s / std::max(1, w.n_seg);
  const int split = (int)std::max<long long>(1, std::min<long long>(512, per_seg / 2048));
  const unsigned grid = (unsigned)(w.n_seg * split);
  const T* os = (const T*)w.osort;
  (void)O;
  if constexpr (std::is_same<T, float>::value) {
    if (w.all_bs4) {
      k_real_to_f32<<<nblk(g.Ns, 256), 256, 0, st>>>(coef, g.Ns, w.coef_f);
      if (sq)
        k_scatter_sorted_f4<true><<<grid, 256, 0, st>>>(g, w.perm, w.seg, w.maxnb, split, os, w.pbs, w.coef_f,
                                                         out, w.seg_v, w.seg_b);
      else
        k_scatter_sorted_f4<false><<<grid, 256, 0, st>>>(g, w.perm, w.seg, w.maxnb, split, os, w.pbs, w.coef_f,
                                                          out, w.seg_v, w.seg_b);
      *launches += 2;
      return cudaGetLastError();
    }
  }
  if (sq)
    k_scatter_sorted<T, false, C, true><<<grid, 256, 0, st>>>(g, w.perm, w.seg, w.maxnb, split, os, w.pbs, coef,
                                                               out, w.seg_v, w.seg_b);
  else if (conj)
    k_scatter_sorted<T, true, C, false><<<grid, 256, 0, st>>>(g, w.perm, w.seg, w.maxnb, split, os, w.pbs, coef,
                                                               out, w.seg_v, w.seg_b);
  else
    k_scatter_sorted<T, false, C, false><<<grid, 256, 0, st>>>(g, w.perm, w.seg, w.maxnb, split, os, w.pbs, coef,
                                                                out, w.seg_v, w.seg_b);
  ++*launches;
  return cudaGetLastError();
}

template <class T>
static cudaError_t dot(const cdouble* a, const cdouble* b, long long n, double* out, cudaStream_t st,
                       long long* launches) {
  cudaError_t err = cudaMemsetAsync(out, 0, 2 * sizeof(double), st);
  if (err != cudaSuccess) return err;
  const int grid = (int)std::min<long long>(nblk(n, 256), 1024);
  k_dot<<<grid, 256, 0, st>>>(a, b, n, out);
  ++*launches;
  return cudaGetLastError();
}

template <class T>
cudaError_t sr_solve_update(const SrGeom& g, SrWork& w, const double* e_loc, const int* bids,
                            const void* Ov, void* params, int n_chains, double shift, double cr,
                            double ci, int max_iter, double tol, double* stats, cudaStream_t st,
                            long long* launches) {
  const T* O = (const T*)Ov;
  const long long Np = g.Np, Ns = g.Ns;
  // 16-byte vector reads of O need a 16-byte aligned base and whole vectors per vertex
  const bool vec_ok = (reinterpret_cast<uintptr_t>(Ov) % 16 == 0) && (g.D4 % (16 / (int)sizeof(T)) == 0);
  // log2(D4) when D4 is a power of two (D_k = 2: 16), else -1
  int d4_shift = -1;
  for (int sh = 0; sh < 31; ++sh)
    if ((1 << sh) == g.D4) d4_shift = sh;
  cudaError_t err;
#define CK(x)                                   \
  do {                                          \
    if ((err = (x)) != cudaSuccess) return err; \
  } while (0)
  // energy mean and error bar (over chain means, or over samples for one chain)
  if (n_chains > 1) {
    k_chain_means<<<n_chains, 256, 0, st>>>(e_loc, (int)(Ns / n_chains), w.chain_mean);
    ++*launches;
    k_mean_err<<<1, 1024, 0, st>>>(w.chain_mean, n_chains, w.scal);
  } else {
    k_e_to_c<<<nblk(Ns, 256), 256, 0, st>>>(e_loc, Ns, w.coef);
    ++*launches;
    k_mean_err<<<1, 1024, 0, st>>>(w.coef, (int)Ns, w.scal);
  }
  ++*launches;
  CK(cudaGetLastError());
  // samples grouped by (vertex, block) for the atomic-free scatter
  k_sort_by_block<<<g.n_s, 1024, 0, st>>>(g, bids, w.maxnb, w.perm, w.seg);
  ++*launches;
  // O in segment order, streamed by every scatter of this step
  {
    dim3 grid((unsigned)std::min<long long>(1024, (Ns * 16 + 255) / 256), (unsigned)g.n_s);
    k_permute_O<T><<<grid, 256, 0, st>>>(g, w.perm, w.pbs, O, (T*)w.osort);
    ++*launches;
  }
  // Obar = (1/Ns) sum_s O_s
  CK(cudaMemsetAsync(w.obar, 0, sizeof(cdouble) * Np, st));
  k_fill_c<<<nblk(Ns, 256), 256, 0, st>>>(w.coef, Ns, 1.0 / (double)Ns, 0.0);
  ++*launches;
  CK(scatter<T>(g, w, O, w.coef, w.obar, false, st, launches));
  // F = (1/Ns) sum_s conj(O_s) (E_s - Ebar)
  k_f_coef<<<nblk(Ns, 256), 256, 0, st>>>(e_loc, Ns, w.scal, w.coef);
  ++*launches;
  CK(cudaMemsetAsync(w.F, 0, sizeof(cdouble) * Np, st));
  CK(scatter<T>(g, w, O, w.coef, w.F, true, st, launches));
  // Preconditioner.  With Ns < Np, S has rank < Ns and S + shift is a
  // low-rank matrix plus a multiple of the identity: plain CG ends in about Ns
  // iterations, and a diagonal preconditioner would destroy that structure.
  // With Ns >= Np (S full rank) the Jacobi preconditioner
  // dinv = 1 / (<|O|^2> - |Obar|^2 + shift) evens out the per-parameter scales.
  const bool jacobi = Ns >= Np;
  if (jacobi) {
    CK(cudaMemsetAsync(w.Ap, 0, sizeof(cdouble) * Np, st));
    k_fill_c<<<nblk(Ns, 256), 256, 0, st>>>(w.t, Ns, 1.0 / (double)Ns, 0.0);
    ++*launches;
    CK(scatter<T>(g, w, O, w.t, w.Ap, false, st, launches, true));
    k_jacobi<<<nblk(Np, 256), 256, 0, st>>>(w.Ap, w.obar, shift, w.dinv, Np);
  } else {
    k_fill_d<<<nblk(Np, 256), 256, 0, st>>>(w.dinv, Np, 1.0);
  }
  ++*launches;
  // preconditioned CG: x = 0, r = F, z = M^-1 r, p = z
  double* sc = w.scal + 8;  // sc[0..1] rz, sc[2..3] pAp, sc[4..5] rz_new, sc[6..7] rr
  CK(cudaMemsetAsync(w.x, 0, sizeof(cdouble) * Np, st));
  CK(cudaMemcpyAsync(w.r, w.F, sizeof(cdouble) * Np, cudaMemcpyDeviceToDevice, st));
  k_precond<<<nblk(Np, 256), 256, 0, st>>>(w.z, w.r, w.dinv, Np);
  ++*launches;
  CK(cudaMemcpyAsync(w.p, w.z, sizeof(cdouble) * Np, cudaMemcpyDeviceToDevice, st));
  CK(dot<T>(w.r, w.z, Np, sc, st, launches));
  CK(dot<T>(w.r, w.r, Np, sc + 6, st, launches));
  double h_sc[16];
  CK(cudaMemcpyAsync(h_sc, w.scal, 16 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  const double e_re = h_sc[0], e_im = h_sc[1], e_err = h_sc[2];
  const double rr0 = h_sc[8 + 6];
  const double fnorm = sqrt(rr0);
  double rr = rr0;
  int it = 0;
  bool converged = !(fnorm > 0.0);
  while (!converged && it < max_iter) {
    // Ap = S p + shift p
    bool quad = false;
    if constexpr (std::is_same<T, float>::value) {
      if (vec_ok && w.all_bs4 && d4_shift >= 2) {
        k_real_to_f32<<<nblk(Np, 256), 256, 0, st>>>(w.p, Np, w.xf);
        k_gather_f4<<<nblk(Ns * 32, 256), 256, 0, st>>>(g, bids, O, w.xf, d4_shift, w.t);
        *launches += 2;
        quad = true;
      }
    }
    if (!quad) {
      if (vec_ok)
        k_gather_vec<T, Traits<T>::cplx><<<nblk(Ns * 32, 256), 256, 0, st>>>(g, bids, O, w.p, w.t);
      else
        k_gather2<T, Traits<T>::cplx><<<nblk(Ns * 32, 256), 256, 0, st>>>(g, bids, O, w.p, w.t);
      ++*launches;
    }
    k_sum_c_part<<<kSumParts, 256, 0, st>>>(w.t, Ns, w.part);
    k_sum_c<<<1, 1024, 0, st>>>(w.part, kSumParts, w.tbar, 1.0 / (double)Ns);
    *launches += 2;
    k_center<<<nblk(Ns, 256), 256, 0, st>>>(w.t, Ns, w.tbar);
    ++*launches;
    CK(cudaMemsetAsync(w.Ap, 0, sizeof(cdouble) * Np, st));
    CK(scatter<T>(g, w, O, w.t, w.Ap, true, st, launches));
    k_axpy_real<<<nblk(Np, 256), 256, 0, st>>>(w.Ap, w.p, shift, Np);
    ++*launches;
    CK(dot<T>(w.p, w.Ap, Np, sc + 2, st, launches));
    k_cg_xr<<<nblk(Np, 256), 256, 0, st>>>(w.x, w.r, w.p, w.Ap, sc, Np);
    ++*launches;
    k_precond<<<nblk(Np, 256), 256, 0, st>>>(w.z, w.r, w.dinv, Np);
    ++*launches;
    CK(dot<T>(w.r, w.z, Np, sc + 4, st, launches));
    CK(dot<T>(w.r, w.r, Np, sc + 6, st, launches));
    k_cg_p<<<nblk(Np, 256), 256, 0, st>>>(w.p, w.z, sc, Np);
    ++*launches;
    k_copy_scalar<<<1, 1, 0, st>>>(sc);
    ++*launches;
    double rn;
    CK(cudaMemcpyAsync(&rn, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    rr = rn;
    ++it;
    if (sqrt(rr) <= tol * fnorm) converged = true;
  }
  CK(cudaGetLastError());
  k_update<T><<<nblk(Np, 256), 256, 0, st>>>((T*)params, w.x, cr, ci, Np);
  ++*launches;
  CK(cudaGetLastError());
  stats[0] = e_re;
  stats[1] = e_im;
  stats[2] = e_err;
  stats[3] = (double)it;
  stats[4] = fnorm > 0.0 ? sqrt(rr) / fnorm : 0.0;
  stats[5] = fnorm;
  stats[6] = converged ? 1.0 : 0.0;
  stats[7] = jacobi ? 1.0 : 0.0;
  return cudaSuccess;
#undef CK
}

// ---------------------------------------------------------------------------
// Vector-Jacobian product of the log-amplitudes (the adjoint of Eq. S3 per
// sample): grad = sum_s w_s d ln psi(s) / d theta, gathered from the sparse
// per-sample blocks O_s.
__global__ void k_weights_to_c(const double* w, int cplx, long long n, cdouble* c) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) c[s] = cplx ? cdouble{w[2 * s], w[2 * s + 1]} : cdouble{w[s], 0.0};
}
__global__ void k_c_to_grad(const cdouble* a, int cplx, long long np, double* grad) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  if (cplx) {
    grad[2 * i] = a[i].x;
    grad[2 * i + 1] = a[i].y;
  } else {
    grad[i] = a[i].x;
  }
}

template <class T>
cudaError_t log_grad_vjp(const SrGeom& g, const int* bids, const void* O, const double* w, int cplx,
                         cdouble* coef, cdouble* acc, double* grad, cudaStream_t st, long long* launches) {
  const int chunk = 64;
  const size_t smem = 2 * sizeof(double) * (size_t)g.max_nb_bs;
  cudaError_t e = cudaFuncSetAttribute(k_scatter<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_weights_to_c<<<(unsigned)((g.Ns + 255) / 256), 256, 0, st>>>(w, cplx, g.Ns, coef);
  e = cudaMemsetAsync(acc, 0, sizeof(cdouble) * g.Np, st);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((g.Ns + chunk - 1) / chunk), (unsigned)g.n_s);
  k_scatter<T, false><<<grid, 256, smem, st>>>(g, bids, (const T*)O, coef, acc, chunk);
  k_c_to_grad<<<(unsigned)((g.Np + 255) / 256), 256, 0, st>>>(acc, cplx, g.Np, grad);
  *launches += 3;
  return cudaGetLastError();
}

template cudaError_t log_grad_vjp<float>(const SrGeom&, const int*, const void*, const double*, int, cdouble*,
                                         cdouble*, double*, cudaStream_t, long long*);
template cudaError_t log_grad_vjp<double>(const SrGeom&, const int*, const void*, const double*, int, cdouble*,
                                          cdouble*, double*, cudaStream_t, long long*);
template cudaError_t log_grad_vjp<cfloat>(const SrGeom&, const int*, const void*, const double*, int, cdouble*,
                                          cdouble*, double*, cudaStream_t, long long*);
template cudaError_t log_grad_vjp<cdouble>(const SrGeom&, const int*, const void*, const double*, int, cdouble*,
                                           cdouble*, double*, cudaStream_t, long long*);

template cudaError_t sr_solve_update<float>(const SrGeom&, SrWork&, const double*, const int*,
                                            const void*, void*, int, double, double, double, int,
                                            double, double*, cudaStream_t, long long*);
template cudaError_t sr_solve_update<double>(const SrGeom&, SrWork&, const double*, const int*,
                                             const void*, void*, int, double, double, double, int,
                                             double, double*, cudaStream_t, long long*);
template cudaError_t sr_solve_update<cfloat>(const SrGeom&, SrWork&, const double*, const int*,
                                             const void*, void*, int, double, double, double, int,
                                             double, double*, cudaStream_t, long long*);
template cudaError_t sr_solve_update<cdouble>(const SrGeom&, SrWork&, const double*, const int*,
                                              const void*, void*, int, double, double, double, int,
                                              double, double*, cudaStream_t, long long*);

}  // namespace gcf
