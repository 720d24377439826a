// Scalar types, complex arithmetic and CTA-wide helpers shared by the
// GB300 kernels of the GCF-PEPS VMC library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#include <type_traits>

namespace gcf {

struct cfloat { float x, y; };
struct cdouble { double x, y; };

// ---- scalar traits -----------------------------------------------------
template <class T> struct Traits;
template <> struct Traits<float> {
  using R = float; static constexpr bool cplx = false;
  __host__ __device__ static constexpr float eps() { return 1.1920929e-07f; }
};
template <> struct Traits<double> {
  using R = double; static constexpr bool cplx = false;
  __host__ __device__ static constexpr double eps() { return 2.220446049250313e-16; }
};
template <> struct Traits<cfloat> {
  using R = float; static constexpr bool cplx = true;
  __host__ __device__ static constexpr float eps() { return 1.1920929e-07f; }
};
template <> struct Traits<cdouble> {
  using R = double; static constexpr bool cplx = true;
  __host__ __device__ static constexpr double eps() { return 2.220446049250313e-16; }
};

// ---- arithmetic (real overloads are the identity where appropriate) ------
__host__ __device__ inline float zero_of(float) { return 0.f; }
__host__ __device__ inline double zero_of(double) { return 0.0; }
__host__ __device__ inline cfloat zero_of(cfloat) { return {0.f, 0.f}; }
__host__ __device__ inline cdouble zero_of(cdouble) { return {0.0, 0.0}; }
template <class T> __host__ __device__ inline T zero() { return zero_of(T()); }

__host__ __device__ inline float one_of(float) { return 1.f; }
__host__ __device__ inline double one_of(double) { return 1.0; }
__host__ __device__ inline cfloat one_of(cfloat) { return {1.f, 0.f}; }
__host__ __device__ inline cdouble one_of(cdouble) { return {1.0, 0.0}; }
template <class T> __host__ __device__ inline T one() { return one_of(T()); }

__host__ __device__ inline float conjg(float a) { return a; }
__host__ __device__ inline double conjg(double a) { return a; }
__host__ __device__ inline cfloat conjg(cfloat a) { return {a.x, -a.y}; }
__host__ __device__ inline cdouble conjg(cdouble a) { return {a.x, -a.y}; }

__host__ __device__ inline float re(float a) { return a; }
__host__ __device__ inline double re(double a) { return a; }
__host__ __device__ inline float re(cfloat a) { return a.x; }
__host__ __device__ inline double re(cdouble a) { return a.x; }
__host__ __device__ inline float im(float) { return 0.f; }
__host__ __device__ inline double im(double) { return 0.0; }
__host__ __device__ inline float im(cfloat a) { return a.y; }
__host__ __device__ inline double im(cdouble a) { return a.y; }

__host__ __device__ inline float abs2(float a) { return a * a; }
__host__ __device__ inline double abs2(double a) { return a * a; }
__host__ __device__ inline float abs2(cfloat a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline double abs2(cdouble a) { return a.x * a.x + a.y * a.y; }

__host__ __device__ inline float absmax1(float a) { return fabsf(a); }
__host__ __device__ inline double absmax1(double a) { return fabs(a); }
__host__ __device__ inline float absmax1(cfloat a) { return fmaxf(fabsf(a.x), fabsf(a.y)); }
__host__ __device__ inline double absmax1(cdouble a) { return fmax(fabs(a.x), fabs(a.y)); }

__host__ __device__ inline cfloat operator+(cfloat a, cfloat b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cdouble operator+(cdouble a, cdouble b) { return {a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cfloat operator-(cfloat a, cfloat b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cdouble operator-(cdouble a, cdouble b) { return {a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cfloat operator-(cfloat a) { return {-a.x, -a.y}; }
__host__ __device__ inline cdouble operator-(cdouble a) { return {-a.x, -a.y}; }
__host__ __device__ inline cfloat operator*(cfloat a, cfloat b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline cdouble operator*(cdouble a, cdouble b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline cfloat operator*(cfloat a, float s) { return {a.x * s, a.y * s}; }
__host__ __device__ inline cdouble operator*(cdouble a, double s) { return {a.x * s, a.y * s}; }
__host__ __device__ inline cfloat& operator+=(cfloat& a, cfloat b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ inline cdouble& operator+=(cdouble& a, cdouble b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ inline cfloat& operator-=(cfloat& a, cfloat b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ inline cdouble& operator-=(cdouble& a, cdouble b) { a.x -= b.x; a.y -= b.y; return a; }

// fused multiply-add acc + a*b
__device__ inline float fmac(float acc, float a, float b) { return fmaf(a, b, acc); }
__device__ inline double fmac(double acc, double a, double b) { return fma(a, b, acc); }
__device__ inline cfloat fmac(cfloat acc, cfloat a, cfloat b) {
  acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
  acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
  return acc;
}
__device__ inline cdouble fmac(cdouble acc, cdouble a, cdouble b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
  return acc;
}

__host__ __device__ inline float scale(float a, float s) { return a * s; }
__host__ __device__ inline double scale(double a, double s) { return a * s; }
__host__ __device__ inline cfloat scale(cfloat a, float s) { return {a.x * s, a.y * s}; }
__host__ __device__ inline cdouble scale(cdouble a, double s) { return {a.x * s, a.y * s}; }

// make_scalar<T>(re, im): the argument type is deduced so that float
// arguments never pass through double.
template <class T> struct MakeS;
template <> struct MakeS<float> {
  template <class A> __host__ __device__ static float f(A r, A) { return (float)r; }
};
template <> struct MakeS<double> {
  template <class A> __host__ __device__ static double f(A r, A) { return (double)r; }
};
template <> struct MakeS<cfloat> {
  template <class A> __host__ __device__ static cfloat f(A r, A i) { return {(float)r, (float)i}; }
};
template <> struct MakeS<cdouble> {
  template <class A> __host__ __device__ static cdouble f(A r, A i) { return {(double)r, (double)i}; }
};
template <class T, class A>
__host__ __device__ inline T make_scalar(A r, A i) { return MakeS<T>::f(r, i); }

// complex division a / b (b != 0)
__device__ inline float cdiv(float a, float b) { return a / b; }
__device__ inline double cdiv(double a, double b) { return a / b; }
__device__ inline cfloat cdiv(cfloat a, cfloat b) {
  float d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__device__ inline cdouble cdiv(cdouble a, cdouble b) {
  double d = b.x * b.x + b.y * b.y;
  return {(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// ---- CTA reductions (all threads must call; result broadcast) -----------
// `red` is shared scratch of at least 32 doubles.
template <class R>
__device__ inline R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <class R>
__device__ inline R warp_max(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

template <class T>
__device__ inline T warp_sum_scalar(T v);
template <>
__device__ inline float warp_sum_scalar<float>(float v) { return warp_sum(v); }
template <>
__device__ inline double warp_sum_scalar<double>(double v) { return warp_sum(v); }
template <>
__device__ inline cfloat warp_sum_scalar<cfloat>(cfloat v) { return {warp_sum(v.x), warp_sum(v.y)}; }
template <>
__device__ inline cdouble warp_sum_scalar<cdouble>(cdouble v) { return {warp_sum(v.x), warp_sum(v.y)}; }

__device__ inline double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  if (wid == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

__device__ inline double block_max(double v, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double t = (threadIdx.x < nw) ? red[threadIdx.x] : -1.0;
  if (wid == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  double r = red[0];
  __syncthreads();
  return r;
}

// complex sum: two doubles
__device__ inline void block_sum2(double& a, double& b, double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a); b = warp_sum(b);
  __syncthreads();
  if (lane == 0) { red[wid] = a; red[32 + wid] = b; }
  __syncthreads();
  double ta = (threadIdx.x < nw) ? red[threadIdx.x] : 0.0;
  double tb = (threadIdx.x < nw) ? red[32 + threadIdx.x] : 0.0;
  if (wid == 0) { ta = warp_sum(ta); tb = warp_sum(tb); }
  if (threadIdx.x == 0) { red[0] = ta; red[32] = tb; }
  __syncthreads();
  a = red[0]; b = red[32];
  __syncthreads();
}

// Block-wide sums in the real type R of the scalar (float for the FP32
// forms: GB300's FP64 pipe is ~1/64 of FP32, so FP64 stays out of hot loops).
// red: shared scratch of >= 64 R values.  All threads call; result broadcast.
template <class R>
__device__ inline R block_sum_r(R v, R* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  R t = (lane < nw) ? red[lane] : R(0);
  t = warp_sum(t);
  __syncthreads();
  return t;
}
template <class R>
__device__ inline void block_sum2_r(R& a, R& b, R* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  __syncthreads();
  if (lane == 0) { red[wid] = a; red[32 + wid] = b; }
  __syncthreads();
  R ta = (lane < nw) ? red[lane] : R(0);
  R tb = (lane < nw) ? red[32 + lane] : R(0);
  a = warp_sum(ta);
  b = warp_sum(tb);
  __syncthreads();
}

// Execution groups.  Every cooperative routine is written once against an
// executor: CtaExec (the whole CTA works on one chain, __syncthreads),
// or GroupExec<G> (chains on groups of G threads, a hardware barrier per
// group).
// Executors hold no data, so passing them costs no registers; reductions use
// one 64-double slot per group of this CTA-wide array.
__shared__ double g_exec_red[4][64];
// Arithmetic of the contraction GEMMs of each group (a GemmMode of mma.cuh),
// set at kernel entry from the launch parameters; a chain may switch its
// own slot between passes.
__shared__ int g_gemm_mode[4];

struct CtaExec {
  __device__ int tid() const { return threadIdx.x; }
  __device__ int size() const { return blockDim.x; }
  __device__ int lane() const { return threadIdx.x & 31; }
  __device__ int warp() const { return threadIdx.x >> 5; }
  __device__ int nwarps() const { return blockDim.x >> 5; }
  __device__ bool leader() const { return threadIdx.x == 0; }
  __device__ void sync() const { __syncthreads(); }
  __device__ int slot() const { return 0; }
  template <class R> __device__ R sum(R v) const { return block_sum_r<R>(v, (R*)g_exec_red[0]); }
  template <class R> __device__ void sum2(R& a, R& b) const { block_sum2_r<R>(a, b, (R*)g_exec_red[0]); }
  __device__ float maxf(float v) const {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_max(v);
    float* r = (float*)g_exec_red[0];
    if (lane == 0) r[wid] = v;
    __syncthreads();
    float t = (lane < nw) ? r[lane] : 0.f;
    t = warp_max(t);
    __syncthreads();
    return t;
  }
};

template <int G>
struct GroupExec {
  static_assert(G % 32 == 0 && G >= 64 && G <= 128, "group of 64 or 128 threads");
  __device__ int group() const { return threadIdx.x / G; }
  __device__ int slot() const { return threadIdx.x / G; }
  __device__ int tid() const { return threadIdx.x % G; }
  __device__ int size() const { return G; }
  __device__ int lane() const { return threadIdx.x & 31; }
  __device__ int warp() const { return (threadIdx.x % G) >> 5; }
  __device__ int nwarps() const { return G >> 5; }
  __device__ bool leader() const { return threadIdx.x % G == 0; }
  __device__ void sync() const { asm volatile("bar.sync %0, %1;" ::"r"(1 + group()), "n"(G) : "memory"); }
  template <class R> __device__ R sum(R v) const {
    R* r = (R*)g_exec_red[group()];
    const int l = lane(), w = warp();
    v = warp_sum(v);
    if (l == 0) r[w] = v;
    sync();
    R t = (l < G / 32) ? r[l] : R(0);
    t = warp_sum(t);
    sync();
    return t;
  }
  template <class R> __device__ void sum2(R& a, R& b) const {
    R* r = (R*)g_exec_red[group()];
    const int l = lane(), w = warp();
    a = warp_sum(a);
    b = warp_sum(b);
    if (l == 0) { r[w] = a; r[32 + w] = b; }
    sync();
    a = (l < G / 32) ? r[l] : R(0);
    b = (l < G / 32) ? r[32 + l] : R(0);
    a = warp_sum(a);
    b = warp_sum(b);
    sync();
  }
  __device__ float maxf(float v) const {
    float* r = (float*)g_exec_red[group()];
    const int l = lane(), w = warp();
    v = warp_max(v);
    if (l == 0) r[w] = v;
    sync();
    float t = (l < G / 32) ? r[l] : 0.f;
    t = warp_max(t);
    sync();
    return t;
  }
};


// Streaming store of an output the kernel never reads back (evict-first in
// L2, so that the chains' scratch stays resident instead).
__device__ __forceinline__ void store_stream(float* p, float v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(double* p, double v) { __stcs(p, v); }
__device__ __forceinline__ void store_stream(cfloat* p, cfloat v) { __stcs((float2*)p, make_float2(v.x, v.y)); }
__device__ __forceinline__ void store_stream(cdouble* p, cdouble v) { __stcs((double2*)p, make_double2(v.x, v.y)); }
__device__ __forceinline__ void store_stream(int* p, int v) { __stcs(p, v); }

// Power-of-two scaling: the exponent e with m = f 2^e, f in [0.5, 1).
// Scaling by 2^-e is exact, so log-scales are integers (units of ln 2).
__device__ inline int exp2_of(float m) {
  int e;
  frexpf(m, &e);
  return e;
}
__device__ inline float pow2f(int e) { return ldexpf(1.0f, e); }
__device__ inline double pow2d(int e) { return ldexp(1.0, e); }
// 2^e built from its IEEE-754 binary64 fields (biased exponent e + 1023, zero
// fraction) for normal e; ldexp outside that range.
__device__ inline double pow2d_exact(int e) {
  if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
  return ldexp(1.0, e);
}
template <class R> __device__ inline R pow2r(int e);
template <> __device__ inline float pow2r<float>(int e) { return ldexpf(1.0f, e); }
template <> __device__ inline double pow2r<double>(int e) { return ldexp(1.0, e); }

// ---- SplitMix64 counter generator (Steele, Lea & Flood 2014) -------------
__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;
__host__ __device__ inline uint64_t stream_key(uint64_t seed, uint64_t stream) {
  return mix64(seed + (stream + 1) * kGamma);
}
__host__ __device__ inline uint64_t stream_word(uint64_t key, uint64_t counter) {
  return mix64(key + (counter + 1) * kGamma);
}
__host__ __device__ inline double word_to_uniform(uint64_t w) {
  return (double)(w >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace gcf
