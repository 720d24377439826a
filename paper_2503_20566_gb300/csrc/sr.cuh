// FP64 stochastic-reconfiguration / tVMC solve (declarations).
#pragma once

#include <algorithm>

#include "common.cuh"

namespace gcf {

struct SrGeom {
  long long Np;        // number of parameters
  long long Ns;        // number of samples
  int n_s;             // vertices
  int D4;              // O slot per vertex (D_k^4)
  const long long* voff;  // device [n_s]
  const int* vbs;         // device [n_s] block size
  const int* vnb;         // device [n_s] number of blocks
  int max_nb_bs;          // max_v nb*bs
};

// blocks of the first stage of a sample sum (two per SM of a 152-SM GPU)
constexpr int kSumParts = 304;

struct SrWork {
  cdouble *obar, *F, *x, *r, *p, *Ap;  // [Np]
  cdouble* z;                          // [Np] preconditioned residual
  double* dinv;                        // [Np] inverse Jacobi preconditioner
  cdouble *t, *coef;                   // [Ns]
  cdouble *chain_mean;                 // [n_chains]
  cdouble *tbar;                       // [1]
  double* scal;                        // [16] device scalars
  // sample order grouped by (vertex, block)
  int* perm;      // [n_s * Ns]
  int* seg;       // [n_s * (maxnb + 1)]
  int* seg_v;     // [n_seg] vertex of segment
  int* seg_b;     // [n_seg] block of segment
  int maxnb, n_seg;
  // O in segment order: vertex v's rows (bs_v entries each, samples in perm
  // order) start at element Ns * pbs[v]
  long long* pbs;  // [n_s] prefix sums of the block sizes
  void* osort;     // [Ns * sum_v bs_v] storage scalars
  int all_bs4;     // every block size is a multiple of 4
  // FP32 copies for the real FP32 storage kernels
  float* xf;       // [Np] CG direction
  float* coef_f;   // [Ns] scatter coefficients
  cdouble* part;   // [kSumParts] first-stage partial sums
};

// Computes <E>, F, solves (S + shift) x = F by CG, then params += (cr + i ci) x.
// stats[8] as documented for gcf_sr_step.
template <class T>
cudaError_t sr_solve_update(const SrGeom& g, SrWork& w, const double* e_loc, const int* bids,
                            const void* O, void* params, int n_chains, double shift, double cr,
                            double ci, int max_iter, double tol, double* stats, cudaStream_t st,
                            long long* launches);

// grad = sum_s w_s O_s scattered into the parameter layout (real: grad[Np],
// complex: grad[2 Np] interleaved; w real [Ns] or complex [2 Ns]).  coef [Ns]
// and acc [Np] are work buffers.
template <class T>
cudaError_t log_grad_vjp(const SrGeom& g, const int* bids, const void* O, const double* w, int cplx,
                         cdouble* coef, cdouble* acc, double* grad, cudaStream_t st, long long* launches);

}  // namespace gcf
