// C ABI of libgcfvmc: context management, the host planner (layout, bond
// dimension tables, scratch plan) and the entry points declared in
// include/gcfvmc.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gcfvmc.h"
#include "launch.h"
#include "peps_dev.cuh"
#include "sr.cuh"

using namespace gcf;

namespace {

enum ScalarKind { S_F32 = 0, S_F64 = 1, S_C64 = 2, S_C128 = 3 };

struct Plan {
  std::vector<int> bondB, bondT, qrB, svdB, qrT, svdT;  // (Ly+1) x (Lx+1) each
  long long mps_stride = 0, qsite_stride = 0, mat_max = 0, tau_max = 0, tmp_max = 0;
  int env_stride = 0, env3_stride = 0;
  long long ws_stride = 0;
  int ck_every = 0;               // boundary-MPS store: keep every K-th (0: all)
  long long o_Bseg = 0, o_Tseg = 0;
  long long o_net, o_prop, o_B, o_T, o_Q, o_M1, o_M2, o_M3, o_tau, o_J, o_envR, o_envL, o_envX,
      o_envY, o_t1, o_t2, o_t3, o_env3R, o_env3L, o_env3X, o_env3Y, o_G;
  // buffers in dynamic shared memory (elements from the hot base)
  long long o_sigma = 0, o_sel = 0;
  long long so_envR = 0, so_env3R = 0, so_sB = 0, so_sT = 0;
  long long o_Z = 0, z_size = 0, q_pack = 0, o_X = 0, o_W1 = 0, o_W2 = 0, o_W3 = 0, o_W4 = 0;
  long long so_net, so_prop, so_cop, so_envL, so_envX, so_envY, so_env3L, so_env3X, so_env3Y, so_t1,
      so_t2, hot_elems = 0, cfg_bytes = 0;
  size_t dyn_smem = 0;
  // shared-memory placement levels of the two kernel forms (see plan_group)
  long long hot_base_elems = 0, hot_mps_elems = 0, hot_all_elems = 0;
  int cta_level = 0, group_level = 0;
  size_t group_smem = 0;
  // BF16 form of real chains: bytes of the tcgen05 operand staging area of
  // one chain (0: the tensor-core GEMMs of that form stay on mma.sync)
  long long tc_bytes = 0;
  // shared-memory factorisation workspace of one chain (scalars; 0: none)
  long long fz_elems = 0;
  long long level_elems(int lv) const {
    return lv <= 0 ? 0 : lv == 1 ? hot_base_elems : lv == 2 ? hot_mps_elems : hot_all_elems;
  }
};

}  // namespace

struct gcf_ctx {
  gcf_model m{};
  std::vector<int> Q;
  int Dk = 0, P = 1, n_h = 0, n_v = 0, n_s = 0, cfg_len = 0, n_plaq = 0, n_slots = 0;
  long long n_params = 0;
  std::vector<long long> voff;
  std::vector<int> vbs, vnb;
  int kind = S_F32;
  size_t sbytes = 4;
  cudaStream_t stream = nullptr;
  int device = 0, sms = 0;
  Plan plan;
  int exec = 0, group_threads = 64;
  int lockstep = 0;  // grouped kernels: chain groups of a CTA in lockstep
  int ck_every = 0;  // boundary-MPS store: keep every K-th slot and recompute between (0: keep all)
  int lock_fault = 0;  // test hook (GCFVMC_LOCK_FAULT): one group never counts in
  int last_phase_timeouts = 0;
  int last_svd_unconverged = 0;  // SVDs that hit the sweep limit in the last synchronous launch
  int last_tc_timeouts = 0;      // tensor-core waits that ran out in the last synchronous launch
  int last_multi_block = 0;      // block size of the last gcf_sample_multi launch (256 or 512)
  int svd_sweeps = 40;           // sweep limit of the one-sided Jacobi SVD
  int tab_ints = 0;  // ints in d_tables
  // device
  void* d_params = nullptr;
  int* d_Q = nullptr;
  long long* d_voff = nullptr;
  int* d_vbs = nullptr;
  int* d_vnb = nullptr;
  int* d_tables = nullptr;
  int* d_status = nullptr;
  void* d_scratch = nullptr;
  long long scratch_ctas = 0;
  // SR work
  SrWork sr{};
  long long sr_ns_cap = 0;
  long long sr_sum_bs = 0;
  int sr_chain_cap = 0;
  // e2e sample buffers
  int8_t* d_cfg = nullptr;
  double* d_e = nullptr;
  double* d_la = nullptr;
  double* d_ph = nullptr;
  int* d_bid = nullptr;
  void* d_O = nullptr;
  int* d_acc = nullptr;
  long long e2e_cap = 0;
  // gcf_log_grad_vjp work buffers
  int* vjp_bid = nullptr;
  void* vjp_O = nullptr;
  cdouble* vjp_coef = nullptr;
  cdouble* vjp_acc = nullptr;
  long long vjp_cap = 0;
  // gcf_sample_multi: scratch arena and launch tables (owned by the first
  // context of the call)
  void* multi_arena = nullptr;
  size_t multi_arena_bytes = 0;
  void* multi_tab = nullptr;
  size_t multi_tab_bytes = 0;
  int e2e_chains = 0;
  long long launches = 0;
  std::string err;
};

namespace {

gcf_status fail(gcf_ctx* c, gcf_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

gcf_status cuda_fail(gcf_ctx* c, cudaError_t e, const char* where) {
  return fail(c, GCF_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CUDA_TRY(ctx, expr)                                      \
  do {                                                           \
    cudaError_t _e = (expr);                                     \
    if (_e != cudaSuccess) return cuda_fail((ctx), _e, #expr);   \
  } while (0)

// Every entry point that touches the context's device memory runs with the
// context's device current: a launch with another device current would run
// there and dereference this context's buffers on the wrong GPU.
gcf_status check_device(gcf_ctx* c, const char* what) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  if (dev != c->device)
    return fail(c, GCF_EINVAL, std::string(what) + ": the context's device (" + std::to_string(c->device) +
                                   ") must be current, device " + std::to_string(dev) + " is");
  return GCF_OK;
}

#define DEVICE_TRY(ctx, what)                                    \
  do {                                                           \
    gcf_status _s = check_device((ctx), (what));                 \
    if (_s != GCF_OK) return _s;                                 \
  } while (0)

// A synchronous launch in which some one-sided Jacobi SVD hit its sweep
// limit: the outputs are written but may be inaccurate, so the call says so.
gcf_status svd_status(gcf_ctx* c) {
  if (c->last_svd_unconverged > 0)
    return fail(c, GCF_ETIMEOUT, std::to_string(c->last_svd_unconverged) +
                                     " truncated SVDs did not converge within the sweep limit");
  return GCF_OK;
}

inline long long al32(long long n) { return (n + 31) / 32 * 32; }

// One absorption step: input bond table bin (Lx+1), output bout, qr, svd.
void plan_step(int Lx, int Dk, int chi, int pout, const int* bin, int* qr, int* svd, int* bout) {
  std::vector<int> ab(Lx + 1);
  ab[0] = 1;
  for (int c = 1; c < Lx; ++c) ab[c] = bin[c] * Dk;
  ab[Lx] = 1;
  qr[0] = 1;
  for (int c = 0; c < Lx - 1; ++c) qr[c + 1] = std::min(qr[c] * pout, ab[c + 1]);
  qr[Lx] = 1;
  bout[Lx] = 1;
  for (int c = Lx - 1; c >= 1; --c) {
    const int k0 = std::min(qr[c], pout * bout[c + 1]);
    svd[c] = k0 > chi ? 1 : 0;
    bout[c] = std::min(chi, k0);
  }
  bout[0] = 1;
  svd[0] = 0;
  svd[Lx] = 0;
}

// Executor for the sampling / measurement kernel: the whole CTA on one
// chain, or two or four chains per CTA on groups of 128 threads (optionally
// in lockstep, see vmc_kernel.cuh).  GCFVMC_EXEC=cta|group|group4,
// GCFVMC_SMEM / GCFVMC_SMEM_CTA (placement level 0-3) and GCFVMC_LOCK=0|1
// override the planner's choice.
enum ExecKind { EXEC_CTA = 0, EXEC_GROUP = 1, EXEC_GROUP4 = 2 };

// Dynamic shared memory of one chain: [configuration][hot buffers of the
// placement level] then, for the tcgen05 path, the operand staging area at
// a 16-byte boundary.  CTA form: from the block's base; group form: each
// group's region also starts with its SharedV.
// The factorisation workspace (fz_elems scalars) shares that area: the
// staging area is live only inside an environment GEMM, the workspace only
// inside a factorisation of the absorption, and neither calls the other.
inline size_t r16(size_t b) { return (b + 15) / 16 * 16; }
size_t scratch_area(const Plan& p, size_t sb) { return std::max(r16((size_t)p.tc_bytes), (size_t)p.fz_elems * sb); }
size_t cta_tc_off(const Plan& p, int level, size_t sb) {
  return r16((size_t)p.cfg_bytes + (size_t)p.level_elems(level) * sb);
}
size_t cta_fz_off(const Plan& p, int level, size_t sb) { return cta_tc_off(p, level, sb); }
size_t cta_smem_bytes(const Plan& p, int level, size_t sb) {
  if (!p.tc_bytes && !p.fz_elems) return (size_t)p.cfg_bytes + (size_t)p.level_elems(level) * sb;
  return cta_tc_off(p, level, sb) + scratch_area(p, sb);
}
size_t group_tc_off(const Plan& p, int level, size_t sb) {
  return r16(sharedv_bytes() + (size_t)p.cfg_bytes + (size_t)p.level_elems(level) * sb);
}
size_t group_fz_off(const Plan& p, int level, size_t sb) { return group_tc_off(p, level, sb); }
size_t group_smem_bytes(const Plan& p, int level, size_t sb) {
  return r16(group_tc_off(p, level, sb) + scratch_area(p, sb));
}
bool grouped(const gcf_ctx* c);
int n_groups(const gcf_ctx* c);

void plan_group(gcf_ctx* c) {
  Plan& p = c->plan;
  const int G = 128;
  c->group_threads = G;
  auto fits = [&](int ng, int lv, size_t budget) {
    return (size_t)ng * group_smem_bytes(p, lv, c->sbytes) <= budget;
  };
  // two groups per CTA: the largest level that leaves room for a second CTA
  int lv2 = 0;
  for (int lv = 1; lv <= 3; ++lv)
    if (fits(2, lv, 110 * 1024)) lv2 = lv;
  // Default form: four chain groups per CTA of 512 threads (one CTA per SM)
  // in lockstep, with the hot buffers in shared memory (level 1; the larger
  // levels measured slower for four groups); else two groups per CTA; else
  // the whole CTA per chain.  The autotuner can pick any other form.
  if (fits(4, 1, 216 * 1024)) {
    c->exec = EXEC_GROUP4;
    p.group_level = 1;
  } else if (lv2 >= 1) {
    c->exec = EXEC_GROUP;
    p.group_level = lv2;
  } else {
    c->exec = EXEC_CTA;
    p.group_level = 0;
  }
  c->lockstep = 1;
  if (const char* e = std::getenv("GCFVMC_LOCK")) c->lockstep = std::atoi(e) ? 1 : 0;
  c->lock_fault = 0;
  if (const char* e = std::getenv("GCFVMC_LOCK_FAULT")) c->lock_fault = std::atoi(e) ? 1 : 0;
  if (const char* e = std::getenv("GCFVMC_EXEC")) {
    if (!std::strcmp(e, "group4")) {
      c->exec = EXEC_GROUP4;
      p.group_level = fits(4, 1, 216 * 1024) ? 1 : 0;
    }
    if (!std::strcmp(e, "group")) {
      c->exec = EXEC_GROUP;
      p.group_level = lv2;
    }
    if (!std::strcmp(e, "cta")) c->exec = EXEC_CTA;
  }
  if (const char* e = std::getenv("GCFVMC_SMEM")) p.group_level = std::max(0, std::min(3, std::atoi(e)));
  p.group_smem = group_smem_bytes(p, p.group_level, c->sbytes);
}

// Tables derived from the bond dimensions, appended after the six plan
// tables (bondB, bondT, qrB, svdB, qrT, svdT; (Ly+1) x (Lx+1) each):
//   offB[j][c]: offset of site c in B slot j (packed bd[c] x phys x bd[c+1]);
//   offT[r][c]: the same for T slot r;
//   denseB[r], denseT[r]: 1 if absorbing row r into B (slot r -> r+1) or into
//   T (slot r+1 -> r) takes the exact identity + core form: every output bond
//   at full rank min(p^c, p^(L-c)) and the dense state within the buffers.
void append_derived_tables(const gcf_ctx* c, std::vector<int>& t) {
  const Plan& p = c->plan;
  const int Lx = c->m.Lx, Ly = c->m.Ly, Dk = c->Dk, W = Lx + 1, R = Ly + 1;
  auto physB = [&](int j) { return j == 0 ? 1 : Dk; };
  auto physT = [&](int r) { return r == Ly ? 1 : Dk; };
  auto offsets = [&](const int* bd, int phys) {
    int o = 0;
    for (int cc = 0; cc < Lx; ++cc) { t.push_back(o); o += bd[cc] * phys * bd[cc + 1]; }
    t.push_back(o);
  };
  for (int j = 0; j < R; ++j) offsets(&p.bondB[j * W], physB(j));
  for (int r = 0; r < R; ++r) offsets(&p.bondT[r * W], physT(r));
  const long long dmax = p.tmp_max;
  auto dense = [&](const int* bdi, int pin, const int* bdo, int pout) {
    int ok = (pout == Dk) ? 1 : 0;
    for (int cc = 0; cc <= Lx; ++cc) {
      long long lo = 1, hi = 1;
      for (int i = 0; i < cc; ++i) lo *= pout;
      for (int i = 0; i < Lx - cc; ++i) hi *= pout;
      if (bdo[cc] != (lo < hi ? lo : hi)) ok = 0;
    }
    long long pw = 1;
    for (int i = 0; i < Lx && pw <= dmax; ++i) pw *= pout;
    if (pw * Dk > dmax) ok = 0;
    long long rows = 1;
    for (int cc = 0; cc < Lx && ok; ++cc) {
      rows *= pin;
      if (rows * bdi[cc + 1] > dmax) ok = 0;
    }
    return ok;
  };
  for (int r = 0; r < R; ++r)
    t.push_back(r + 1 < R ? dense(&p.bondB[r * W], physB(r), &p.bondB[(r + 1) * W], physB(r + 1)) : 0);
  for (int r = 0; r < R; ++r)
    t.push_back(r + 1 < R ? dense(&p.bondT[(r + 1) * W], physT(r + 1), &p.bondT[r * W], physT(r)) : 0);
}

bool grouped(const gcf_ctx* c) { return c->exec == EXEC_GROUP || c->exec == EXEC_GROUP4; }
int n_groups(const gcf_ctx* c) { return c->exec == EXEC_GROUP4 ? 4 : 2; }

// Kernel form: executor and shared-memory level (sizes follow from the plan).
void set_form(gcf_ctx* c, int exec, int level) {
  Plan& p = c->plan;
  c->exec = exec;
  if (exec == EXEC_GROUP || exec == EXEC_GROUP4) {
    p.group_level = level;
    p.group_smem = group_smem_bytes(p, level, c->sbytes);
  } else {
    p.cta_level = level;
    p.hot_elems = p.level_elems(level);
    p.dyn_smem = cta_smem_bytes(p, level, c->sbytes);
  }
}

void build_plan(gcf_ctx* c) {
  const int Lx = c->m.Lx, Ly = c->m.Ly, Dk = c->Dk, chi = c->m.chi;
  const int W = Lx + 1;
  Plan& p = c->plan;
  p.bondB.assign((Ly + 1) * W, 1);
  p.bondT.assign((Ly + 1) * W, 1);
  p.qrB.assign((Ly + 1) * W, 1);
  p.svdB.assign((Ly + 1) * W, 0);
  p.qrT.assign((Ly + 1) * W, 1);
  p.svdT.assign((Ly + 1) * W, 0);
  // B: slot j holds B[j-1]; step r absorbs row r: slot r -> slot r+1
  for (int r = 0; r <= Ly - 2; ++r)
    plan_step(Lx, Dk, chi, Dk, &p.bondB[r * W], &p.qrB[r * W], &p.svdB[r * W], &p.bondB[(r + 1) * W]);
  // T: slot r holds T[r]; step r: slot r+1 -> slot r
  for (int r = Ly - 1; r >= 1; --r)
    plan_step(Lx, Dk, chi, Dk, &p.bondT[(r + 1) * W], &p.qrT[r * W], &p.svdT[r * W], &p.bondT[r * W]);
  auto mps_size = [&](const int* bd, int phys) {
    long long s = 0;
    for (int cc = 0; cc < Lx; ++cc) s += (long long)bd[cc] * phys * bd[cc + 1];
    return s;
  };
  long long ms = Lx;
  for (int j = 0; j <= Ly; ++j) {
    ms = std::max(ms, mps_size(&p.bondB[j * W], j == 0 ? 1 : Dk));
    ms = std::max(ms, mps_size(&p.bondT[j * W], j == Ly ? 1 : Dk));
  }
  p.mps_stride = al32(ms);
  // QR-pass sites, matrices, taus
  long long qs = 1, mat = 1, tau = 1, fzq = 0, fzj = 0;
  bool truncates = false;
  auto step_sizes = [&](const int* bin, const int* qr, const int* svd, const int* bout, int pin,
                        int pout) {
    std::vector<int> ab(Lx + 1);
    ab[0] = 1;
    for (int cc = 1; cc < Lx; ++cc) ab[cc] = bin[cc] * Dk;
    ab[Lx] = 1;
    for (int cc = 0; cc < Lx; ++cc) {
      const long long rows = (long long)qr[cc] * pout, cols = ab[cc + 1];
      // columns padded to whole 4-row chunks (the FP32 column-major form)
      fzq = std::max(fzq, ((rows + 3) & ~3LL) * (cols + std::min(rows, cols)));
      qs = std::max(qs, rows * std::min(rows, cols));
      mat = std::max(mat, (long long)ab[cc] * pout * ab[cc + 1]);  // Z
      mat = std::max(mat, rows * cols);                             // X
      mat = std::max(mat, (long long)std::max(rows, cols) * std::max(rows, cols));
      tau = std::max(tau, std::max(rows, cols));
      tau = std::max(tau, (long long)std::max(ab[cc], ab[cc + 1]) * pout);
    }
    for (int cc = Lx - 1; cc >= 1; --cc) {
      const long long yr = qr[cc], yc = (long long)pout * bout[cc + 1];
      const long long k0 = std::min(yr, yc);
      fzq = std::max(fzq, ((yc + 3) & ~3LL) * (yr + k0));
      if (svd[cc]) {
        truncates = true;
        // FP32 column-major form: W and J with columns padded to whole 4-row
        // chunks, the kept columns of J before and after re-orthogonalisation
        // and their Gram matrix
        const long long kk = bout[cc], ldj = (k0 + 3) & ~3LL;
        fzj = std::max(fzj, ((yr + 3) & ~3LL) * k0 + ldj * k0 + 2 * ldj * kk + kk * kk);
      }
      mat = std::max(mat, std::max(yr, yc) * std::max(yr, yc));
      mat = std::max(mat, k0 * k0);
      mat = std::max(mat, (long long)qr[cc - 1] * pout * bout[cc]);
      tau = std::max(tau, std::max(yr, yc));
    }
    (void)pin;
  };
  for (int r = 0; r <= Ly - 2; ++r)
    step_sizes(&p.bondB[r * W], &p.qrB[r * W], &p.svdB[r * W], &p.bondB[(r + 1) * W], r == 0 ? 1 : Dk, Dk);
  for (int r = Ly - 1; r >= 1; --r)
    step_sizes(&p.bondT[(r + 1) * W], &p.qrT[r * W], &p.svdT[r * W], &p.bondT[r * W], r == Ly - 1 ? 1 : Dk, Dk);
  // shared-memory factorisation workspace: for plans that truncate (the
  // QR, Q formation and Jacobi sweeps then dominate), the largest of the QR
  // and Jacobi needs that fits 64 KB; the other runs in global scratch
  {
    const long long cap = (64 * 1024) / (long long)c->sbytes;
    p.fz_elems = 0;
    if (truncates) {
      if (fzq <= cap) p.fz_elems = std::max(p.fz_elems, fzq);
      if (fzj <= cap) p.fz_elems = std::max(p.fz_elems, fzj);
    }
  }
  p.qsite_stride = al32(qs);
  p.mat_max = al32(mat);
  p.tau_max = al32(tau);
  // strip / row environments and intermediates
  long long env = 1, env3 = 1, tmp = 1;
  for (int r = 0; r <= Ly - 2; ++r) {
    const int* bb = &p.bondB[r * W];
    const int* bt = &p.bondT[(r + 2) * W];
    const int pB = r == 0 ? 1 : Dk, pT = (r + 2 == Ly) ? 1 : Dk;
    for (int cc = 0; cc <= Lx; ++cc) {
      const int h = (cc == 0 || cc == Lx) ? 1 : Dk;
      env = std::max(env, (long long)bb[cc] * h * h * bt[cc]);
    }
    for (int cc = 0; cc < Lx; ++cc) {
      const long long nA = bb[cc], nB = bt[cc], nA2 = bb[cc + 1], nB2 = bt[cc + 1];
      const long long hI = cc == 0 ? 1 : Dk, hO = cc == Lx - 1 ? 1 : Dk;
      tmp = std::max(tmp, hI * hI * nB * pB * nA2);
      tmp = std::max(tmp, hI * nB * nA2 * hO * Dk);
      tmp = std::max(tmp, nA2 * hO * hO * nB * pT);
      tmp = std::max(tmp, nA2 * hO * hI * Dk * nB);
      tmp = std::max(tmp, nA2 * hI * hI * pB * nB);
      (void)nA;
      (void)nB2;
    }
  }
  for (int r = 0; r <= Ly - 1; ++r) {
    const int* bb = &p.bondB[r * W];
    const int* bt = &p.bondT[(r + 1) * W];
    const int pB = r == 0 ? 1 : Dk, pT = (r + 1 == Ly) ? 1 : Dk;
    for (int cc = 0; cc <= Lx; ++cc) {
      const int h = (cc == 0 || cc == Lx) ? 1 : Dk;
      env3 = std::max(env3, (long long)bb[cc] * h * bt[cc]);
    }
    for (int cc = 0; cc < Lx; ++cc) {
      const long long nB = bt[cc], nA2 = bb[cc + 1];
      const long long hI = cc == 0 ? 1 : Dk, hO = cc == Lx - 1 ? 1 : Dk;
      tmp = std::max(tmp, hI * nB * pB * nA2);
      tmp = std::max(tmp, nB * nA2 * hO * pT);
      tmp = std::max(tmp, nA2 * hO * nB * pT);
      tmp = std::max(tmp, nA2 * hI * pB * nB);
    }
  }
  p.env_stride = (int)al32(env);
  p.env3_stride = (int)al32(env3);
  // dense (identity + core) compression buffers: D_k * D_k^Lx when small
  {
    long long pw = 1;
    for (int i = 0; i < Lx && pw <= 8192; ++i) pw *= Dk;
    if (pw * Dk <= 8192) tmp = std::max(tmp, pw * Dk);
  }
  p.tmp_max = al32(tmp);
  const long long D4 = (long long)Dk * Dk * Dk * Dk;
  long long o = 0;
  auto take = [&](long long n) { long long r = o; o += al32(n); return r; };
  p.o_net = take((long long)Lx * Ly * D4);
  p.o_prop = take(4 * D4);
  // boundary-MPS store: every slot, or every K-th plus one segment buffer
  // (B slots 0..Ly-1, T slots 1..Ly)
  p.ck_every = c->ck_every;
  if (p.ck_every) {
    const int K = p.ck_every;
    p.o_B = take((long long)((Ly - 1) / K + 1) * p.mps_stride);
    p.o_Bseg = take((long long)K * p.mps_stride);
    p.o_T = take((long long)((Ly - 1) / K + 1) * p.mps_stride);
    p.o_Tseg = take((long long)K * p.mps_stride);
  } else {
    p.o_B = take((Ly + 1) * p.mps_stride);
    p.o_T = take((Ly + 1) * p.mps_stride);
  }
  p.o_Q = take((long long)Lx * p.qsite_stride);
  p.o_M1 = take(p.mat_max);
  p.o_M2 = take(p.mat_max);
  p.o_M3 = take(p.mat_max);
  p.o_tau = take(p.tau_max);
  p.o_J = take(p.mat_max);
  p.o_envR = take((long long)(Lx + 1) * p.env_stride);
  p.o_envL = take(p.env_stride);
  p.o_envX = take(p.env_stride);
  p.o_envY = take(p.env_stride);
  p.o_t1 = take(p.tmp_max);
  p.o_t2 = take(p.tmp_max);
  p.o_t3 = take(std::max<long long>(p.tmp_max, D4 * D4 / (Dk * Dk) * Dk * Dk));
  p.o_env3R = take((long long)(Lx + 1) * p.env3_stride);
  p.o_env3L = take(p.env3_stride);
  p.o_env3X = take(p.env3_stride);
  p.o_env3Y = take(p.env3_stride);
  p.o_G = take(D4);
  p.o_sigma = take(2 * p.tau_max + 32);  // SVD column norms (doubles)
  p.o_sel = take(p.tau_max + 32);         // selected columns (ints)
  // absorbed sites of one step (warp compression path)
  long long zmax = 1;
  for (int j = 0; j <= Ly; ++j)
    for (const std::vector<int>* bt : {&p.bondB, &p.bondT}) {
      const int* bd = &(*bt)[j * W];
      long long z = 0;
      for (int cc = 0; cc < Lx; ++cc) {
        const long long abl = (cc == 0) ? 1 : (long long)bd[cc] * Dk;
        const long long abr = (cc + 1 == Lx) ? 1 : (long long)bd[cc + 1] * Dk;
        z += abl * Dk * abr;
      }
      zmax = std::max(zmax, z);
    }
  p.z_size = zmax;
  p.o_Z = take(zmax);
  // packed QR-pass sites of one step (rows_c x qr[c+1])
  long long qmax = 1;
  for (int r = 0; r <= Ly; ++r)
    for (const std::vector<int>* qt : {&p.qrB, &p.qrT}) {
      const int* q = &(*qt)[r * W];
      long long z = 0;
      for (int cc = 0; cc < Lx; ++cc) z += (long long)q[cc] * Dk * q[cc + 1];
      qmax = std::max(qmax, z);
    }
  p.q_pack = qmax;
  p.o_X = take(p.mat_max);
  p.o_W1 = take(p.mat_max);
  p.o_W2 = take(p.mat_max);
  p.o_W3 = take(p.mat_max);
  p.o_W4 = take(p.mat_max);
  p.ws_stride = o;
  // hot buffers: shared memory if they fit the budget
  long long h = 0;
  auto hot = [&](long long n) { long long r = h; h += (n + 3) / 4 * 4; return r; };
  p.so_net = hot((long long)Lx * Ly * D4);
  p.so_prop = hot(4 * D4);
  p.so_cop = hot(D4 * D4 / (Dk * Dk) * Dk * Dk);  // D_k^6
  p.so_envL = hot(p.env_stride);
  p.so_envX = hot(p.env_stride);
  p.so_envY = hot(p.env_stride);
  p.so_env3L = hot(p.env3_stride);
  p.so_env3X = hot(p.env3_stride);
  p.so_env3Y = hot(p.env3_stride);
  p.so_t1 = hot(p.tmp_max);
  p.so_t2 = hot(p.tmp_max);
  p.cfg_bytes = (c->cfg_len + 15) / 16 * 16;
  // shared-memory placement levels: 1 = hot buffers, 2 = + the staged B / T
  // rows of the current pass, 3 = + the right environments of the pass
  p.hot_base_elems = h;
  p.so_sB = hot(p.mps_stride);
  p.so_sT = hot(p.mps_stride);
  p.hot_mps_elems = h;
  p.so_envR = hot((long long)(Lx + 1) * p.env_stride);
  p.so_env3R = hot((long long)(Lx + 1) * p.env3_stride);
  p.hot_all_elems = h;
  // tcgen05 staging of the BF16 form (real chains): the largest environment
  // GEMM has N <= D_k^2 chi_b and K <= D_k chi_b (chi_b the largest bond of
  // any B / T); the tensor-core path takes N <= 128 (its TMEM columns)
  p.tc_bytes = 0;
  if (c->m.precision == GCF_BF16 && c->kind == S_F32) {
    int chib = 1;
    for (int v : p.bondB) chib = std::max(chib, v);
    for (int v : p.bondT) chib = std::max(chib, v);
    const int Nmax = Dk * Dk * chib, Kmax = Dk * chib;
    if (Nmax <= 128) p.tc_bytes = (tc_stage_bytes(Nmax, Kmax) + 15) / 16 * 16;
  }
  // one chain per CTA: the largest level that keeps two CTAs on an SM
  const size_t budget = 100 * 1024;
  p.cta_level = 0;
  for (int lv = 1; lv <= 3; ++lv)
    if (cta_smem_bytes(p, lv, c->sbytes) <= budget) p.cta_level = lv;
  if (const char* e = std::getenv("GCFVMC_SMEM_CTA")) p.cta_level = std::max(0, std::min(3, std::atoi(e)));
  p.hot_elems = p.level_elems(p.cta_level);
  p.dyn_smem = cta_smem_bytes(p, p.cta_level, c->sbytes);
  plan_group(c);
}

template <class T>
KParams<T> make_params(gcf_ctx* c) {
  KParams<T> k{};
  const Plan& p = c->plan;
  k.N = c->m.N; k.Lx = c->m.Lx; k.Ly = c->m.Ly; k.Dk = c->Dk; k.chi = c->m.chi;
  k.matter = c->m.has_matter; k.P = c->P;
  k.n_h = c->n_h; k.n_v = c->n_v; k.n_s = c->n_s; k.cfg_len = c->cfg_len;
  k.n_plaq = c->n_plaq; k.n_slots = c->n_slots;
  k.h = c->m.h; k.g = c->m.g; k.J = c->m.J; k.m = c->m.m;
  for (int n = 0; n < 8; ++n)
    k.elink[n] = n < c->m.N ? c->m.g * (2.0 - 2.0 * std::cos(2.0 * 3.14159265358979323846 * n / c->m.N)) : 0.0;
  k.Q = c->d_Q; k.voff = c->d_voff; k.vbs = c->d_vbs; k.params = (const T*)c->d_params;
  const int W = c->m.Lx + 1, R = c->m.Ly + 1;
  k.bondB = c->d_tables;
  k.bondT = c->d_tables + R * W;
  k.qrB = c->d_tables + 2 * R * W;
  k.svdB = c->d_tables + 3 * R * W;
  k.qrT = c->d_tables + 4 * R * W;
  k.svdT = c->d_tables + 5 * R * W;
  k.tab = c->d_tables;
  k.tab_ints = c->tab_ints;
  k.scratch = (T*)c->d_scratch;
  k.ws_stride = p.ws_stride;
  k.o_net = p.o_net; k.o_prop = p.o_prop; k.o_B = p.o_B; k.o_T = p.o_T; k.o_Q = p.o_Q;
  k.ck_every = p.ck_every; k.o_Bseg = p.o_Bseg; k.o_Tseg = p.o_Tseg;
  k.o_M1 = p.o_M1; k.o_M2 = p.o_M2; k.o_M3 = p.o_M3; k.o_tau = p.o_tau; k.o_J = p.o_J;
  k.o_envR = p.o_envR; k.o_envL = p.o_envL; k.o_envX = p.o_envX; k.o_envY = p.o_envY;
  k.o_t1 = p.o_t1; k.o_t2 = p.o_t2; k.o_t3 = p.o_t3;
  k.o_env3R = p.o_env3R; k.o_env3L = p.o_env3L; k.o_env3X = p.o_env3X; k.o_env3Y = p.o_env3Y;
  k.o_G = p.o_G;
  k.mps_stride = p.mps_stride; k.qsite_stride = p.qsite_stride;
  k.env_stride = p.env_stride; k.env3_stride = p.env3_stride;
  k.max_sweeps_svd = c->svd_sweeps;
  k.hot_in_smem = p.cta_level >= 1;
  k.mps_in_smem = p.cta_level >= 2;
  k.renv_in_smem = p.cta_level >= 3;
  k.so_envR = p.so_envR; k.so_env3R = p.so_env3R; k.so_sB = p.so_sB; k.so_sT = p.so_sT;
  k.o_sigma = p.o_sigma; k.o_sel = p.o_sel;
  k.dense_max = p.tmp_max;
  k.o_Z = p.o_Z; k.z_size = p.z_size; k.o_X = p.o_X; k.o_W1 = p.o_W1; k.o_W2 = p.o_W2; k.o_W3 = p.o_W3;
  k.o_W4 = p.o_W4;
  k.q_pack = p.q_pack;
  k.so_net = p.so_net; k.so_prop = p.so_prop; k.so_cop = p.so_cop;
  k.so_envL = p.so_envL; k.so_envX = p.so_envX; k.so_envY = p.so_envY;
  k.so_env3L = p.so_env3L; k.so_env3X = p.so_env3X; k.so_env3Y = p.so_env3Y;
  k.so_t1 = p.so_t1; k.so_t2 = p.so_t2; k.smem_cfg_bytes = p.cfg_bytes;
  k.group_smem_bytes = (long long)p.group_smem;
  k.lockstep = c->lockstep;
  k.lock_fault = c->lock_fault;
  k.group_threads = c->group_threads;
  // tensor-core forms exist for FP32 storage only
  k.gemm_mode = GEMM_FFMA;
  if (c->kind == S_F32 || c->kind == S_C64) {
    if (c->m.precision == GCF_TF32) k.gemm_mode = GEMM_TF32X3;
    if (c->m.precision == GCF_BF16) k.gemm_mode = GEMM_BF16;
  }
  // Tensor-core forms.  The boundary-MPS absorption keeps FP32 products in
  // every form: its truncations amplify operand rounding (the 3-pass TF32
  // split, about 21 bits with tensor-core accumulation, measured 1.4-1.8e-4
  // amplitude error on the truncated 10x10 and 16x16 lattices against
  // 3e-6-1.6e-5 in FP32).  BF16 form: BF16 operands only in the strip
  // environments (plaquette and vertical-hop ratios: Metropolis decisions and
  // E_loc); the row environments (amplitude, O, horizontal-hop ratios) run in
  // the 3-pass TF32 form.
  k.row_gemm_mode = k.gemm_mode == GEMM_BF16 ? GEMM_TF32X3 : k.gemm_mode;
  k.absorb_gemm_mode = GEMM_FFMA;
  k.tc_bf16 = p.tc_bytes > 0 && k.gemm_mode == GEMM_BF16 ? 1 : 0;
  k.tc_bytes = p.tc_bytes;
  k.tc_off = (long long)cta_tc_off(p, p.cta_level, c->sbytes);
  k.fz_elems = p.fz_elems;
  k.fz_off = (long long)cta_fz_off(p, p.cta_level, c->sbytes);
  k.status = c->d_status;
  return k;
}

// Chain slots for n chains when at most max_slots run at once: the fewest
// slots that still need the same number of rounds, so every slot runs the
// same number of chains (no partly filled last round).
long long balanced_slots(long long n, long long max_slots) {
  max_slots = std::max<long long>(1, max_slots);
  const long long rounds = (n + max_slots - 1) / max_slots;
  return std::max<long long>(1, (n + rounds - 1) / std::max<long long>(1, rounds));
}

int grid_for(gcf_ctx* c, int n_chains) {
  int per_sm = 1;
  switch (c->kind) {
    case S_F32: per_sm = occupancy_vmc<float>(256, c->plan.dyn_smem); break;
    case S_F64: per_sm = occupancy_vmc<double>(256, c->plan.dyn_smem); break;
    case S_C64: per_sm = occupancy_vmc<cfloat>(256, c->plan.dyn_smem); break;
    default: per_sm = occupancy_vmc<cdouble>(256, c->plan.dyn_smem); break;
  }
  return (int)balanced_slots(n_chains, (long long)c->sms * std::max(1, per_sm));
}

// cudaMalloc that leaves the pointer null when it fails (retry paths free
// whatever a group holds)
template <class P>
bool dalloc(P** p, size_t bytes) {
  if (cudaMalloc((void**)p, bytes) == cudaSuccess) return true;
  *p = nullptr;
  return false;
}

gcf_status ensure_scratch(gcf_ctx* c, long long ctas) {
  if (ctas <= c->scratch_ctas) return GCF_OK;
  if (c->d_scratch) cudaFree(c->d_scratch);
  c->d_scratch = nullptr;
  c->scratch_ctas = 0;
  const size_t bytes = (size_t)ctas * c->plan.ws_stride * c->sbytes;
  cudaError_t e = cudaMalloc(&c->d_scratch, bytes);
  if (e != cudaSuccess) return fail(c, GCF_ENOMEM, "scratch allocation failed");
  c->scratch_ctas = ctas;
  return GCF_OK;
}

template <class T>
gcf_status run_vmc(gcf_ctx* c, int mode, int want, int n, int n_sweeps, uint64_t seed,
                   int8_t* configs, const gcf_samples* out, int* gauss_count, cudaStream_t stream,
                   bool async) {
  const bool warp = grouped(c);
  const int W = n_groups(c);  // chains per CTA
  int grid = 1;
  if (warp) {
    const int per_sm = occupancy_vmc_grouped<T>(128 * W, W * c->plan.group_smem);
    if (per_sm < 1) return fail(c, GCF_EINVAL, "grouped launch does not fit an SM");
    const long long slots = balanced_slots(n, (long long)c->sms * per_sm * W);
    grid = (int)std::max<long long>(1, (slots + W - 1) / W);
  } else {
    grid = grid_for(c, n);
  }
  gcf_status st = ensure_scratch(c, warp ? (long long)grid * W : grid);
  if (st != GCF_OK) return st;
  KParams<T> k = make_params<T>(c);
  if (warp) {
    k.hot_in_smem = c->plan.group_level >= 1;
    k.mps_in_smem = c->plan.group_level >= 2;
    k.renv_in_smem = c->plan.group_level >= 3;
    k.tc_off = (long long)group_tc_off(c->plan, c->plan.group_level, c->sbytes);
    k.fz_off = (long long)group_fz_off(c->plan, c->plan.group_level, c->sbytes);
  }
  k.n_chains = n; k.n_sweeps = n_sweeps; k.mode = mode; k.want = want; k.seed = seed;
  k.configs = configs;
  if (out) {
    k.log_abs = out->log_abs; k.phase = out->phase; k.e_loc = out->e_loc;
    k.block_ids = out->block_ids; k.O = (T*)out->O;
    k.accepted = out->accepted; k.proposed = out->proposed;
  }
  CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), stream));
  if (warp)
    CUDA_TRY(c, launch_vmc_grouped<T>(k, grid, 128 * W, W * c->plan.group_smem, stream));
  else
    CUDA_TRY(c, launch_vmc<T>(k, grid, 256, c->plan.dyn_smem, stream));
  c->launches += 1;
  if (async) return GCF_OK;
  int h_status[4];
  CUDA_TRY(c, cudaMemcpyAsync(h_status, c->d_status, sizeof(h_status), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (gauss_count) *gauss_count = h_status[ST_GAUSS];
  c->last_phase_timeouts = h_status[ST_PHASE_TIMEOUT];
  c->last_svd_unconverged = h_status[ST_SVD];
  c->last_tc_timeouts = h_status[ST_TC_TIMEOUT];
  return GCF_OK;
}

template <class T>
gcf_status run_multi(gcf_ctx* const* cs, int n_ctx, const int* n_chains, int n_sweeps, const uint64_t* seeds,
                     int8_t* const* configs, const gcf_samples* outs) {
  gcf_ctx* c0 = cs[0];
  std::vector<KParams<T>> ks(n_ctx);
  std::vector<long long> start(n_ctx + 1, 0);
  size_t smem = 0, tc_off = 0, tc_bytes = 0;
  long long ws = 0;
  // The chains form one queue that the kernel's chain slots draw from when
  // free: contexts in decreasing order of the work of one chain (sites x
  // chi^3, the factorisations' scaling), so the longest chains start first.
  std::vector<int> order(n_ctx);
  for (int i = 0; i < n_ctx; ++i) order[i] = i;
  auto cost = [&](int i) {
    const double chi = cs[i]->m.chi;
    return (double)cs[i]->m.Lx * cs[i]->m.Ly * chi * chi * chi * cs[i]->Dk;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  for (int j = 0; j < n_ctx; ++j) {
    const int i = order[j];
    gcf_ctx* c = cs[i];
    KParams<T> k = make_params<T>(c);
    gcf_samples o{};
    if (outs) o = outs[i];
    k.n_chains = n_chains[i]; k.n_sweeps = n_sweeps; k.mode = 1; k.seed = seeds[i]; k.configs = configs[i];
    k.want = (o.log_abs || o.phase ? WANT_AMP : 0) | (o.e_loc ? WANT_ELOC : 0) | (o.O || o.block_ids ? WANT_GRAD : 0);
    k.log_abs = o.log_abs; k.phase = o.phase; k.e_loc = o.e_loc; k.block_ids = o.block_ids; k.O = (T*)o.O;
    k.accepted = o.accepted; k.proposed = o.proposed;
    ks[j] = k;
    start[j + 1] = start[j] + n_chains[i];
    smem = std::max(smem, c->plan.dyn_smem);
    tc_off = std::max(tc_off, cta_tc_off(c->plan, c->plan.cta_level, c->sbytes));
    tc_bytes = std::max(tc_bytes, (size_t)c->plan.tc_bytes);
    ws = std::max(ws, c->plan.ws_stride);
    CUDA_TRY(c0, cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), c0->stream));
  }
  const long long total = start[n_ctx];
  if (total == 0) return GCF_OK;
  // one staging area after the largest context's configuration and hot
  // buffers; the tensor-core path runs only if every context takes it
  bool tc_all = true;
  long long fz = 0;
  for (int i = 0; i < n_ctx; ++i) {
    tc_all = tc_all && ks[i].tc_bf16;
    fz = std::max(fz, ks[i].fz_elems);
  }
  const size_t fz_off = tc_off;  // the two share one area (see cta_tc_off)
  const size_t area = std::max((tc_bytes + 15) / 16 * 16, (size_t)fz * c0->sbytes);
  if (tc_bytes > 0 || fz > 0) smem = std::max(smem, tc_off + area);
  for (int i = 0; i < n_ctx; ++i) {
    ks[i].tc_bf16 = tc_all ? 1 : 0;
    ks[i].tc_off = (long long)tc_off;
    ks[i].tc_bytes = (long long)tc_bytes;
    ks[i].fz_elems = fz;
    ks[i].fz_off = (long long)fz_off;
  }
  // Four chains per CTA (vmc_kernel_multi4) when some context truncates: its
  // sampling is bound by the latency of the factorisations, which more
  // resident chains hide; hot buffers then stay in scratch (level 0).
  // GCFVMC_MULTI=cta|group4 forces a form.
  int block = 256;
  long long group_bytes = 0;
  {
    size_t cfg_max = 0;
    for (int i = 0; i < n_ctx; ++i) cfg_max = std::max(cfg_max, (size_t)cs[i]->plan.cfg_bytes);
    const size_t g_tc = (sharedv_bytes() + cfg_max + 15) / 16 * 16;
    const size_t g_fz = g_tc;
    const size_t gb = (g_tc + area + 15) / 16 * 16;
    bool want4 = fz > 0;
    if (const char* e = std::getenv("GCFVMC_MULTI")) want4 = !std::strcmp(e, "group4");
    if (want4 && 4 * gb <= 216 * 1024 && occupancy_vmc_multi<T>(512, 4 * gb) >= 1) {
      block = 512;
      group_bytes = (long long)gb;
      smem = 4 * gb;
      for (int i = 0; i < n_ctx; ++i) {
        ks[i].hot_in_smem = 0;
        ks[i].mps_in_smem = 0;
        ks[i].renv_in_smem = 0;
        ks[i].tc_off = (long long)g_tc;
        ks[i].fz_off = (long long)g_fz;
        ks[i].group_smem_bytes = group_bytes;
      }
    }
  }
  const int per_sm = occupancy_vmc_multi<T>(block, smem);
  if (per_sm < 1) return fail(c0, GCF_EINVAL, "gcf_sample_multi: the largest context does not fit an SM");
  const int per_cta = block == 512 ? 4 : 1;
  // every resident slot draws from the queue: as many slots as fit, at most
  // one per chain
  const long long slots = std::min<long long>(total, (long long)c0->sms * per_sm * per_cta);
  const long long grid = (slots + per_cta - 1) / per_cta;
  const size_t arena = (size_t)grid * per_cta * ws * c0->sbytes;
  if (arena > c0->multi_arena_bytes) {
    if (c0->multi_arena) cudaFree(c0->multi_arena);
    c0->multi_arena = nullptr;
    c0->multi_arena_bytes = 0;
    if (cudaMalloc(&c0->multi_arena, arena) != cudaSuccess) return fail(c0, GCF_ENOMEM, "multi-context scratch");
    c0->multi_arena_bytes = arena;
  }
  const size_t kb = sizeof(KParams<T>) * n_ctx,
               tb = (kb + 15) / 16 * 16 + sizeof(long long) * (n_ctx + 1) + 16;
  if (tb > c0->multi_tab_bytes) {
    if (c0->multi_tab) cudaFree(c0->multi_tab);
    c0->multi_tab = nullptr;
    c0->multi_tab_bytes = 0;
    if (cudaMalloc(&c0->multi_tab, tb) != cudaSuccess) return fail(c0, GCF_ENOMEM, "multi-context tables");
    c0->multi_tab_bytes = tb;
  }
  KParams<T>* d_ks = (KParams<T>*)c0->multi_tab;
  long long* d_start = (long long*)((char*)c0->multi_tab + (kb + 15) / 16 * 16);
  CUDA_TRY(c0, cudaMemcpyAsync(d_ks, ks.data(), kb, cudaMemcpyHostToDevice, c0->stream));
  CUDA_TRY(c0, cudaMemcpyAsync(d_start, start.data(), sizeof(long long) * (n_ctx + 1), cudaMemcpyHostToDevice,
                               c0->stream));
  unsigned long long* d_queue = (unsigned long long*)(d_start + n_ctx + 1);
  CUDA_TRY(c0, cudaMemsetAsync(d_queue, 0, sizeof(unsigned long long), c0->stream));
  CUDA_TRY(c0, launch_vmc_multi<T>(d_ks, n_ctx, d_start, total, (T*)c0->multi_arena, ws, (int)grid, block,
                                   group_bytes, d_queue, smem, c0->stream));
  c0->last_multi_block = block;
  c0->launches += 1;
  std::vector<int> h(4 * n_ctx);
  for (int i = 0; i < n_ctx; ++i)
    CUDA_TRY(c0, cudaMemcpyAsync(&h[4 * i], cs[i]->d_status, 4 * sizeof(int), cudaMemcpyDeviceToHost, c0->stream));
  CUDA_TRY(c0, cudaStreamSynchronize(c0->stream));
  c0->last_svd_unconverged = 0;
  c0->last_phase_timeouts = 0;
  c0->last_tc_timeouts = 0;
  for (int i = 0; i < n_ctx; ++i) {
    c0->last_svd_unconverged += h[4 * i + ST_SVD];
    c0->last_phase_timeouts += h[4 * i + ST_PHASE_TIMEOUT];
    c0->last_tc_timeouts += h[4 * i + ST_TC_TIMEOUT];
  }
  for (int i = 0; i < n_ctx; ++i)
    if (h[4 * i + ST_GAUSS]) return fail(c0, GCF_EGAUSS, "a starting configuration violates the Gauss law");
  return svd_status(c0);
}

gcf_status dispatch(gcf_ctx* c, int mode, int want, int n, int n_sweeps, uint64_t seed, int8_t* cfg,
                    const gcf_samples* out, int* gauss, cudaStream_t stream = nullptr, bool async = false) {
  cudaStream_t st = async ? stream : c->stream;
  switch (c->kind) {
    case S_F32: return run_vmc<float>(c, mode, want, n, n_sweeps, seed, cfg, out, gauss, st, async);
    case S_F64: return run_vmc<double>(c, mode, want, n, n_sweeps, seed, cfg, out, gauss, st, async);
    case S_C64: return run_vmc<cfloat>(c, mode, want, n, n_sweeps, seed, cfg, out, gauss, st, async);
    default: return run_vmc<cdouble>(c, mode, want, n, n_sweeps, seed, cfg, out, gauss, st, async);
  }
}

// host SplitMix64 / Box-Muller normals (stream 0), same definition as the
// documented generator
double host_normal(uint64_t seed, uint64_t j) {
  const uint64_t key = stream_key(seed, 0);
  const double u0 = word_to_uniform(stream_word(key, 2 * j));
  const double u1 = word_to_uniform(stream_word(key, 2 * j + 1));
  return std::sqrt(-2.0 * std::log1p(-u0)) * std::cos(2.0 * 3.14159265358979323846 * u1);
}

gcf_status upload_params(gcf_ctx* c, const double* vals /* n_params or 2*n_params */) {
  const long long n = c->n_params;
  const bool cplx = c->m.dtype == GCF_COMPLEX;
  const long long nv = cplx ? 2 * n : n;
  for (long long i = 0; i < nv; ++i)
    if (!std::isfinite(vals[i])) return fail(c, GCF_ENUMERIC, "non-finite tensor entry");
  std::vector<char> buf(n * c->sbytes);
  if (c->kind == S_F32 || c->kind == S_C64) {
    float* f = (float*)buf.data();
    for (long long i = 0; i < nv; ++i) f[i] = (float)vals[i];
  } else {
    std::memcpy(buf.data(), vals, nv * sizeof(double));
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_params, buf.data(), buf.size(), cudaMemcpyHostToDevice, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return GCF_OK;
}

// Each group of SR buffers is (re)allocated as a whole: a group is marked
// ready (its last pointer set, or its capacity raised) only after every
// allocation in it succeeded, so a call after an allocation failure retries
// instead of running on missing buffers.
gcf_status ensure_sr(gcf_ctx* c, long long Ns, int n_chains) {
  if (!c->sr.part) {
    void** grp[12] = {(void**)&c->sr.obar, (void**)&c->sr.F, (void**)&c->sr.x, (void**)&c->sr.r,
                      (void**)&c->sr.p, (void**)&c->sr.Ap, (void**)&c->sr.z, (void**)&c->sr.dinv,
                      (void**)&c->sr.xf, (void**)&c->sr.tbar, (void**)&c->sr.scal, (void**)&c->sr.part};
    for (auto q : grp) {
      if (*q) cudaFree(*q);
      *q = nullptr;
    }
    const long long Np = c->n_params;
    cdouble** vecs[7] = {&c->sr.obar, &c->sr.F, &c->sr.x, &c->sr.r, &c->sr.p, &c->sr.Ap, &c->sr.z};
    for (auto v : vecs)
      if (!dalloc(v, sizeof(cdouble) * Np)) return fail(c, GCF_ENOMEM, "SR vectors");
    if (!dalloc(&c->sr.dinv, sizeof(double) * Np) ||
        !dalloc(&c->sr.xf, sizeof(float) * Np) ||
        !dalloc(&c->sr.tbar, sizeof(cdouble)) ||
        !dalloc(&c->sr.scal, 32 * sizeof(double)) ||
        !dalloc(&c->sr.part, sizeof(cdouble) * kSumParts))
      return fail(c, GCF_ENOMEM, "SR vectors");
  }
  if (!c->sr.pbs) {
    void** grp[4] = {(void**)&c->sr.seg, (void**)&c->sr.seg_v, (void**)&c->sr.seg_b, (void**)&c->sr.pbs};
    for (auto q : grp) {
      if (*q) cudaFree(*q);
      *q = nullptr;
    }
    int maxnb = 1;
    for (int v = 0; v < c->n_s; ++v) maxnb = std::max(maxnb, c->vnb[v]);
    std::vector<int> sv, sb;
    for (int v = 0; v < c->n_s; ++v)
      for (int b = 0; b < c->vnb[v]; ++b) { sv.push_back(v); sb.push_back(b); }
    c->sr.maxnb = maxnb;
    c->sr.n_seg = (int)sv.size();
    if (!dalloc(&c->sr.seg, sizeof(int) * ((size_t)c->n_s * (maxnb + 1) + 1)) ||
        !dalloc(&c->sr.seg_v, sizeof(int) * sv.size()) ||
        !dalloc(&c->sr.seg_b, sizeof(int) * sb.size()))
      return fail(c, GCF_ENOMEM, "SR segment tables");
    if (cudaMemcpy(c->sr.seg_v, sv.data(), sizeof(int) * sv.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(c->sr.seg_b, sb.data(), sizeof(int) * sb.size(), cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(c, GCF_ECUDA, "SR segment tables");
    std::vector<long long> pbs(c->n_s);
    long long acc = 0;
    for (int v = 0; v < c->n_s; ++v) { pbs[v] = acc; acc += c->vbs[v]; }
    c->sr_sum_bs = acc;
    c->sr.all_bs4 = 1;
    for (int v = 0; v < c->n_s; ++v)
      if (c->vbs[v] % 4) c->sr.all_bs4 = 0;
    long long* d_pbs = nullptr;
    if (!dalloc(&d_pbs, sizeof(long long) * c->n_s))
      return fail(c, GCF_ENOMEM, "SR segment tables");
    if (cudaMemcpy(d_pbs, pbs.data(), sizeof(long long) * c->n_s, cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaFree(d_pbs);
      return fail(c, GCF_ECUDA, "SR segment tables");
    }
    c->sr.pbs = d_pbs;
  }
  if (Ns > c->sr_ns_cap) {
    if (c->sr.t) cudaFree(c->sr.t);
    if (c->sr.coef) cudaFree(c->sr.coef);
    if (c->sr.perm) cudaFree(c->sr.perm);
    if (c->sr.osort) cudaFree(c->sr.osort);
    if (c->sr.coef_f) cudaFree(c->sr.coef_f);
    c->sr.t = c->sr.coef = nullptr;
    c->sr.perm = nullptr;
    c->sr.osort = nullptr;
    c->sr.coef_f = nullptr;
    c->sr_ns_cap = 0;
    if (!dalloc(&c->sr.t, sizeof(cdouble) * Ns) ||
        !dalloc(&c->sr.coef, sizeof(cdouble) * Ns) ||
        !dalloc(&c->sr.coef_f, sizeof(float) * Ns) ||
        !dalloc(&c->sr.perm, sizeof(int) * Ns * c->n_s) ||
        !dalloc(&c->sr.osort, c->sbytes * (size_t)Ns * c->sr_sum_bs))
      return fail(c, GCF_ENOMEM, "SR sample vectors");
    c->sr_ns_cap = Ns;
  }
  if (n_chains > c->sr_chain_cap) {
    if (c->sr.chain_mean) cudaFree(c->sr.chain_mean);
    c->sr.chain_mean = nullptr;
    c->sr_chain_cap = 0;
    if (!dalloc(&c->sr.chain_mean, sizeof(cdouble) * n_chains))
      return fail(c, GCF_ENOMEM, "SR chain means");
    c->sr_chain_cap = n_chains;
  }
  return GCF_OK;
}

}  // namespace

extern "C" {

gcf_status gcf_init_peps(const gcf_model* model, uint64_t seed, void* cuda_stream, gcf_ctx** out) {
  if (!model || !out) return GCF_EINVAL;
  *out = nullptr;
  const gcf_model& m = *model;
  if (m.N < 2 || m.N > 8 || m.Lx < 2 || m.Ly < 2 || m.Lx > MAX_L || m.Ly > MAX_L || m.D < m.N ||
      m.D % m.N != 0 || m.D / m.N > 3 || m.chi < 1 || (m.dtype != GCF_REAL && m.dtype != GCF_COMPLEX) ||
      m.precision < GCF_FP64 || m.precision > GCF_BF16 || (m.has_matter != 0 && m.has_matter != 1) ||
      m.trunc != GCF_TRUNC_SVD || m.recompute_env < -1 || m.recompute_env == 1 || m.recompute_env > m.Ly)
    return GCF_EINVAL;
  gcf_ctx* c = new gcf_ctx();
  c->m = m;
  c->m.Q = nullptr;
  c->Dk = m.D / m.N;
  c->P = m.has_matter ? 2 : 1;
  c->n_h = m.Ly * (m.Lx - 1);
  c->n_v = (m.Ly - 1) * m.Lx;
  c->n_s = m.Lx * m.Ly;
  c->cfg_len = c->n_h + c->n_v + c->n_s;
  c->n_plaq = (m.Lx - 1) * (m.Ly - 1);
  c->n_slots = 2 * c->n_plaq + (m.has_matter ? c->n_h + c->n_v : 0);
  c->Q.assign(c->n_s, 0);
  if (m.recompute_env == -1) {
    int K = 2;
    while (K * K < m.Ly + 1) ++K;
    c->ck_every = K;
  } else {
    c->ck_every = m.recompute_env;
  }
  if (m.Q)
    for (int i = 0; i < c->n_s; ++i) c->Q[i] = ((m.Q[i] % m.N) + m.N) % m.N;
  const bool cplx = m.dtype == GCF_COMPLEX;
  if (m.precision == GCF_FP64) { c->kind = cplx ? S_C128 : S_F64; c->sbytes = cplx ? 16 : 8; }
  else { c->kind = cplx ? S_C64 : S_F32; c->sbytes = cplx ? 8 : 4; }
  c->stream = (cudaStream_t)cuda_stream;
  // layout (Eqs. 6, 9): per vertex P * N^(k-1) blocks of D_k^k
  long long off = 0;
  for (int y = 0; y < m.Ly; ++y)
    for (int x = 0; x < m.Lx; ++x) {
      const int k = (x > 0) + (x < m.Lx - 1) + (y > 0) + (y < m.Ly - 1);
      int nb = c->P, bs = 1;
      for (int i = 0; i < k - 1; ++i) nb *= m.N;
      for (int i = 0; i < k; ++i) bs *= c->Dk;
      c->voff.push_back(off);
      c->vbs.push_back(bs);
      c->vnb.push_back(nb);
      off += (long long)nb * bs;
    }
  c->n_params = off;
  build_plan(c);
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device)) != cudaSuccess) {
    delete c;
    return GCF_ECUDA;
  }
  const int W = m.Lx + 1, R = m.Ly + 1;
  std::vector<int> tables;
  for (auto* v : {&c->plan.bondB, &c->plan.bondT, &c->plan.qrB, &c->plan.svdB, &c->plan.qrT, &c->plan.svdT})
    tables.insert(tables.end(), v->begin(), v->end());
  append_derived_tables(c, tables);
  c->tab_ints = (int)tables.size();
  bool ok = cudaMalloc(&c->d_params, c->n_params * c->sbytes) == cudaSuccess &&
            cudaMalloc(&c->d_Q, sizeof(int) * c->n_s) == cudaSuccess &&
            cudaMalloc(&c->d_voff, sizeof(long long) * c->n_s) == cudaSuccess &&
            cudaMalloc(&c->d_vbs, sizeof(int) * c->n_s) == cudaSuccess &&
            cudaMalloc(&c->d_vnb, sizeof(int) * c->n_s) == cudaSuccess &&
            cudaMalloc(&c->d_tables, sizeof(int) * tables.size()) == cudaSuccess &&
            cudaMalloc(&c->d_status, sizeof(int) * 4) == cudaSuccess;
  (void)W; (void)R;
  if (!ok) { gcf_destroy(c); return GCF_ENOMEM; }
  if (cudaMemcpy(c->d_Q, c->Q.data(), sizeof(int) * c->n_s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_voff, c->voff.data(), sizeof(long long) * c->n_s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_vbs, c->vbs.data(), sizeof(int) * c->n_s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_vnb, c->vnb.data(), sizeof(int) * c->n_s, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(c->d_tables, tables.data(), sizeof(int) * tables.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
    gcf_destroy(c);
    return GCF_ECUDA;
  }
  // N(0,1) initial tensors from the documented counter-based generator
  const long long nv = cplx ? 2 * c->n_params : c->n_params;
  std::vector<double> vals(nv);
  for (long long i = 0; i < nv; ++i) vals[i] = host_normal(seed, (uint64_t)i);
  if (upload_params(c, vals.data()) != GCF_OK) { gcf_destroy(c); return GCF_ECUDA; }
  *out = c;
  return GCF_OK;
}

void gcf_destroy(gcf_ctx* c) {
  if (!c) return;
  void* ptrs[] = {c->d_params, c->d_Q, c->d_voff, c->d_vbs, c->d_vnb, c->d_tables, c->d_status,
                  c->d_scratch, c->sr.obar, c->sr.F, c->sr.x, c->sr.r, c->sr.p, c->sr.Ap, c->sr.z, c->sr.dinv,
                  c->sr.t, c->sr.coef, c->sr.chain_mean, c->sr.tbar, c->sr.scal, c->sr.perm, c->sr.seg,
                  c->sr.pbs, c->sr.osort, c->sr.xf, c->sr.coef_f, c->sr.part,
                  c->sr.seg_v, c->sr.seg_b, c->d_cfg, c->d_e,
                  c->d_la, c->d_ph, c->d_bid, c->d_O, c->d_acc, c->vjp_bid, c->vjp_O, c->vjp_coef,
                  c->vjp_acc, c->multi_arena, c->multi_tab};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete c;
}

const char* gcf_last_error(const gcf_ctx* c) { return c ? c->err.c_str() : "null context"; }
int64_t gcf_num_params(const gcf_ctx* c) { return c ? c->n_params : -1; }
int gcf_config_len(const gcf_ctx* c) { return c ? c->cfg_len : -1; }
int gcf_scalar_bytes(const gcf_ctx* c) { return c ? (int)c->sbytes : -1; }
int64_t gcf_launch_count(const gcf_ctx* c) { return c ? c->launches : -1; }

int gcf_executor(const gcf_ctx* ctx) { return ctx ? ctx->exec : -1; }

gcf_status gcf_set_tensors(gcf_ctx* c, const void* host, size_t bytes) {
  if (!c || !host) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_set_tensors");
  const bool cplx = c->m.dtype == GCF_COMPLEX;
  if (bytes != (size_t)c->n_params * (cplx ? 16 : 8))
    return fail(c, GCF_EINVAL, "gcf_set_tensors: byte count does not match the layout");
  return upload_params(c, (const double*)host);
}

gcf_status gcf_get_tensors(gcf_ctx* c, void* host, size_t bytes) {
  if (!c || !host) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_get_tensors");
  const bool cplx = c->m.dtype == GCF_COMPLEX;
  const long long nv = cplx ? 2 * c->n_params : c->n_params;
  if (bytes != (size_t)nv * 8) return fail(c, GCF_EINVAL, "gcf_get_tensors: byte count mismatch");
  std::vector<char> buf(c->n_params * c->sbytes);
  CUDA_TRY(c, cudaMemcpyAsync(buf.data(), c->d_params, buf.size(), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  double* d = (double*)host;
  if (c->kind == S_F32 || c->kind == S_C64) {
    const float* f = (const float*)buf.data();
    for (long long i = 0; i < nv; ++i) d[i] = f[i];
  } else {
    std::memcpy(d, buf.data(), nv * sizeof(double));
  }
  return GCF_OK;
}

gcf_status gcf_init_configs(gcf_ctx* c, int n_chains, const int8_t* occ, const int8_t* powers,
                            int8_t* configs) {
  if (!c || n_chains < 0 || (n_chains > 0 && !configs)) return GCF_EINVAL;
  if (n_chains == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_init_configs");
  CUDA_TRY(c, cudaMemsetAsync(c->d_status, 0, 4 * sizeof(int), c->stream));
  CUDA_TRY(c, launch_init_configs(c->m.N, c->m.Lx, c->m.Ly, c->m.has_matter, c->d_Q, n_chains, occ,
                                  powers, configs, c->d_status, c->stream));
  c->launches += 1;
  int st[4];
  CUDA_TRY(c, cudaMemcpyAsync(st, c->d_status, sizeof(st), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (st[0]) return fail(c, GCF_EGAUSS, "occupations violate sum(p) = sum(Q) mod N");
  return GCF_OK;
}

gcf_status gcf_amplitude(gcf_ctx* c, int n, const int8_t* configs, double* log_abs, double* phase) {
  if (!c || n < 0 || (n > 0 && (!configs || !log_abs || !phase))) return GCF_EINVAL;
  if (n == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_amplitude");
  gcf_samples out{};
  out.log_abs = log_abs;
  out.phase = phase;
  gcf_status st = dispatch(c, 0, WANT_AMP, n, 1, 0, (int8_t*)configs, &out, nullptr);
  if (st != GCF_OK) return st;
  return svd_status(c);
}

gcf_status gcf_local_energy(gcf_ctx* c, int n, const int8_t* configs, double* e_loc) {
  if (!c || n < 0 || (n > 0 && (!configs || !e_loc))) return GCF_EINVAL;
  if (n == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_local_energy");
  gcf_samples out{};
  out.e_loc = e_loc;
  int gauss = 0;
  gcf_status st = dispatch(c, 0, WANT_ELOC, n, 1, 0, (int8_t*)configs, &out, &gauss);
  if (st != GCF_OK) return st;
  if (gauss) return fail(c, GCF_EGAUSS, "configuration violates the Gauss law");
  return svd_status(c);
}

gcf_status gcf_log_grad(gcf_ctx* c, int n, const int8_t* configs, int32_t* block_ids, void* O) {
  if (!c || n < 0 || (n > 0 && (!configs || !block_ids || !O))) return GCF_EINVAL;
  if (n == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_log_grad");
  gcf_samples out{};
  out.block_ids = block_ids;
  out.O = O;
  int gauss = 0;
  gcf_status st = dispatch(c, 0, WANT_GRAD, n, 1, 0, (int8_t*)configs, &out, &gauss);
  if (st != GCF_OK) return st;
  if (gauss) return fail(c, GCF_EGAUSS, "configuration violates the Gauss law");
  return svd_status(c);
}

gcf_status gcf_log_grad_vjp(gcf_ctx* c, int n, const int8_t* configs, const double* weights, double* grad) {
  if (!c || n < 0 || !grad || (n > 0 && (!configs || !weights))) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_log_grad_vjp");
  const bool cplx = c->m.dtype == GCF_COMPLEX;
  if (n == 0) {
    CUDA_TRY(c, cudaMemsetAsync(grad, 0, sizeof(double) * (cplx ? 2 : 1) * c->n_params, c->stream));
    return GCF_OK;
  }
  const long long D4 = (long long)c->Dk * c->Dk * c->Dk * c->Dk;
  if (n > c->vjp_cap) {
    cudaFree(c->vjp_bid); cudaFree(c->vjp_O); cudaFree(c->vjp_coef);
    c->vjp_bid = nullptr; c->vjp_O = nullptr; c->vjp_coef = nullptr; c->vjp_cap = 0;
    if (cudaMalloc(&c->vjp_bid, sizeof(int) * (size_t)n * c->n_s) != cudaSuccess ||
        cudaMalloc(&c->vjp_O, c->sbytes * (size_t)n * c->n_s * D4) != cudaSuccess ||
        cudaMalloc(&c->vjp_coef, sizeof(cdouble) * (size_t)n) != cudaSuccess)
      return fail(c, GCF_ENOMEM, "log_grad_vjp buffers");
    c->vjp_cap = n;
  }
  if (!c->vjp_acc && !dalloc(&c->vjp_acc, sizeof(cdouble) * c->n_params))
    return fail(c, GCF_ENOMEM, "log_grad_vjp buffers");
  gcf_samples out{};
  out.block_ids = c->vjp_bid;
  out.O = c->vjp_O;
  int gauss = 0;
  gcf_status st = dispatch(c, 0, WANT_GRAD, n, 1, 0, (int8_t*)configs, &out, &gauss);
  if (st != GCF_OK) return st;
  if (gauss) return fail(c, GCF_EGAUSS, "configuration violates the Gauss law");
  SrGeom g{};
  g.Np = c->n_params; g.Ns = n; g.n_s = c->n_s; g.D4 = (int)D4;
  g.voff = c->d_voff; g.vbs = c->d_vbs; g.vnb = c->d_vnb;
  int mx = 1;
  for (int v = 0; v < c->n_s; ++v) mx = std::max(mx, c->vbs[v] * c->vnb[v]);
  g.max_nb_bs = mx;
  cudaError_t e;
  switch (c->kind) {
    case S_F32:
      e = log_grad_vjp<float>(g, c->vjp_bid, c->vjp_O, weights, cplx, c->vjp_coef, c->vjp_acc, grad, c->stream,
                              &c->launches);
      break;
    case S_F64:
      e = log_grad_vjp<double>(g, c->vjp_bid, c->vjp_O, weights, cplx, c->vjp_coef, c->vjp_acc, grad, c->stream,
                               &c->launches);
      break;
    case S_C64:
      e = log_grad_vjp<cfloat>(g, c->vjp_bid, c->vjp_O, weights, cplx, c->vjp_coef, c->vjp_acc, grad, c->stream,
                               &c->launches);
      break;
    default:
      e = log_grad_vjp<cdouble>(g, c->vjp_bid, c->vjp_O, weights, cplx, c->vjp_coef, c->vjp_acc, grad,
                                c->stream, &c->launches);
      break;
  }
  CUDA_TRY(c, e);
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return svd_status(c);
}

gcf_status gcf_autotune(gcf_ctx* c, int n_chains, int n_sweeps, const int8_t* configs, double* ms, int* n_forms) {
  if (!c || n_chains < 1 || n_sweeps < 1 || !configs) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_autotune");
  // candidate forms that fit an SM (227 KB of shared memory per block)
  const size_t limit = 227 * 1024 - 8 * 1024;
  std::vector<std::pair<int, int>> forms;
  for (int lv = 0; lv <= 3; ++lv) {
    const size_t cta = cta_smem_bytes(c->plan, lv, c->sbytes);
    if (cta <= limit) forms.push_back({EXEC_CTA, lv});
    const size_t grp = 2 * group_smem_bytes(c->plan, lv, c->sbytes);
    if (lv >= 1 && grp <= limit) forms.push_back({EXEC_GROUP, lv});
    if (lv >= 1 && 2 * grp <= limit) forms.push_back({EXEC_GROUP4, lv});
  }
  const int keep_exec = c->exec, keep_cta = c->plan.cta_level, keep_grp = c->plan.group_level;
  const size_t bytes = (size_t)n_chains * c->cfg_len;
  int8_t* work = nullptr;
  double* la = nullptr;
  if (cudaMalloc(&work, bytes) != cudaSuccess || cudaMalloc(&la, sizeof(double) * (size_t)n_chains * n_sweeps) != cudaSuccess) {
    cudaFree(work);
    return fail(c, GCF_ENOMEM, "autotune buffers");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  gcf_samples out{};
  out.log_abs = la;
  double best = 1e300;
  int best_i = -1;
  gcf_status st = GCF_OK;
  for (size_t i = 0; i < forms.size() && st == GCF_OK; ++i) {
    set_form(c, forms[i].first, forms[i].second);
    double t = 1e300;
    for (int rep = 0; rep < 2 && st == GCF_OK; ++rep) {  // first run warms up
      if (cudaMemcpyAsync(work, configs, bytes, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
        st = fail(c, GCF_ECUDA, "autotune copy");
        break;
      }
      cudaEventRecord(e0, c->stream);
      int gauss = 0;
      const gcf_status r = dispatch(c, 1, WANT_AMP, n_chains, n_sweeps, 1, work, &out, &gauss);
      cudaEventRecord(e1, c->stream);
      cudaEventSynchronize(e1);
      if (r == GCF_EINVAL || r == GCF_ECUDA) { t = 1e300; c->err.clear(); break; }  // form does not launch
      if (r != GCF_OK) { st = r; break; }
      if (gauss) { st = fail(c, GCF_EGAUSS, "configuration violates the Gauss law"); break; }
      float f = 0.f;
      cudaEventElapsedTime(&f, e0, e1);
      t = f;
    }
    if (ms && n_forms && (int)i < *n_forms) ms[i] = t;
    if (t < best) { best = t; best_i = (int)i; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(work);
  cudaFree(la);
  if (n_forms) *n_forms = (int)forms.size();
  // restore the planned levels of both executors, then take the winner
  c->plan.cta_level = keep_cta;
  c->plan.group_level = keep_grp;
  set_form(c, EXEC_CTA, keep_cta);
  set_form(c, EXEC_GROUP, keep_grp);
  c->exec = keep_exec;
  if (st != GCF_OK) return st;
  if (best_i < 0) return fail(c, GCF_ECUDA, "no kernel form launched");
  set_form(c, forms[best_i].first, forms[best_i].second);
  return GCF_OK;
}

int gcf_phase_timeouts(const gcf_ctx* c) { return c ? c->last_phase_timeouts : -1; }

int gcf_svd_unconverged(const gcf_ctx* c) { return c ? c->last_svd_unconverged : -1; }

int64_t gcf_scratch_bytes_per_chain(const gcf_ctx* c) {
  return c ? (int64_t)c->plan.ws_stride * (int64_t)c->sbytes : -1;
}

int gcf_checkpoint_interval(const gcf_ctx* c) { return c ? c->ck_every : -1; }

int gcf_tensor_core_form(const gcf_ctx* c) { return c ? (c->plan.tc_bytes > 0 ? 1 : 0) : -1; }

int gcf_tensor_timeouts(const gcf_ctx* c) { return c ? c->last_tc_timeouts : -1; }

int gcf_multi_chains_per_cta(const gcf_ctx* c) {
  return c ? (c->last_multi_block == 512 ? 4 : c->last_multi_block == 256 ? 1 : 0) : -1;
}

gcf_status gcf_set_svd_sweeps(gcf_ctx* c, int max_sweeps) {
  if (!c || max_sweeps < 1 || max_sweeps > 1000) return GCF_EINVAL;
  c->svd_sweeps = max_sweeps;
  return GCF_OK;
}

int gcf_smem_level(const gcf_ctx* c) {
  if (!c) return -1;
  return grouped(c) ? c->plan.group_level : c->plan.cta_level;
}

gcf_status gcf_sample_multi(gcf_ctx* const* ctxs, int n_ctx, const int* n_chains, int n_sweeps,
                            const uint64_t* seeds, int8_t* const* configs, const gcf_samples* outs) {
  if (!ctxs || n_ctx < 1 || !n_chains || !seeds || !configs || n_sweeps < 1) return GCF_EINVAL;
  gcf_ctx* c0 = ctxs[0];
  if (!c0) return GCF_EINVAL;
  for (int i = 0; i < n_ctx; ++i) {
    if (!ctxs[i] || n_chains[i] < 0 || (n_chains[i] > 0 && !configs[i])) return fail(c0, GCF_EINVAL, "bad argument");
    if (ctxs[i]->kind != c0->kind) return fail(c0, GCF_EINVAL, "contexts differ in scalar type");
    if (ctxs[i]->device != c0->device) return fail(c0, GCF_EINVAL, "contexts on different devices");
  }
  DEVICE_TRY(c0, "gcf_sample_multi");
  // the other contexts' work (parameter uploads) precedes this launch
  for (int i = 1; i < n_ctx; ++i)
    if (ctxs[i]->stream != c0->stream) CUDA_TRY(c0, cudaStreamSynchronize(ctxs[i]->stream));
  switch (c0->kind) {
    case S_F32: return run_multi<float>(ctxs, n_ctx, n_chains, n_sweeps, seeds, configs, outs);
    case S_F64: return run_multi<double>(ctxs, n_ctx, n_chains, n_sweeps, seeds, configs, outs);
    case S_C64: return run_multi<cfloat>(ctxs, n_ctx, n_chains, n_sweeps, seeds, configs, outs);
    default: return run_multi<cdouble>(ctxs, n_ctx, n_chains, n_sweeps, seeds, configs, outs);
  }
}

gcf_status gcf_sample_batch_async(gcf_ctx* c, int n_chains, int n_sweeps, uint64_t seed, int8_t* configs,
                                  const gcf_samples* out, void* stream) {
  if (!c || n_chains < 0 || n_sweeps < 1 || (n_chains > 0 && !configs)) return GCF_EINVAL;
  if (n_chains == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_sample_batch_async");
  cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
  // scratch must already cover this launch: no allocation here
  {
    const bool grp = grouped(c);
    const int W = n_groups(c);
    long long slots = 1;
    if (grp) {
      int per_sm = 0;
      switch (c->kind) {
        case S_F32: per_sm = occupancy_vmc_grouped<float>(128 * W, W * c->plan.group_smem); break;
        case S_F64: per_sm = occupancy_vmc_grouped<double>(128 * W, W * c->plan.group_smem); break;
        case S_C64: per_sm = occupancy_vmc_grouped<cfloat>(128 * W, W * c->plan.group_smem); break;
        default: per_sm = occupancy_vmc_grouped<cdouble>(128 * W, W * c->plan.group_smem); break;
      }
      const long long sl = balanced_slots(n_chains, (long long)c->sms * std::max(1, per_sm) * W);
      slots = (sl + W - 1) / W * W;
    } else {
      slots = grid_for(c, n_chains);
    }
    if (slots > c->scratch_ctas)
      return fail(c, GCF_EINVAL, "gcf_sample_batch_async: scratch not yet sized for this many chains; call "
                                 "gcf_sample_batch with at least as many chains first");
  }
  gcf_samples o{};
  if (out) o = *out;
  int want = (o.log_abs || o.phase ? WANT_AMP : 0) | (o.e_loc ? WANT_ELOC : 0) |
             (o.O || o.block_ids ? WANT_GRAD : 0);
  return dispatch(c, 1, want, n_chains, n_sweeps, seed, configs, &o, nullptr, st, true);
}

gcf_status gcf_sample_batch(gcf_ctx* c, int n_chains, int n_sweeps, uint64_t seed, int8_t* configs,
                            const gcf_samples* out) {
  if (!c || n_chains < 0 || n_sweeps < 1 || (n_chains > 0 && !configs)) return GCF_EINVAL;
  if (n_chains == 0) return GCF_OK;
  DEVICE_TRY(c, "gcf_sample_batch");
  gcf_samples o{};
  if (out) o = *out;
  int want = (o.log_abs || o.phase ? WANT_AMP : 0) | (o.e_loc ? WANT_ELOC : 0) |
             (o.O || o.block_ids ? WANT_GRAD : 0);
  int gauss = 0;
  gcf_status st = dispatch(c, 1, want, n_chains, n_sweeps, seed, configs, &o, &gauss);
  if (st != GCF_OK) return st;
  if (gauss) return fail(c, GCF_EGAUSS, "starting configuration violates the Gauss law");
  return svd_status(c);
}

gcf_status gcf_sr_step(gcf_ctx* c, int n_samples, int n_chains, const double* e_loc,
                       const int32_t* block_ids, const void* O, double diag_shift, double lr,
                       int mode, double dt, int max_iter, double tol, double* stats) {
  if (!c || n_samples < 1 || n_chains < 1 || n_samples % n_chains != 0 || !e_loc || !block_ids ||
      !O || !stats || max_iter < 0 || !(diag_shift >= 0.0))
    return GCF_EINVAL;
  if (mode != GCF_SR && mode != GCF_TDVP_STAGE1 && mode != GCF_TDVP_STAGE2) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_sr_step");
  if (mode != GCF_SR && c->m.dtype != GCF_COMPLEX)
    return fail(c, GCF_EINVAL, "TDVP modes need complex tensors");
  gcf_status st = ensure_sr(c, n_samples, n_chains);
  if (st != GCF_OK) return st;
  double cr = -lr, ci = 0.0;
  if (mode != GCF_SR) {
    // A += c_k dt (-i x), c_{1,2} = (1 +- i)/2  ->  coefficient c_k * dt * (-i)
    const double sgn = mode == GCF_TDVP_STAGE1 ? 1.0 : -1.0;
    const double kr = 0.5 * dt, ki = 0.5 * sgn * dt;  // c_k dt
    cr = ki;    // (kr + i ki)(-i) = ki - i kr
    ci = -kr;
  }
  SrGeom g{};
  g.Np = c->n_params; g.Ns = n_samples; g.n_s = c->n_s;
  g.D4 = c->Dk * c->Dk * c->Dk * c->Dk;
  g.voff = c->d_voff; g.vbs = c->d_vbs; g.vnb = c->d_vnb;
  int mx = 1;
  for (int v = 0; v < c->n_s; ++v) mx = std::max(mx, c->vbs[v] * c->vnb[v]);
  g.max_nb_bs = mx;
  cudaError_t e;
  switch (c->kind) {
    case S_F32:
      e = sr_solve_update<float>(g, c->sr, e_loc, block_ids, O, c->d_params, n_chains, diag_shift, cr, ci,
                                 max_iter, tol, stats, c->stream, &c->launches);
      break;
    case S_F64:
      e = sr_solve_update<double>(g, c->sr, e_loc, block_ids, O, c->d_params, n_chains, diag_shift, cr, ci,
                                  max_iter, tol, stats, c->stream, &c->launches);
      break;
    case S_C64:
      e = sr_solve_update<cfloat>(g, c->sr, e_loc, block_ids, O, c->d_params, n_chains, diag_shift, cr, ci,
                                  max_iter, tol, stats, c->stream, &c->launches);
      break;
    default:
      e = sr_solve_update<cdouble>(g, c->sr, e_loc, block_ids, O, c->d_params, n_chains, diag_shift, cr, ci,
                                   max_iter, tol, stats, c->stream, &c->launches);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "gcf_sr_step");
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (stats[6] == 0.0 && max_iter > 0) return fail(c, GCF_ETIMEOUT, "CG reached max_iter before tol");
  return GCF_OK;
}

gcf_status gcf_vmc_step_host(gcf_ctx* c, int n_chains, int n_sweeps, uint64_t seed, int8_t* host_configs,
                             double diag_shift, double lr, int mode, double dt, int max_iter, double tol,
                             double* stats) {
  if (!c || n_chains < 1 || n_sweeps < 1 || !host_configs || !stats) return GCF_EINVAL;
  DEVICE_TRY(c, "gcf_vmc_step_host");
  const long long ns = (long long)n_chains * n_sweeps;
  const int D4 = c->Dk * c->Dk * c->Dk * c->Dk;
  if (ns > c->e2e_cap || n_chains > c->e2e_chains) {
    void* ptrs[] = {c->d_cfg, c->d_e, c->d_la, c->d_ph, c->d_bid, c->d_O, c->d_acc};
    for (void* p : ptrs)
      if (p) cudaFree(p);
    c->d_cfg = nullptr; c->d_e = c->d_la = c->d_ph = nullptr; c->d_bid = c->d_acc = nullptr;
    c->d_O = nullptr;
    c->e2e_cap = 0;
    c->e2e_chains = 0;
    bool ok = cudaMalloc(&c->d_cfg, (size_t)n_chains * c->cfg_len) == cudaSuccess &&
              cudaMalloc(&c->d_e, sizeof(double) * 2 * ns) == cudaSuccess &&
              cudaMalloc(&c->d_la, sizeof(double) * ns) == cudaSuccess &&
              cudaMalloc(&c->d_ph, sizeof(double) * ns) == cudaSuccess &&
              cudaMalloc(&c->d_bid, sizeof(int) * ns * c->n_s) == cudaSuccess &&
              cudaMalloc(&c->d_O, c->sbytes * ns * c->n_s * D4) == cudaSuccess &&
              cudaMalloc(&c->d_acc, sizeof(int) * 2 * n_chains) == cudaSuccess;
    if (!ok) return fail(c, GCF_ENOMEM, "e2e sample buffers");
    c->e2e_cap = ns;
    c->e2e_chains = n_chains;
  }
  CUDA_TRY(c, cudaMemcpyAsync(c->d_cfg, host_configs, (size_t)n_chains * c->cfg_len,
                              cudaMemcpyHostToDevice, c->stream));
  gcf_samples o{};
  o.log_abs = c->d_la; o.phase = c->d_ph; o.e_loc = c->d_e; o.block_ids = c->d_bid; o.O = c->d_O;
  o.accepted = c->d_acc; o.proposed = c->d_acc + n_chains;
  gcf_status st = gcf_sample_batch(c, n_chains, n_sweeps, seed, c->d_cfg, &o);
  if (st != GCF_OK) return st;
  st = gcf_sr_step(c, (int)ns, n_chains, c->d_e, c->d_bid, c->d_O, diag_shift, lr, mode, dt, max_iter,
                   tol, stats);
  if (st != GCF_OK && st != GCF_ETIMEOUT) return st;
  CUDA_TRY(c, cudaMemcpyAsync(host_configs, c->d_cfg, (size_t)n_chains * c->cfg_len,
                              cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  return st;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// gcf_amplitude_noalloc: scratch from a fixed device array instead of
// cudaMalloc.  In host code g_noalloc_scratch / g_noalloc_status name host-side
// stand-ins, not device addresses: the kernel is given the address returned
// by cudaGetSymbolAddress, looked up once per device with that device current.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_scratch_ptr[kMaxDevices] = {};
int* g_noalloc_status_ptr[kMaxDevices] = {};
}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static __device__ __align__(256) int g_noalloc_status[4];

namespace {
gcf_status noalloc_setup(gcf_ctx* c, void** scratch, int** status) {
  int dev = -1;
  CUDA_TRY(c, cudaGetDevice(&dev));
  if (dev != c->device || dev < 0 || dev >= kMaxDevices)
    return fail(c, GCF_EINVAL, "gcf_amplitude_noalloc: the context's device must be current");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_scratch_ptr[dev]) {
    void* p = nullptr;
    void* q = nullptr;
    CUDA_TRY(c, cudaGetSymbolAddress(&p, g_noalloc_scratch));
    CUDA_TRY(c, cudaGetSymbolAddress(&q, g_noalloc_status));
    g_noalloc_scratch_ptr[dev] = p;
    g_noalloc_status_ptr[dev] = (int*)q;
  }
  *scratch = g_noalloc_scratch_ptr[dev];
  *status = g_noalloc_status_ptr[dev];
  return GCF_OK;
}

template <class T>
gcf_status amplitude_noalloc_impl(gcf_ctx* c, int n, const int8_t* configs, double* log_abs,
                                  double* phase, void* scratch, int* status) {
  const size_t per_cta = (size_t)c->plan.ws_stride * c->sbytes;
  const long long fit = (long long)(kNoAllocScratchBytes / per_cta);
  if (fit < 1) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "gcf_amplitude_noalloc: lattice needs %zu bytes of scratch per CTA, above the "
                  "fixed 33554432-byte array",
                  per_cta);
    return fail(c, GCF_EINVAL, msg);
  }
  const int grid = (int)std::max<long long>(1, std::min<long long>(fit, grid_for(c, n)));
  KParams<T> k = make_params<T>(c);
  k.scratch = (T*)scratch;
  k.status = status;
  k.n_chains = n; k.n_sweeps = 1; k.mode = 0; k.want = WANT_AMP; k.seed = 0;
  k.configs = (int8_t*)configs;
  k.log_abs = log_abs;
  k.phase = phase;
  // the status counters start at zero for every call (the array keeps the
  // previous call's values otherwise); the kernel writes every scratch word
  // it reads before reading it
  CUDA_TRY(c, cudaMemsetAsync(status, 0, 4 * sizeof(int), c->stream));
  CUDA_TRY(c, launch_vmc<T>(k, grid, 256, c->plan.dyn_smem, c->stream));
  c->launches += 1;
  return GCF_OK;
}
}  // namespace

extern "C" gcf_status gcf_amplitude_noalloc(gcf_ctx* c, int n, const int8_t* configs, double* log_abs,
                                            double* phase) {
  if (!c || n < 0 || (n > 0 && (!configs || !log_abs || !phase))) return GCF_EINVAL;
  if (n == 0) return GCF_OK;
  void* scratch = nullptr;
  int* status = nullptr;
  gcf_status st = noalloc_setup(c, &scratch, &status);
  if (st != GCF_OK) return st;
  switch (c->kind) {
    case S_F32: return amplitude_noalloc_impl<float>(c, n, configs, log_abs, phase, scratch, status);
    case S_F64: return amplitude_noalloc_impl<double>(c, n, configs, log_abs, phase, scratch, status);
    case S_C64: return amplitude_noalloc_impl<cfloat>(c, n, configs, log_abs, phase, scratch, status);
    default: return amplitude_noalloc_impl<cdouble>(c, n, configs, log_abs, phase, scratch, status);
  }
}


