/*
 * gcfvmc.h - C ABI of the GB300 library for variational Monte Carlo of
 * gauge-canonical-form (GCF) gauge-invariant PEPS for Z_N lattice gauge
 * theories in (2+1)D, following Wu & Liu, "Accurate gauge-invariant tensor
 * network simulations for Abelian lattice gauge theory in (2+1)D".
 *
 * Library: libgcfvmc.so (hand-written CUDA for sm_103a).  No torch types
 * appear here; the Python binding passes raw pointers, after checking each
 * buffer's shape, dtype, size and placement (the library cannot).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Lattice: open Lx x Ly square lattice, vertex (x, y), x to the right,
 *   y up.  Horizontal link (x,1) joins (x,y)-(x+1,y); vertical link (x,2)
 *   joins (x,y)-(x,y+1).
 * - Configuration (int8, cfg_len = Ly*(Lx-1) + (Ly-1)*Lx + Lx*Ly bytes per
 *   chain): [h: Ly x (Lx-1), row-major][v: (Ly-1) x Lx][p: Ly x Lx], link
 *   values in [0, N), occupations in {0,1} (0 without matter).  A
 *   configuration is physical iff every vertex satisfies the Gauss law
 *   p + n_l + n_d - n_r - n_u = Q_x (mod N)   (paper Eq. 1 and Eq. S4).
 * - Parameters: the GCF matter tensors A^p_{lrdu} (Eqs. 6 and 9), stored
 *   block-sparse.  Vertex v = y*Lx + x in order.  At a vertex the existing
 *   legs in the order (l, r, d, u) are legs[0..k-1]; block index =
 *   mixed radix (p, n_legs[0], ..., n_legs[k-2]) with p most significant and
 *   radix N for the charges; the last leg's charge follows from the Gauss
 *   law.  P = 2 occupation values with matter, 1 without.  A block holds
 *   D_k^k entries [i_l][i_r][i_d][i_u] over the existing legs, row-major.
 *   D_k = D / N (every charge sector has the same degeneracy).
 * - Pointers documented "device" are CUDA device pointers, read/written in
 *   order on the context's stream; "host" pointers are ordinary memory.
 *   The caller owns every buffer it passes; the context owns its own
 *   parameter store and scratch.
 * - Every entry point returns a gcf_status and never aborts; on failure the
 *   reason is available from gcf_last_error().  Calls on one context are not
 *   thread-safe.
 * - The device that was current at gcf_init_peps is the context's device; every
 *   later call on the context must be made with that device current, else it
 *   returns GCF_EINVAL and launches nothing (a launch with another device
 *   current would run on that device against this context's memory).
 * - Truncated bonds are cut with a one-sided Jacobi SVD that stops after a
 *   sweep limit (40 by default, gcf_set_svd_sweeps).  A synchronous call in
 *   which some SVD reached the limit before converging still writes all its
 *   outputs but returns GCF_ETIMEOUT (gcf_svd_unconverged gives the count):
 *   those outputs may be less accurate than the contraction's precision.
 * - A batch of zero configurations or chains is valid wherever a count may
 *   be 0 (gcf_init_configs, gcf_amplitude, gcf_amplitude_noalloc,
 *   gcf_local_energy, gcf_log_grad, gcf_log_grad_vjp, gcf_sample_batch,
 *   gcf_sample_batch_async, contexts of gcf_sample_multi): the call returns
 *   GCF_OK without launching a kernel, its configuration and per-sample
 *   pointers may be NULL, and it writes nothing (gcf_log_grad_vjp writes a
 *   zero gradient to grad, which must be valid).  An SR step
 *   (gcf_sr_step, gcf_vmc_step_host) needs at least one sample.
 */
#ifndef GCFVMC_H
#define GCFVMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GCF_API_VERSION 1

typedef struct gcf_ctx gcf_ctx;

typedef enum {
  GCF_OK = 0,
  GCF_EINVAL = 1,    /* invalid argument (sizes, null pointers, bad enum)   */
  GCF_ENOMEM = 2,    /* device or host allocation failed                    */
  GCF_ECUDA = 3,     /* a CUDA runtime call or kernel launch failed         */
  GCF_EGAUSS = 4,    /* an input configuration violates the Gauss law       */
  GCF_ENUMERIC = 5,  /* non-finite value met (NaN/Inf tensors, zero psi)    */
  GCF_ETIMEOUT = 6   /* a bounded iterative routine did not converge        */
} gcf_status;

/* tensor element type */
enum { GCF_REAL = 0, GCF_COMPLEX = 1 };
/* contraction precision: FP64 (reference form), FP32 (plain CUDA-core form),
 * TF32 / BF16 (tensor-core operand rounding with FP32 accumulation). */
enum { GCF_FP64 = 0, GCF_FP32 = 1, GCF_TF32 = 2, GCF_BF16 = 3 };
/* parameter update of gcf_sr_step */
enum { GCF_SR = 0, GCF_TDVP_STAGE1 = 1, GCF_TDVP_STAGE2 = 2 };
/* truncation of the boundary MPS (gcf_model.trunc): the SVD sweep of
 * Sec. S-2 (QR left to right, then LQ / truncated SVD right to left).  A
 * randomized range finder is not built; any other value is GCF_EINVAL. */
enum { GCF_TRUNC_SVD = 0 };

/* Model and ansatz.  Couplings are in the paper's form, Eqs. (2)-(5):
 *   H = m sum_x p_x + J sum (c^dag U c + h.c.) - h sum_x (P_x + P_x^dag)
 *       + g sum_links (2 - 2 cos(2 pi n / N));
 * for N = 2, P_x = P_x^dag so the magnetic term is -2h P_x.  J is real. */
typedef struct {
  int N;            /* gauge group Z_N, 2 <= N <= 8                          */
  int Lx, Ly;       /* 2 <= Lx, Ly <= 64                                     */
  int D;            /* total bond dimension, multiple of N; D_k = D/N <= 3   */
  int chi;          /* boundary-MPS cutoff, >= 1                              */
  int has_matter;   /* 1: hard-core bosons on the vertices                   */
  const int32_t* Q; /* host, Lx*Ly background charges (row-major) or NULL=0  */
  double h, g, J, m;
  int dtype;        /* GCF_REAL | GCF_COMPLEX                                */
  int precision;    /* GCF_FP64 | GCF_FP32 | GCF_TF32 | GCF_BF16             */
  int trunc;        /* GCF_TRUNC_SVD                                         */
  int recompute_env;/* boundary-MPS store of each chain: 0 keeps every B[r]
                       and T[r]; K in [2, Ly] keeps every K-th and recomputes
                       the ones between from the kept one when a pass needs
                       them (main-text cost paragraph: environments
                       recomputed instead of stored when chi is large);
                       -1 takes K = ceil(sqrt(Ly + 1)).  Results are the
                       same bit for bit; the store shrinks from 2(Ly+1)
                       MPS to about 2(Ly/K + K), and every pass absorbs
                       up to one extra row per row it visits.            */
} gcf_model;

/* Measurement outputs of gcf_sample_batch (all device pointers, chain-major:
 * sample s = chain * n_sweeps + sweep).  Any member may be NULL to skip it. */
typedef struct {
  double* log_abs;    /* [n_samples]   log|psi(s)|                           */
  double* phase;      /* [n_samples]   arg psi(s) (0 or pi for real tensors) */
  double* e_loc;      /* [2*n_samples] (re, im) of E_loc(s), Eq. S2          */
  int32_t* block_ids; /* [n_samples*Lx*Ly] block selected at each vertex     */
  void* O;            /* [n_samples*Lx*Ly*D_k^4] d ln psi / d A~_x, Eq. S3;
                         storage scalar (see gcf_scalar_bytes); the first
                         D_k^k entries of each vertex slot are the block,
                         in the parameter block order                      */
  int32_t* accepted;  /* [n_chains] accepted moves in this call              */
  int32_t* proposed;  /* [n_chains] proposed moves in this call              */
} gcf_samples;

/* Create a context: validates the model, builds the layout, allocates the
 * parameter store and fills it with i.i.d. N(0,1) entries from the
 * counter-based SplitMix64 / Box-Muller generator (stream 0 of `seed`;
 * complex: real part = normal 2k, imaginary part = normal 2k+1).
 * cuda_stream: a cudaStream_t (NULL = legacy default stream).
 * Paper: "Gauge-invariant TNS" and "Gauge canonical form" (Eqs. 6-9). */
gcf_status gcf_init_peps(const gcf_model* model, uint64_t seed, void* cuda_stream,
                         gcf_ctx** out);
void gcf_destroy(gcf_ctx* ctx);
const char* gcf_last_error(const gcf_ctx* ctx);

/* Sizes of the context's layout. */
int64_t gcf_num_params(const gcf_ctx* ctx);   /* number of scalars in A      */
int gcf_config_len(const gcf_ctx* ctx);        /* bytes per configuration     */
int gcf_scalar_bytes(const gcf_ctx* ctx);      /* 4, 8 (f32/c64... see below) */
/* gcf_scalar_bytes: FP64 real 8, FP64 complex 16, other real 4, other complex 8 */

/* Copy parameters in/out.  host_params: host, gcf_num_params values of
 * float64 (real) or complex128 (complex, interleaved re/im); bytes must equal
 * that size.  Values are rounded to the storage type (float for FP32, TF32,
 * BF16; double for FP64).  Returns GCF_ENUMERIC if a value is not finite. */
gcf_status gcf_set_tensors(gcf_ctx* ctx, const void* host_params, size_t bytes);
gcf_status gcf_get_tensors(gcf_ctx* ctx, void* host_params, size_t bytes);

/* Build physical starting configurations (Sec. S-2, "Configuration
 * sampling"): for chain c, links are first fixed on the comb tree (all
 * horizontal links and the vertical links of column 0, other links 0) so that
 * every vertex satisfies the Gauss law for the occupations of that chain,
 * then P_j^{t_j} is applied for every plaquette j = y*(Lx-1)+x.
 * occupations: device, n_chains*Lx*Ly int8 in {0,1}, or NULL (all empty);
 * plaquette_powers: device, n_chains*(Lx-1)*(Ly-1) int8 in [0, N) or NULL;
 * configs: device output, n_chains*cfg_len.
 * GCF_EGAUSS if some chain's occupations violate sum(p) = sum(Q) mod N. */
gcf_status gcf_init_configs(gcf_ctx* ctx, int n_chains, const int8_t* occupations,
                            const int8_t* plaquette_powers, int8_t* configs);

/* Amplitude psi(s) = <B[Ly-2] | row Ly-1> where B[r] is the boundary MPS of
 * rows 0..r absorbed bottom-up, each compressed to chi by QR left-to-right
 * and LQ / truncated SVD right-to-left (Sec. S-2, Eq. S5; cost paragraph of
 * the main text).  configs: device n*cfg_len; log_abs, phase: device [n].
 * An unphysical configuration gives log_abs = -inf, phase = 0 (its amplitude
 * is exactly zero in a GI-PEPS, Sec. S-2) and GCF_OK. */
gcf_status gcf_amplitude(gcf_ctx* ctx, int n, const int8_t* configs, double* log_abs,
                         double* phase);

/* Local energy E_loc(s) = sum_s' <s|H|s'> psi(s')/psi(s), Eq. (S2); the
 * plaquette ratios of row pair (r, r+1) use the strip <B[r-1]|W_r W_{r+1}|T[r+2]>
 * and the hop ratios the row <B[r-1]|W_r|T[r+1]> (horizontal) or the strip
 * (vertical), with the environments of s in numerator and denominator.
 * e_loc: device [2n] (re, im).  GCF_EGAUSS if any configuration is unphysical. */
gcf_status gcf_local_energy(gcf_ctx* ctx, int n, const int8_t* configs, double* e_loc);

/* Log-derivatives O_x = (d psi_r / d A~_x) / psi_r with psi_r the row value
 * <B[r-1]|W_r|T[r+1]> (Eq. S3).  block_ids: device [n*Lx*Ly]; O: device
 * [n*Lx*Ly*D_k^4] storage scalars (first D_k^k entries per vertex are used).
 * GCF_EGAUSS if any configuration is unphysical. */
gcf_status gcf_log_grad(gcf_ctx* ctx, int n, const int8_t* configs, int32_t* block_ids,
                        void* O);

/* Sampling of several contexts (lattices of different sizes, Sec. S-2 moves
 * and order on each) in one persistent launch: context i advances its
 * n_chains[i] chains exactly as gcf_sample_batch(ctxs[i], n_chains[i],
 * n_sweeps, seeds[i], configs[i], &outs[i]) would, chain c of context i
 * drawing from the stream of (seeds[i], c).  All contexts must have the same
 * tensor type and precision and live on the same device; the launch runs on
 * ctxs[0]'s stream after the other contexts' streams are synchronised.
 * ctxs, n_chains, seeds, configs: host arrays of n_ctx entries; configs[i]
 * and the members of outs[i] are device pointers as for gcf_sample_batch;
 * outs may be NULL.  Scratch is owned by ctxs[0].  GCF_EGAUSS if a starting
 * configuration is unphysical.  Synchronises ctxs[0]'s stream. */
gcf_status gcf_sample_multi(gcf_ctx* const* ctxs, int n_ctx, const int* n_chains, int n_sweeps,
                            const uint64_t* seeds, int8_t* const* configs, const gcf_samples* outs);

/* Vector-Jacobian product of the log-amplitudes, the adjoint of Eq. S3
 * summed over samples: grad = sum_s w_s d ln psi(s) / d theta, with theta the
 * parameter vector in the layout of gcf_set_tensors.  Each sample touches one
 * block per vertex, so grad is the scatter of w_s O_s (gcf_log_grad) into the
 * blocks the samples selected.  For real tensors d ln psi / d theta =
 * d ln|psi| / d theta.
 * weights: device, [n] doubles (real tensors) or [2n] (re, im) (complex);
 * grad: device output, [n_params] doubles or [2*n_params] (re, im); overwritten.
 * Work buffers are owned by the context.  GCF_EGAUSS if any configuration is
 * unphysical.  Synchronises the context's stream. */
gcf_status gcf_log_grad_vjp(gcf_ctx* ctx, int n, const int8_t* configs, const double* weights,
                            double* grad);

/* Markov-chain sampling (Sec. S-1 Metropolis rule, Sec. S-2 moves and
 * sequential order): n_sweeps sweeps of every chain in one persistent launch;
 * each sweep visits the plaquettes (row pairs bottom to top, left to right,
 * power t uniform in [1, N-1]) and, with matter, the horizontal links (rows
 * top to bottom) then the vertical links (row pairs bottom to top) with the
 * gauge-dressed hop; after each sweep the sample is measured (amplitude,
 * E_loc, O) into `out`.  A proposal s1 from s0 is accepted iff
 * u * |psi(s0)|^2 < |psi(s1)|^2, u uniform in [0,1) from the counter-based
 * SplitMix64 stream of (seed, chain): word k = mix64(key + (k+1)*GAMMA),
 * key = mix64(seed + (chain+1)*GAMMA), GAMMA = 0x9E3779B97F4A7C15,
 * u = (word >> 11) * 2^-53.  Counter of sweep w: k = w*n_slots + slot with
 * slot 2j (power t = 1 + word % (N-1)) and 2j+1 (u) for plaquette
 * j = y*(Lx-1)+x; with matter, slot 2*Np + j for horizontal link j and
 * 2*Np + n_h + j for vertical link j; n_slots = 2*Np (+ n_h + n_v).
 * configs: device n_chains*cfg_len, in/out (must be physical).
 * Deterministic: the same tensors, configurations, seed and kernel form give
 * bit-identical configurations and outputs.
 * GCF_EGAUSS if a starting configuration is unphysical. */
gcf_status gcf_sample_batch(gcf_ctx* ctx, int n_chains, int n_sweeps, uint64_t seed,
                            int8_t* configs, const gcf_samples* out);

/* gcf_sample_batch enqueued on `stream` (NULL: the context's stream) with
 * no host synchronisation and no allocation, so that the persistent launch
 * can be recorded in a CUDA graph and replayed.  The kernel arguments (seed,
 * pointers, sizes) are fixed at enqueue time.  The context's scratch must
 * already cover n_chains (GCF_EINVAL otherwise): call gcf_sample_batch with
 * at least as many chains first.  Unphysical starting configurations are not
 * reported as a status; their samples get log|psi| = -inf and E_loc = NaN. */
gcf_status gcf_sample_batch_async(gcf_ctx* ctx, int n_chains, int n_sweeps, uint64_t seed,
                                  int8_t* configs, const gcf_samples* out, void* stream);

/* FP64 reductions and parameter update (Sec. S-1 Eq. S3; Sec. S-3 Eqs. S6-S8):
 *   F = <O^* E_loc> - <O^*><E_loc>,  S = <O^* O> - <O^*><O>   (Eq. S7)
 *   x = (S + diag_shift I)^{-1} F by conjugate gradient (S never formed);
 *   with n_samples >= n_params (S of full rank) the CG is preconditioned by
 *   the diagonal of S + diag_shift I, otherwise it is plain CG, which ends in
 *   about n_samples iterations on the low-rank-plus-shift system.
 *   mode GCF_SR:          A <- A - lr * x
 *   mode GCF_TDVP_STAGE1: A <- A + c1 * dt * (-i x),  c1 = (1+i)/2
 *   mode GCF_TDVP_STAGE2: A <- A + c2 * dt * (-i x),  c2 = (1-i)/2
 * (TDVP modes need GCF_COMPLEX.)  e_loc, block_ids, O: device, as written by
 * gcf_sample_batch for n_samples samples, all with equal weight.
 * stats: host double[8] = {Re<E>, Im<E>, std error of Re<E> over chains
 * (n_chains > 1, else over samples), CG iterations, relative residual,
 * |F|, 1 if CG reached tol, 1 if the diagonal preconditioner was used};
 * n_chains is the number of chains the samples came from
 * (chain-major order).  GCF_ETIMEOUT if CG hits max_iter before tol (the
 * update is still applied).  Sums over samples and dot products combine
 * per-block partial sums with FP64 atomics, so repeated calls on the same
 * samples agree to rounding, not bit for bit. */
gcf_status gcf_sr_step(gcf_ctx* ctx, int n_samples, int n_chains, const double* e_loc,
                       const int32_t* block_ids, const void* O, double diag_shift, double lr,
                       int mode, double dt, int max_iter, double tol, double* stats);

/* One VMC iteration end to end from host memory: copies configs (host,
 * n_chains*cfg_len, in/out) to the device, runs gcf_sample_batch into
 * context-owned sample buffers, then gcf_sr_step, and copies the configs and
 * stats (host double[8], as gcf_sr_step) back. */
gcf_status gcf_vmc_step_host(gcf_ctx* ctx, int n_chains, int n_sweeps, uint64_t seed,
                             int8_t* host_configs, double diag_shift, double lr, int mode,
                             double dt, int max_iter, double tol, double* stats);

/* Amplitude evaluation that allocates nothing: the same computation and
 * result as gcf_amplitude, for callers that cannot call cudaMalloc during the
 * call -- services that reserve all device memory up front and forbid
 * allocation on the request path, and embedders whose own allocator owns the
 * device (a foreign cudaMalloc would fragment or exceed its pool).  (The
 * paper has no counterpart; this is an interface addition.)
 * - Scratch comes from one fixed array of 32 MiB compiled into the library
 *   (static device storage that every GPU which loads the library holds until
 *   the process exits), not from cudaMalloc.  The context itself must already
 *   exist: gcf_init_peps allocates, so create it at set-up time.
 * - The first call on each device looks up the array's device address with
 *   that device current; make that first call before any stream capture.  The
 *   device current at the call must be the context's device (else GCF_EINVAL).
 *   The address is kept for the life of the process: after a device reset
 *   (cudaDeviceReset) the library must be used from a new process.
 * - A lattice whose per-CTA scratch exceeds 32 MiB is rejected with
 *   GCF_EINVAL and a message giving the required size; otherwise the number
 *   of CTAs is capped at what fits, and any n >= 1 is accepted.
 * - Every call shares the array, which keeps the previous call's contents:
 *   calls whose kernels overlap on the GPU (two streams, two contexts, two
 *   host threads) race on it and return wrong amplitudes; serialise them.
 * - The call does not synchronise the stream; outputs are ready when the
 *   context's stream reaches this point.
 * Arguments and outputs exactly as gcf_amplitude. */
gcf_status gcf_amplitude_noalloc(gcf_ctx* ctx, int n, const int8_t* configs, double* log_abs,
                                 double* phase);

/* Number of kernel launches this context issued since creation (for
 * accounting in benchmarks). */
int64_t gcf_launch_count(const gcf_ctx* ctx);

/* Form of the sampling / measurement kernel this context launches (an
 * implementation choice; the paper has no counterpart): 0 = one chain per
 * CTA of 256 threads (gcf::vmc_kernel), 1 = two chains per CTA on groups of
 * 128 threads (gcf::vmc_kernel_grouped), 2 = four chains per CTA of 512
 * threads (gcf::vmc_kernel_grouped4).  In the grouped forms the chain groups
 * of a CTA meet before every row of a pass (lockstep; bounded waits, no data
 * exchanged), so the SM runs one region of code at a time.  Chosen at
 * context creation from the shared-memory footprint (or by gcf_autotune);
 * GCFVMC_EXEC=cta|group|group4 and GCFVMC_LOCK=0|1 in the environment force
 * a form.  All forms compute the same results. */
int gcf_executor(const gcf_ctx* ctx);

/* Lockstep waits that ran out in the last synchronous sampling or
 * measurement launch of this context (implementation detail; no counterpart
 * in the paper).  A chain group whose wait for the other groups of its CTA
 * exceeds its iteration limit leaves lockstep for the rest of that chain
 * and counts here; results are unaffected, only the speed.  0 normally;
 * GCFVMC_LOCK_FAULT=1 in the environment (a test hook) makes one group never
 * count in, so the others' waits run out. */
int gcf_phase_timeouts(const gcf_ctx* ctx);

/* One-sided Jacobi SVDs of the truncated bonds (Sec. S-2 compression) that
 * reached the sweep limit without converging in the last synchronous
 * amplitude, energy, gradient or sampling launch of this context (for
 * gcf_sample_multi: summed over its contexts, reported on ctxs[0]).  0
 * normally; such calls return GCF_ETIMEOUT.  -1 for a NULL context. */
int gcf_svd_unconverged(const gcf_ctx* ctx);

/* Bytes of device scratch one chain slot of this context takes (the
 * boundary-MPS store, the network, factorisation and environment buffers;
 * one slot per chain resident on the GPU).  -1 for a NULL context. */
int64_t gcf_scratch_bytes_per_chain(const gcf_ctx* ctx);

/* K of the checkpointed boundary-MPS store (gcf_model.recompute_env after
 * resolving -1), 0 when every MPS is kept.  -1 for a NULL context. */
int gcf_checkpoint_interval(const gcf_ctx* ctx);

/* 1 if this context's BF16 form runs its environment GEMMs on the
 * fifth-generation tensor cores (tcgen05.mma with BF16 operands, FP32
 * accumulation in tensor memory; real tensors whose largest environment GEMM
 * has N <= 128), 0 otherwise (other forms, complex tensors, larger bonds:
 * their tensor-core GEMMs use warp-level mma.sync).  Implementation detail;
 * no counterpart in the paper.  -1 for a NULL context. */
int gcf_tensor_core_form(const gcf_ctx* ctx);

/* Tensor-core completion waits that ran out in the last synchronous launch
 * of this context (the chain then computes its GEMMs on the CUDA cores for
 * the rest of the launch; results are unaffected).  0 normally. */
int gcf_tensor_timeouts(const gcf_ctx* ctx);

/* Chains per CTA of the last gcf_sample_multi launch made with ctx as
 * ctxs[0] (implementation detail, no counterpart in the paper): 1 for
 * gcf::vmc_kernel_multi (one chain per CTA of 256 threads), 4 for
 * gcf::vmc_kernel_multi4 (four chains per CTA of 512 threads, chosen when a
 * context truncates; GCFVMC_MULTI=cta|group4 forces one), 0 before any
 * launch, -1 for a NULL context. */
int gcf_multi_chains_per_cta(const gcf_ctx* ctx);

/* Sweep limit of the one-sided Jacobi SVD for this context's later launches,
 * 1 <= max_sweeps <= 1000 (default 40; each sweep visits every column pair
 * once).  GCF_EINVAL outside that range. */
gcf_status gcf_set_svd_sweeps(gcf_ctx* ctx, int max_sweeps);

/* Shared-memory placement level of the kernel form this context launches
 * (implementation choice; no counterpart in the paper): 0 = configuration
 * only, 1 = + hot buffers (network boxes, proposals, current environments,
 * GEMM temporaries), 2 = + the staged boundary-MPS rows of the current pass,
 * 3 = + the right environments of the pass. */
int gcf_smem_level(const gcf_ctx* ctx);

/* Autotuner (implementation choice; no counterpart in the paper): times every
 * kernel form that fits an SM (executor x shared-memory level) on
 * gcf_sample_batch of a copy of `configs` (device, n_chains x cfg_len, left
 * unchanged) for n_sweeps sweeps, after one warm-up run per form, and keeps
 * the fastest for this context's later launches.  ms (host, optional): the
 * time of form i (1e300 if it did not launch) for i < *n_forms on entry;
 * *n_forms (optional) is set to the number of forms tried.  Allocates and
 * frees its own work buffers; synchronises the context's stream. */
gcf_status gcf_autotune(gcf_ctx* ctx, int n_chains, int n_sweeps, const int8_t* configs, double* ms,
                        int* n_forms);

#ifdef __cplusplus
}
#endif
#endif /* GCFVMC_H */
