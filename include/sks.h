/*
 * sks.h -- C ABI of the GB300 (sm_103a) adaptive sketching-based solvers for
 *
 *     x* = argmin_x  1/2 <x, H x> - b^T x,   H = A^T A + nu^2 Lambda      (eq. 1)
 *
 * of Lacotte & Pilanci, "Fast Convex Quadratic Optimization Solvers with
 * Adaptive Sketching-based Preconditioners" (arXiv 2104.14101).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named "device" point to GPU global memory of the current device;
 *   they are borrowed, never freed, and must stay valid until the work queued
 *   on `stream` has finished.  Host pointers are read before the call returns.
 * - A is n x d, row-major, leading dimension lda >= d (elements), stored as
 *   float64 (SKS_F64, d <= 14336) or float32 (SKS_F32, d <= 16384); rows with
 *   d > 4096 take one right-hand side per pass.  The base address must be 16-byte
 *   aligned and lda * sizeof(element) a multiple of 16 bytes (A is streamed by
 *   the Tensor Memory Accelerator); otherwise SKS_ERR_INVALID_ARG.
 * - Vectors of length d with k right-hand sides are d x k column-major
 *   float64 arrays (column c starts at element c*d).
 * - `stream` is a cudaStream_t passed as void*; NULL means the legacy stream.
 *   All GPU work is queued on it in order.
 * - Scratch memory is caller-allocated device memory (`ws`, `ws_bytes`), sized
 *   by the matching *_workspace_size query; the library allocates no device
 *   memory.  Handles (sks_sketch, sks_precond) are small host objects that
 *   refer to their own caller-allocated device storage.
 * - Every entry point returns an sks_status and never aborts; on failure
 *   sks_last_error() describes the cause (thread-local string).
 */
#ifndef SKS_H_
#define SKS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SKS_OK = 0,
  SKS_ERR_INVALID_ARG = 1,    /* bad size, pointer, alignment, nu <= 0, lambda_i < 1 */
  SKS_ERR_NOT_PD = 2,         /* non-positive pivot in a Cholesky factorisation      */
  SKS_ERR_NO_CONVERGENCE = 3, /* max_iter reached; x holds the last accepted iterate */
  SKS_ERR_NUMERIC = 4,        /* NaN / Inf met in the iteration                      */
  SKS_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out                  */
  SKS_ERR_CUDA = 6,           /* a CUDA runtime call failed                          */
  SKS_ERR_WORKSPACE = 7,      /* ws_bytes smaller than the size query returned       */
  SKS_ERR_UNSUPPORTED = 8     /* valid request that the library does not implement   */
} sks_status;

/* Random embeddings of Section 2.1. */
typedef enum {
  SKS_SRHT = 0,     /* S = R H E: Walsh-Hadamard of the sign-flipped, zero-padded A, rows subsampled */
  SKS_GAUSSIAN = 1, /* i.i.d. N(0, 1/m) entries, generated from Philox, never stored               */
  SKS_SJLT = 2,     /* s nonzeros +-1/sqrt(s) per column at distinct hashed rows                    */
  SKS_RADEMACHER = 3, /* sub-Gaussian: i.i.d. +-1/sqrt(m) entries from Philox bits, never stored       */
  /* The Gaussian embedding with 8-bit tensor-core arithmetic (float32 A only):
   * the entries of G rounded to e4m3 and A quantised to e4m3 against one
   * power-of-two scale per column and per slice of 16384 rows (per-tile
   * scales), each slice's product scaled back in float32.  The adaptive
   * solvers use it only when the rounding noise of A, 2^-8/3 ||A||_F^2 / d,
   * is at most 0.1 nu^2 min lambda (else the bfloat16 split serves the same G;
   * sks_stats.sketch_e4m3 says which); sks_sketch_create uses it as asked.   */
  SKS_GAUSSIAN_E4M3 = 4
} sks_kind;

typedef enum { SKS_F64 = 0, SKS_F32 = 1 } sks_dtype;

/* Arithmetic of a solve. */
typedef enum {
  SKS_PLAIN_F64 = 0,    /* everything in float64 (A must be SKS_F64)                           */
  SKS_MIXED_REFINED = 1 /* float32 A, BF16/float32 sketch and inner PCG, float64 refinement      */
} sks_precision;

/* Problem (1).  A, b, lambda_diag: device pointers. */
typedef struct {
  sks_dtype dtype;
  int64_t n, d, lda, k;        /* k = number of right-hand sides (columns of b)    */
  const void* A;               /* n x d row-major, leading dimension lda           */
  const double* b;             /* d x k column-major float64                       */
  double nu;                   /* nu > 0                                           */
  const double* lambda_diag;   /* d entries, each >= 1 (Lambda >= I_d, eq. 1)      */
} sks_problem;

/* One improvement test of Algorithm 1 / 2 (optional host-side trace). */
typedef struct {
  int64_t t;         /* time index of the step                        */
  int64_t m;         /* sketch size used by the step                  */
  double ratio;      /* delta~+ / delta~_I                            */
  double threshold;  /* c(rho) phi(rho)^(t+1-I)                       */
  int32_t accepted;  /* 1: x+ accepted; 0: rejected, m doubled        */
  int32_t outer;     /* refinement step (mixed form), 0 otherwise     */
  int32_t column;    /* right-hand side the test belongs to           */
  int32_t reserved;
  double delta;      /* with opts.x_star: 1/2 ||x - x*||_H^2 at the iterate kept after the event
                        (x+ if accepted, x_t otherwise); 0 without x_star                      */
  double delta0;     /* the same at the column's x_0                               */
} sks_trace_event;

/* Options of Algorithms 1 and 2 (defaults by sks_opts_default). */
typedef struct {
  double rho;          /* rate parameter rho in (0, 1); default 1/8 (Section 4.1)            */
  int64_t m_init;      /* initial sketch size m_init >= 1                                    */
  int64_t m_max;       /* cap on m; 0 = n_pad (SRHT) or n (Gaussian, SJLT)                   */
  sks_kind kind;       /* embedding                                                          */
  int sjlt_s;          /* nonzeros per column of the SJLT (>= 1)                             */
  double tol;          /* target ||x - x*||_H / ||x*||_H                                     */
  int64_t max_iter;    /* bound T on accepted iterations                                     */
  sks_precision precision;
  int reuse_residual;  /* 1: keep the recursive r_t at a restart (Algorithm 2 recomputes it) */
  uint64_t seed;       /* Philox key of every random draw                                    */
  int64_t max_outer;   /* refinement steps of SKS_MIXED_REFINED                              */
  double inner_tol;    /* relative accuracy asked of each inner solve (mixed form)           */
  sks_trace_event* trace; /* optional host array receiving every test; NULL = none            */
  int64_t trace_cap;   /* capacity of `trace`                                                */
  int stop_rule;       /* SKS_STOP_ESTIMATE or SKS_STOP_CERTIFIED (below)                    */
  double cert_delta;   /* failure probability delta of SKS_STOP_CERTIFIED, in (0, 1)         */
  double cert_de;      /* effective dimension put into m_delta; 0 = d (the conservative d_e) */
  const double* x_star; /* optional device d x k solution, for traces only: each trace event
                           then carries delta_t = 1/2 ||x_t - x*||_H^2 (Section 1.1), formed
                           exactly as 1/2 (x* - x_t)^T r_t from the iteration's residual
                           (one extra dot per step; plain float64 form; NULL = off)          */
} sks_opts;

/* Stop rules (the paper prescribes none; Section 1.3 and Remark 4.2).  With
 * eps = 1/2 tol^2 ||x*||_H^2 and ||x*||_H^2 = b^T x* estimated by b^T x_t:
 * SKS_STOP_ESTIMATE:  stop when delta~_t <= eps / 4 (the decrement estimates
 *                     delta_t, Lemma 2.1, with a factor 2 of safety in norm);
 * SKS_STOP_CERTIFIED: Remark 4.2, stop when delta~_t <= eps / (m_delta + 1),
 *                     which gives delta_t <= eps with probability >= 1 - delta
 *                     whatever the sketch size; m_delta of Theorem 5.1 (SRHT),
 *                     Theorem 5.2 with omega^2 <= d_e (Gaussian, and the
 *                     sub-Gaussian Rademacher embedding), d_e^2 / delta
 *                     (SJLT: the order of Table 1 with constant 1).  Not
 *                     available for the unpreconditioned CG or the batch. */
enum { SKS_STOP_ESTIMATE = 0, SKS_STOP_CERTIFIED = 1 };

/* Per-solve statistics (host struct, filled before the solve returns). */
typedef struct {
  int64_t iters;          /* accepted iterations t                              */
  int64_t rejections;     /* failed improvement tests (= sketch doublings)      */
  int64_t final_m;        /* sketch size at exit                                */
  int64_t a_passes;       /* full reads of A by the iteration (H p, residuals)  */
  int64_t sketch_passes;  /* sketch formations / extensions                     */
  int64_t factorizations; /* preconditioner builds                              */
  int64_t outer_iters;    /* refinement steps (mixed form)                      */
  double final_delta_tilde;
  double est_rel_err;     /* sqrt(delta~_t / b^T x_t): the stop rule's estimate */
  int64_t trace_len;      /* events written to opts.trace                       */
  float ms_total, ms_sketch, ms_factor, ms_iter;
  float ms_apass;         /* device time of the A-pass kernels (CUDA events)    */
  int64_t apass_timed;    /* A-pass launches covered by ms_apass                */
  sks_status status;
  int32_t sketch_e4m3;    /* SKS_GAUSSIAN_E4M3: 1 if the 8-bit sketch served the solve */
} sks_stats;

typedef struct sks_sketch sks_sketch;
typedef struct sks_precond sks_precond;

/* Fill `o` with the defaults: rho = 1/8, m_init = 1, m_max = 0, SRHT, s = 1,
 * tol = 1e-10, max_iter = 1000, plain float64, reuse_residual = 1, seed = 0,
 * max_outer = 20, inner_tol = 1e-4, no trace, SKS_STOP_ESTIMATE,
 * cert_delta = 0.01, cert_de = 0, x_star = NULL. */
void sks_opts_default(sks_opts* o);

/* Version string of the library build. */
const char* sks_version(void);

/* Last error message of the calling thread ("" if none). */
const char* sks_last_error(void);

/* Number of CUDA kernels the calling thread has launched through this
 * library since it was loaded (monotone counter, for launch accounting). */
uint64_t sks_kernel_launch_count(void);

/* ---------------------------------------------------------------------------
 * Hessian pass (Section 4.1.2: the O(nd) per-iteration cost).
 * y = A^T (A x) + nu^2 Lambda x for the k columns of x, in ONE read of A.
 * x, y: device d x k column-major float64 (y may not alias x).  Arithmetic in
 * the precision of A (float32 A: float32 products and row sums, float64
 * cross-block accumulation), or with `extended` = 1 on a float32 A:
 * double-float arithmetic (float32 pairs, unit roundoff ~2^-44; float64 x
 * split into two floats), the refinement residual of the mixed form.
 * ws: device scratch of sks_hess_apply_workspace_size(problem) bytes.
 * ------------------------------------------------------------------------- */
sks_status sks_hess_apply_workspace_size(const sks_problem* p, size_t* bytes);
sks_status sks_hess_apply(const sks_problem* p, const double* x, double* y, int extended,
                          void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Allocation-free Hessian pass.  The paper has no counterpart: this is a
 * deployment variant of sks_hess_apply for callers that must not allocate
 * device memory at the moment they need H x -- for example code inside a host
 * framework that owns every device allocation through its own fixed-budget
 * allocator, or a latency-critical loop that cannot pay for cudaMalloc's
 * device-wide synchronisation -- and therefore cannot hand over the
 * workspace sks_hess_apply asks for.
 * Same operation, arguments and results as sks_hess_apply, minus `ws`: the
 * per-block partial sums live in a library-owned static device array of
 * 8 MiB, which every GPU that loads the library holds until the process
 * exits.  The pass needs grid * g * k * d partial sums of the vector type
 * (float32 for a float32 A without `extended`, else float64), plus two
 * float32 d x k vectors in the float32 case, where grid = SMs x blocks per SM
 * (1 for float64 A, `extended` or d > 4096, else 2) and g = 8, 2 or 1 row
 * groups per block for rows of at most 32 q, 128 q or more column vectors
 * (q = 8 vectors of 2 float64 columns, or 4 vectors of 4 float32 columns;
 * g = 1 when k = 8).  On a 152-SM GPU every d <= 4096
 * with k = 1 fits.  A larger problem is rejected with SKS_ERR_INVALID_ARG
 * and a message giving the size it needs.
 * The first call on a device looks up the array's device address with that
 * device current and caches it; make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * the status word is cleared on every call, but calls whose GPU work overlaps
 * (other streams, other host threads on the same device) race on it and must
 * be serialised by the caller.  The call synchronises `stream` to read its
 * status and calls no cudaMalloc or cudaFree.
 * ------------------------------------------------------------------------- */
sks_status sks_hess_apply_noalloc(const sks_problem* p, const double* x, double* y, int extended, void* stream);

/* ---------------------------------------------------------------------------
 * Sketch S A of Section 2.1 with nested growth.
 * sks_sketch_create forms S_m A for m = m_init (SRHT: also the n_pad x d
 * matrix H E A_pad, once); sks_sketch_grow(new_m) extends it to new_m >= m
 * rows (SRHT: gathers more rows of H E A_pad; Gaussian and Rademacher: append
 * rows of G A; SJLT: re-hashes and re-forms S A in one pass over A).  The sketch is kept in the
 * precision of A and "unscaled": S A = scale * Y with scale = 1/sqrt(m) (SRHT,
 * Gaussian) or 1 (SJLT); sks_sketch_copy_out writes the scaled S A (m x d
 * row-major float64).
 * Random draws: Philox4x32-10 keyed by `seed`, bit-identical to the oracle.
 * ws: device scratch of sks_sketch_workspace_size bytes, owned by the handle
 * until sks_sketch_destroy.
 * ------------------------------------------------------------------------- */
sks_status sks_sketch_workspace_size(const sks_problem* p, sks_kind kind, int64_t m_max, int sjlt_s,
                                     size_t* bytes);
sks_status sks_sketch_create(sks_sketch** out, const sks_problem* p, sks_kind kind, int64_t m_init,
                             int64_t m_max, int sjlt_s, uint64_t seed, void* ws, size_t ws_bytes,
                             void* stream);
sks_status sks_sketch_grow(sks_sketch* s, int64_t new_m, void* stream);
sks_status sks_sketch_rows(const sks_sketch* s, int64_t* m);
sks_status sks_sketch_copy_out(const sks_sketch* s, double* SA, void* stream);
void sks_sketch_destroy(sks_sketch* s);

/* ---------------------------------------------------------------------------
 * Sketched preconditioner H_S = (SA)^T SA + nu^2 Lambda (Section 4.1.1).
 * m >= d: float64 Cholesky of the d x d matrix H_S; m < d: float64 Cholesky of
 * W_S = SA Lambda^{-1} (SA)^T + nu^2 I_m and the Woodbury identity
 *   v = (Lambda^{-1}/nu^2) (I - (SA)^T W_S^{-1} SA Lambda^{-1}) z.
 * The triangular factor is inverted explicitly so that an apply is two
 * matrix-vector products.  Returns SKS_ERR_NOT_PD on a non-positive pivot.
 * sks_precond_apply: v = H_S^{-1} z for k columns (device float64 d x k).
 * ------------------------------------------------------------------------- */
sks_status sks_precond_workspace_size(const sks_problem* p, int64_t m_max, size_t* bytes);
sks_status sks_precond_build(sks_precond** out, const sks_sketch* s, const sks_problem* p,
                             void* ws, size_t ws_bytes, void* stream);
/* sks_precond_build_ex: sks_precond_build with the factorisation of the given
 * form.  SKS_PLAIN_F64: as sks_precond_build.  SKS_MIXED_REFINED (float32 A
 * only, else SKS_ERR_INVALID_ARG): the factorisation the mixed solvers use --
 * the Gram matrix on the tensor cores, the Cholesky factorisation in
 * double-float arithmetic (pairs of float32, ~2^-47 per operation, on the
 * float32 pipe), and the inverse factor merged in float32 (m >= d: the apply
 * X^T X stays positive definite) or in double-float (m < d, Woodbury). */
sks_status sks_precond_build_ex(sks_precond** out, const sks_sketch* s, const sks_problem* p,
                                sks_precision precision, void* ws, size_t ws_bytes, void* stream);
sks_status sks_precond_apply(const sks_precond* P, const double* z, double* v, int64_t k, void* stream);
void sks_precond_destroy(sks_precond* P);

/* ---------------------------------------------------------------------------
 * Adaptive solvers.
 * sks_adaptive_pcg_solve: Algorithm 2 (adaptive PCG).
 * sks_adaptive_ihs_solve: Algorithm 1 with the IHS step x - (1-rho) H_S^{-1} grad f(x)
 *                         (Theorem 3.2).
 * Both start from m = m_init, test delta~+/delta~_I > c(rho) phi(rho)^(t+1-I)
 * after every step, and on failure double m (capped at m_max, where the step is
 * accepted instead), extend the sketch, refactor H_S and restart at x_t.
 * Stop rule (the paper prescribes none; Remark 4.2): after an accepted step,
 * opts.stop_rule decides; by default (SKS_STOP_ESTIMATE) stop when the
 * estimate delta~_t / (b^T x_t) of ||x_t - x*||_H^2/||x*||_H^2 is <= (tol/2)^2
 * (IHS: 2 delta~_t); SKS_STOP_CERTIFIED uses tol^2 / (m_delta + 1) instead.
 * Between re-sketches the iteration runs on the device in one launch (fused
 * A-pass, preconditioner apply, step and test; see the loop below), and up
 * to 8 right-hand sides (d <= 1024) run in lockstep sharing every pass over
 * A: each column has its own test and stop, a failed test of any column
 * doubles m and every live column restarts at its current iterate with the
 * new preconditioner; more columns run in batches of 8, wider rows one by one.
 * x: device float64 d x k, in: x_0, out: the solution.  stats: host, may be NULL.
 * ws: device scratch of sks_solve_workspace_size bytes.
 * Returns SKS_ERR_NO_CONVERGENCE if max_iter accepted steps did not reach tol.
 * ------------------------------------------------------------------------- */
sks_status sks_solve_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes);
sks_status sks_adaptive_pcg_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                  void* ws, size_t ws_bytes, void* stream);
sks_status sks_adaptive_ihs_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                  void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Dual formulation (eq. 2), for n < d (more columns than rows): the dual
 *   w* = argmin 1/2 <w, (A~ A~^T + nu^2 I_n) w> - (A Lambda^{-1} b)^T w,
 *   A~ = A Lambda^{-1/2},
 * is itself an instance of eq. 1 with the d x n data matrix Lambda^{-1/2} A^T,
 * Lambda = I_n and right-hand side A Lambda^{-1} b; it is solved by adaptive
 * PCG (Algorithm 2) or adaptive IHS (Algorithm 1) exactly as the primal, and
 * x = Lambda^{-1} (b - A^T w) / nu^2 is returned (the optimality condition of
 * eq. 1 written with w = (A Lambda^{-1} A^T + nu^2 I)^{-1} A Lambda^{-1} b).
 * Same problem description, options, x (d x k; its input is ignored: the dual
 * starts at w = 0), stats (of the dual solve) and errors as
 * sks_adaptive_pcg_solve; o->tol is the dual's relative H-error target, and
 * the primal error obeys ||x - x*||_H <= ||H_dual (w - w*)||_2 / nu^2.  The
 * workspace (sks_dual_workspace_size) holds the dual matrix, a transposed copy
 * of A of the same size, in A's precision: for a float32 A (mixed form) with
 * Lambda != I its entries a_ij / sqrt(lambda_j) are rounded to float32, so the
 * dual solved is that rounded one (exact for Lambda = I).  Any n, d within the
 * A-pass limits (the dual's d is n).
 * ------------------------------------------------------------------------- */
sks_status sks_dual_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes);
sks_status sks_dual_pcg_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                              void* ws, size_t ws_bytes, void* stream);
sks_status sks_dual_ihs_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                              void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Non-adaptive solvers: the baselines of Section 6 and the Polyak-IHS of
 * Appendix A.  The sketch size stays at m = min(m_init, m_max) (Section 6
 * compares with PCG at m = 2d); no improvement test rejects a step.
 *   SKS_FIXED_PCG:    PCG (eq. 5) with the preconditioner H_S.
 *   SKS_FIXED_IHS:    IHS (eq. 4) with mu = 1 - rho (Theorem 3.2).
 *   SKS_POLYAK_IHS:   heavy-ball IHS x+ = x - mu H_S^{-1} grad f(x) + beta (x - x_prev)
 *                     with mu = 2(1-rho)/(1+sqrt(1-rho)), beta = (1-sqrt(1-rho))/(1+sqrt(1-rho))
 *                     (Corollary A.2); x_prev = x_0 at the start.
 *   SKS_CG:           conjugate gradient without preconditioner (H_S = I); no
 *                     sketch is formed.  Plain float64 form only
 *                     (SKS_ERR_UNSUPPORTED otherwise).
 * Stop rules: PCG, IHS and Polyak-IHS as the adaptive solvers (the decrement
 * estimate delta~_t / b^T x_t, 2 delta~_t for the IHS family, <= (tol/2)^2);
 * CG stops when ||r_t||_2 <= tol ||b||_2 (without a preconditioner there is no
 * estimate of the H-norm error), and stats.est_rel_err is ||r_t|| / ||b||.
 * Arguments, workspace (sks_solve_workspace_size), precisions (the mixed form
 * refines around the fixed-sketch inner solver) and errors as for
 * sks_adaptive_pcg_solve; stats.rejections is always 0.  Returns
 * SKS_ERR_NO_CONVERGENCE with x = x_T after max_iter steps, so a run with a
 * tiny tol and max_iter = T yields the T-th iterate.
 * ------------------------------------------------------------------------- */
typedef enum { SKS_FIXED_PCG = 0, SKS_FIXED_IHS = 1, SKS_POLYAK_IHS = 2, SKS_CG = 3 } sks_fixed_method;
sks_status sks_fixed_solve(sks_fixed_method method, const sks_problem* p, const sks_opts* o, double* x,
                           sks_stats* stats, void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Adjoint of the solve (gradients of x*(A, b, nu, Lambda), implicit
 * differentiation of H x = b, eq. 1).  For an upstream gradient g = dL/dx
 * (d x k, device float64) the adjoint solve gives u = H^{-1} g and
 *   db = u,   dA = -A (u x^T + x u^T)   (summed over the k columns),
 *   dnu = -2 nu sum_k u_k^T Lambda x_k,   dlambda_i = -nu^2 sum_k u_ik x_ik.
 * Must be called with the workspace of a preceding sks_adaptive_pcg_solve (or
 * _ihs_) of the same problem and options: the adjoint solve reuses the sketch
 * and factored preconditioner left there (adaptive PCG continues from its
 * final m), and SKS_ERR_INVALID_ARG is returned if the workspace holds none.
 * x: the forward solution (d x k).  db (required, d x k float64), dA (optional,
 * n x d in the precision of A, leading dimension ldda), dnu (optional, host
 * double), dlambda (optional, device d float64).  k <= 8 when dA is asked for.
 * ------------------------------------------------------------------------- */
sks_status sks_adjoint(const sks_problem* p, const sks_opts* o, const double* x, const double* g, double* db,
                       void* dA, int64_t ldda, double* dnu, double* dlambda, sks_stats* stats,
                       void* ws, size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------
 * Batched solve: `count` independent problems of eq. 1, each by the adaptive
 * PCG of Algorithm 2 with the same options (SRHT embedding, one right-hand
 * side per problem, d <= 1024, n >= 1, the estimate stop rule), in the plain
 * form (o->precision SKS_PLAIN_F64, every A float64) or the mixed form
 * (SKS_MIXED_REFINED, every A float32: float32 inner passes over A, refinement
 * residuals b - H x and the preconditioner's Gram, factor and apply in
 * double-float, max_outer refinement steps of relative accuracy inner_tol).
 * Every decision of Algorithm 2 is taken on the device, per problem, so one
 * round of batched kernels advances every unfinished problem by one step or
 * one re-sketch; the rounds run inside one CUDA graph launch (a while loop on
 * the device, see the batch plans below) until all problems have stopped.  In
 * the plain form each problem's iterates, m sequence and stop are those of
 * sks_adaptive_pcg_solve with the same options (up to the rounding order of
 * the sums); the same seed serves every problem.
 * probs:  host array of `count` problem descriptions (device A, b, lambda).
 * x:      host array of `count` device pointers, d_i float64 each; in: x_0,
 *         out: the solution (the last accepted iterate for a problem that
 *         stopped with an error).
 * stats:  host array of `count`, may be NULL; stats[i].status is the problem's
 *         own status.
 * info:   host, may be NULL; batch timings and the chosen A-pass unit height.
 * rows_per_unit: rows of A per A-pass work unit; 0 = chosen by timing the
 *         candidates 32..512 on this batch (autotuning), else in [32, 65536].
 * ws:     device scratch of sks_batch_workspace_size bytes (holds H E A_pad of
 *         every problem, the factors and the per-problem state).
 * The call synchronises `stream` twice (the input check and the results).
 * Returns SKS_OK when every problem met tol, else the status of the first
 * failing problem (the others are still solved and reported in stats).
 * ------------------------------------------------------------------------- */
typedef struct {
  int64_t rounds;            /* graph replays until every problem stopped            */
  int64_t kernels_per_round; /* kernel nodes in the captured round                   */
  int64_t rows_per_unit;     /* A-pass unit height used                              */
  float ms_setup;            /* input checks, H E A_pad of every problem, states     */
  float ms_autotune;         /* timing of the candidate unit heights                 */
  float ms_solve;            /* graph replays                                        */
  float ms_apass;            /* summed duration of the rounds' A-pass kernels (device
                                clock: first CTA start to last CTA end per round)   */
  double apass_flops;        /* 4 n d per A-pass of every problem, summed            */
  float ms_gram;             /* the same for the sketched-Hessian (Gram) kernels     */
  double gram_flops;         /* 2 x 64 x 64 per sketch row of every Gram tile        */
  float ms_factor;           /* the same window for the factorisation kernels        */
  float ms_apply;            /* ... for the preconditioner apply                     */
  float ms_rounds;           /* ... for whole rounds (first kernel to the last); the
                                rest of ms_solve is the setup (H E A of every problem) */
} sks_batch_info;

sks_status sks_batch_workspace_size(const sks_problem* probs, int count, const sks_opts* o, size_t* bytes);
/* One-shot solve: sks_batch_create + sks_batch_solve + sks_batch_destroy. */
sks_status sks_solve_batched(const sks_problem* probs, int count, const sks_opts* o, double* const* x,
                             sks_stats* stats, sks_batch_info* info, int rows_per_unit, void* ws, size_t ws_bytes,
                             void* stream);

/* ---------------------------------------------------------------------------
 * Batch plans: the same solve as sks_solve_batched, with the planning done
 * once.  sks_batch_create checks the problems (Lambda >= I on the device;
 * one stream synchronisation), chooses the A-pass unit height (rows_per_unit
 * 0: by timing the candidates 32..512 on this batch) and builds and
 * instantiates ONE CUDA graph:
 *     reset counters -> every problem in INIT -> H E A_pad of every problem
 *     -> WHILE (some problem unfinished and rounds < bound) { one round }
 * where the round's last kernel sets the loop condition on the device.
 * sks_batch_solve uploads the x pointers and launches that graph once: the
 * rounds repeat on the device with no host round trip, and the call
 * synchronises `stream` once at the end to read the per-problem results
 * (the H E A_pad transform is part of every solve).  The problems' device
 * pointers (A, b, lambda) and the workspace are borrowed by the plan and must
 * stay valid and unchanged (A, lambda) until sks_batch_destroy; b may change
 * between solves.  info->ms_setup is the planning time of the create call,
 * info->ms_solve the graph's device time.  Plans are not thread-safe: one
 * solve at a time per plan.  With the environment variable
 * SKS_BATCH_STEPWISE=1 sks_batch_solve launches the same setup and rounds one
 * by one from the host instead (one synchronisation per round), for
 * profilers that do not see the kernels inside a conditional graph node; the
 * results are the same.
 * ------------------------------------------------------------------------- */
typedef struct sks_batch sks_batch;
sks_status sks_batch_create(sks_batch** out, const sks_problem* probs, int count, const sks_opts* o,
                            int rows_per_unit, void* ws, size_t ws_bytes, void* stream);
sks_status sks_batch_solve(sks_batch* plan, double* const* x, sks_stats* stats, sks_batch_info* info, void* stream);
void sks_batch_destroy(sks_batch* plan);

/* ---------------------------------------------------------------------------
 * Self-test of the failure path (the paper has no counterpart).  Every
 * device-side wait of the library (mbarrier phases of the tensor-copy and
 * tensor-core pipelines) is bounded; a wait that runs out records
 * SKS_ERR_TIMEOUT in a device status word, the kernel leaves, and the call
 * returns the status -- no trap, and the context stays usable.  This entry
 * point launches one kernel whose wait can never complete (nothing arrives on
 * its mbarrier) with a limit of limit_ns nanoseconds (1e3 .. 1e9), so the
 * expected return is SKS_ERR_TIMEOUT with sks_last_error() naming site 99;
 * SKS_ERR_INVALID_ARG for a limit out of range.  Synchronises `stream`.
 * ------------------------------------------------------------------------- */
sks_status sks_selftest_wait_timeout(int64_t limit_ns, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* SKS_H_ */
