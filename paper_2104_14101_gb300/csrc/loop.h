// loop.h -- the device-resident iteration of Algorithms 1 and 2 (loop.cu).
#pragma once

#include "internal.h"

namespace sks {

constexpr int kLoopMaxK = 8;  // right-hand sides iterated in lockstep by one launch
constexpr int kLoopDots = 5;  // per-CTA dot partials per column: pHp, delta~+, b^T x, restart, delta

// State of one right-hand side (column), kept on the device between launches.
struct LoopCol {
  double dt, dI, dp, ratio, thr, btx;
  double dt0;       // decrement at the first restart of this solve
  double stop_abs;  // stop when dt <= stop_abs (inner solves of the mixed form: rel2 * dt0)
  double btx_outer; // b^T x_o of the refinement's outer iterate (mixed form)
  double delta, delta0;  // trace mode: 1/2 ||x - x*||_H^2 at the current iterate and at x_0
  long long t, I;
  int active;       // 0: finished before this solve (e.g. its refinement converged)
  int stop, numeric, accept, rejected, outer_done, pad0, pad1;
};

// Header of the control block: per-launch results and the grid barrier.
struct LoopHead {
  unsigned bar_count, bar_gen;
  int any_reject;   // some column failed its test with m < m_max: re-sketch
  int abort;        // a device wait ran out (status word has the site)
  long long iters;  // accepted steps in this launch (max over columns)
  long long apass_ns;  // A-pass phases, device clock (slowest CTA's sum)
  long long apasses;   // passes over A made by the launch
  int trace_len;
  int pad;
};

struct LoopTraceEv {
  long long t, m;
  double ratio, thr;
  int accepted, column;
  double delta, delta0;
};

// Sketched preconditioner as the loop applies it (see precond_apply1).
struct LoopPrecond {
  int woodbury;
  int m;
  const double* X;    // inverse Cholesky factor (lower), d x d or m x m
  const double* Xt;   // its transpose
  const double* Y;    // m x d float64 sketch (Woodbury), leading dimension ldy
  long long ldy;
  const double* Yt;   // d x m (Woodbury)
  double c;           // sqrt of the sketch scale
};

// One launch: prologue (optional residual pass, optional restart) and then
// iterations until a column fails its test, every column stops, or a column
// reaches max_iter.
struct LoopTask {
  int method;         // 0: adaptive PCG (Algorithm 2); 1: adaptive IHS (Algorithm 1)
  int K;              // lockstep width of the instantiation (1 or 8)
  int kc;             // columns in use (<= K); the rest are inert
  int resid;          // prologue: r = b - H x (PCG) / g = H x - b (IHS) from a pass over A
  int restart;        // prologue: r~ = H_S^{-1} r, p = r~ (PCG), delta~_I = delta~_t, I = t
  int first;          // this restart opens a solve: set dt0, stop_abs = rel2 dt0, outer test
  int can_double;     // m < m_max (and the sketch may grow)
  long long m;        // sketch size (trace)
  long long max_iter; // per column
  double c, phi;      // threshold c(rho) phi(rho)^(t+1-I)
  double mu;          // IHS step 1 - rho
  double tol2;        // stop: dt <= tol2 b^T x (PCG), 2 dt <= tol2 b^T x (IHS)
  double rel2;        // stop: dt <= rel2 dt0 (0: off)
  double outer_tol2;  // first restart: fac dt0 <= outer_tol2 b^T x_o ends the column's refinement (0: off)
  double fac;         // 1 (PCG) or 2 (IHS)
  double nu2;
  const double* lam;
  // vectors: d x K column-major float64 (b, x, r, rt, p, Hp, xp, rp, rtp), scratch t1, t2 (ld x K)
  const double* b;
  double *x, *r, *rt, *p, *Hp, *xp, *rp, *rtp, *t1, *t2;
  long long ld_t;     // leading dimension of t1, t2 (>= max(d, m))
  float* v32;         // float32 copy of the vector the A-pass reads (float32 A-pass), d x K
  void* partials;     // A-pass partial sums [grid * NG][K][d]
  double* dots;       // [grid][K][kLoopDots]
  const double* xstar; // trace mode: the solution (d x K), NULL = off
  LoopCol* cols;      // [K]
  LoopHead* head;
  LoopTraceEv* trace; // optional device trace buffer
  int trace_cap;
  DevStatus* st;
  LoopPrecond P;
};

// Launch of the device-resident loop on the A-pass plan `plan` (a_f32: float32
// A; vec_f32: float32 pass vectors, i.e. the mixed form's inner solve).
// Returns SKS_ERR_UNSUPPORTED when the shape has no loop instantiation (rows
// wider than 4096 columns) or the grid cannot be co-resident; the caller
// then iterates from the host.
sks_status loop_supported(const ApassPlan& plan, int64_t d, int K, bool a_f32, bool vec_f32);
sks_status loop_launch(const ApassPlan& plan, const CUtensorMap* tmap, int64_t n, int64_t d, bool a_f32,
                       bool vec_f32, const LoopTask& task, cudaStream_t stream);
// Drops pipeline stages of an A-pass plan (made by apass_plan, before
// apass_use_bulk) so that the loop's extra shared memory still lets the plan's
// CTAs per SM be resident.
void loop_adjust_plan(ApassPlan* pl, bool a_f32, bool vec_f32);
// Bytes of partial sums and dot partials the loop needs (on top of the vectors).
size_t loop_partial_bytes(const ApassPlan& plan, int64_t d, int K, bool vec_f32);
size_t loop_dots_bytes(const ApassPlan& plan, int K);

}  // namespace sks
