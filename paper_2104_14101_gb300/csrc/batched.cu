// batched.cu -- many independent problems (1) solved together by the adaptive
// PCG of Algorithm 2 with the SRHT embedding of Section 2.1, in the plain
// float64 form or in the mixed form (float32 A, see below).
//
// Every decision of Algorithm 2 (accept / reject, doubling of m, stop) is
// taken on the device, per problem, so one ROUND -- a fixed sequence of
// batched kernels -- advances every unfinished problem by one event: an
// iteration, or a re-sketch with a new factorisation and a restart.  The
// round is captured once as a CUDA graph and replayed until every problem has
// finished; the host reads one counter every few replays.
//
// Per problem p the state machine is
//   INIT  : r = b - H x0                         (one A-pass)      -> GROW
//   GROW  : m <- m_init or min(2m, m_max); rows of the nested SRHT; form and
//           factor the sketched Hessian (d x d Cholesky form when m >= d,
//           m x m Woodbury form otherwise, Section 4.2); r~ = H_S^{-1} r;
//           p = r~, delta~_t = delta~_I = r^T r~                 -> ITER
//   ITER  : one PCG step with the improvement test of Algorithm 2; on
//           rejection I = t                                        -> GROW
//           on acceptance, stop when delta~ <= (tol/2)^2 b^T x   -> DONE
// Mixed form (float32 A, iterative refinement around Algorithm 2): INIT
// computes the refinement residual r = b - H x_o with a double-float pass
// over the float32 A and starts an inner solve of H dx = r from dx = 0
// (t = I = 0); the first restart of the inner solve (GROW when no sketch
// exists yet, else RESTART: r~ = H_S^{-1} r with the current factor) stops
// the whole solve when delta~ <= (tol/2)^2 b^T x_o; inner iterations run
// their A-pass in float32 and end when delta~ <= inner_tol^2 delta~_0, then
// x_o += dx -> INIT.  The sketch (float32 H E A_pad) and m carry over from
// one inner solve to the next; the Gram sums exact float32 products in
// double-float arithmetic on the float32 pipe; factor, apply and the vector
// steps stay in float64.
// A round runs, in order: m update, permutation rows, Gram / Woodbury
// matrix, blocked Cholesky (three kernels per 64-column panel), the A-pass of
// every INIT / ITER problem, its reduction, the first half of the step, the
// preconditioner apply, the second half of the step and the counter.
//
// Work distribution: each batched kernel walks a static list of units (row
// tiles of A, 64 x 64 tiles of a factor, column chunks, problems) over all
// problems with a persistent grid; a unit whose problem is not in the phase
// the kernel serves is skipped.  The A-pass unit height (rows of A per unit)
// is chosen by timing candidate heights on the actual batch (autotuning).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "df32.cuh"
#include "internal.h"
#include "sketch.h"

namespace sks {
namespace {

enum : int { PH_INIT = 0, PH_GROW = 1, PH_ITER = 2, PH_RESTART = 3, PH_DONE = 4, PH_FAIL = 5 };
// d-vector slots of a problem (V_XI: the inner iterate dx of the mixed form)
// V_ISC: 1 / (nu^2 lambda) (mixed form)
enum : int { V_R = 0, V_RT, V_P, V_HV, V_XP, V_RP, V_RTP, V_U, V_W, V_DINV, V_XI, V_ISC, kNumVec };

// phase timers: A-pass, sketched-Hessian matrix (Gram), its factorisation,
// preconditioner apply, the whole round (first kernel to the count kernel)
enum : int { TK_APASS = 0, TK_GRAM, TK_FACTOR, TK_APPLY, TK_ROUND, kTimers };

constexpr int kTile = 64;           // dense tiles and Cholesky panels
constexpr int kTP = kTile + 2;      // padded shared-memory row
constexpr int kMaxD = 1024;         // A-pass: 32 lanes x 32 columns
constexpr int kApWarps = 8;
constexpr int kApThreads = 32 * kApWarps;

struct BDesc {
  const double* A;
  long long lda;
  int64_t n;
  int d, bits;       // n_pad = 2^bits
  const double* b;
  const double* lam;
  double nu2;
  double* x;         // caller's x (x0 on entry)
  const double* B;   // H E A_pad, n_pad x d, ld d (plain form)
  const float* Af;   // mixed form: the float32 A (A is NULL)
  float* Bf;         // mixed form: float32 H E A_pad, n_pad x d, ld d (B is NULL)
  float* ilam;       // mixed form: 1 / lambda rounded to float32 (Woodbury Gram)
  // mixed form: the factor L' = 2^(-sexp) L as float pairs (lower part, its
  // transpose mirrored in the upper part; d x d, ld d) and the inverses of
  // its 64 x 64 diagonal blocks (block b at b * 4096, row-major, zero above
  // the diagonal)
  float2* Lf;
  float2* Lif;
  uint32_t* perm;    // sketch row r is B[perm[r]]
  double* M;         // d x d, ld d: lower = factor L, strict upper = L^T
  double* vec;       // kNumVec d-vectors
  double* part;      // A-pass partial sums, one d-vector per unit
  double* gpart;     // Gram slice partials: [kGramSplit][ntri][64 x 64]
  double* G;         // d x d, ld d: unscaled Y^T Y of the rows summed so far
  int ntri;          // lower 64 x 64 tiles of a d x d matrix
  int64_t m_max, m_init;
};

struct BState {
  int phase, form;   // form 0: Cholesky (N = d), 1: Woodbury (N = m)
  int status, pad;
  int64_t m, m_old, t, I;
  int64_t gram_rows;  // sketch rows already summed into G (Cholesky form)
  int64_t k_begin;    // first sketch row this round's Gram adds
  double dt, dI, btx;
  int64_t rejections, a_passes, factorizations;
  // mixed form: refinement steps done, 1 until the first restart of an inner
  // solve, delta~ at that restart, iterations over all inner solves
  int outer, fresh;
  double d0;
  int64_t t_all;
  int sexp;   // mixed form: the factorisation works on 2^(-2 sexp) M
  int xzero;  // x_0 = 0: the first residual is b, without a pass over A
};

struct BCtl {
  int P;
  int rows_per_unit;
  int64_t max_iter;
  double c, phi, tol2;
  int mixed;           // 1: float32 A with refinement (the mixed form)
  int64_t max_outer;   // mixed form: refinement steps
  double inner2;       // mixed form: inner_tol^2
  Key key;
  const int* pre_tri;  // prefix over problems of T(T+1)/2, T = ceil(d / 64)
  const int* pre_T;    // prefix of T
  const int* pre_ap;   // prefix of ceil(n / rows_per_unit)
  const int* pre_red;  // prefix of ceil(d / 256)
  int* active;         // problems not finished after the round
  // 64-column panels of the largest matrix factored this round (0: no problem
  // grows); set by b_begin_kernel, cleared by the count kernel.  Gram and
  // factorisation launches beyond it return at once instead of walking units.
  int* round_kmax;
  // Phase timers, kTimers x 3: [0] earliest CTA start and [1] latest CTA end
  // of the phase's kernels in this round (%globaltimer ns), [2] the windows
  // summed over rounds (TK_* order; null in the autotuner's launches).
  // flops: 4 n d per A-pass unit row block, summed over rounds
  unsigned long long* tk;
  double* apass_flops;
  double* gram_flops;         // 2 x 64 x 64 per sketch row (or column) of every Gram unit
  // the graph's while loop: rounds run while some problem is unfinished and
  // fewer than max_rounds have run (the count kernel sets the condition)
  cudaGraphConditionalHandle cond;
  int use_cond;        // 0: rounds launched one by one (stepwise mode), no graph condition
  long long* rounds;
  long long max_rounds;
};

// phase timer window: the first CTA start and the last CTA end of a phase
SKS_DEV void tk_start(const BCtl& c, int id) {
  if (threadIdx.x == 0 && c.tk) atomicMin(&c.tk[3 * id], (unsigned long long)global_ns());
}
SKS_DEV void tk_stop(const BCtl& c, int id) {
  if (threadIdx.x == 0 && c.tk) atomicMax(&c.tk[3 * id + 1], (unsigned long long)global_ns());
}

// largest p with pre[p] <= u  (pre[0] = 0 <= u < pre[P])
SKS_DEV int find_problem(const int* __restrict__ pre, int P, int u) {
  int lo = 0, hi = P;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(pre + mid) <= u) lo = mid;
    else hi = mid;
  }
  return lo;
}

SKS_DEV void tri_index(int l, int* ti, int* tj) {
  int i = (int)((sqrtf(8.0f * (float)l + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= l) ++i;
  while (i * (i + 1) / 2 > l) --i;
  *ti = i;
  *tj = l - i * (i + 1) / 2;
}

SKS_DEV double block_dot(int d, const double* a, const double* b, double* scratch) {
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s += a[j] * b[j];
  return block_sum(s, scratch);
}

SKS_DEV int factor_size(const BState& s, const BDesc& q) { return s.form == 0 ? q.d : (int)s.m; }

// ------------------------------------------------------------------ round kernels

__global__ void b_begin_kernel(BCtl c, const BDesc* __restrict__ D, BState* S) {
  if (blockIdx.x == 0) tk_start(c, TK_ROUND);
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= c.P) return;
  BState& s = S[p];
  if (s.phase != PH_GROW) return;
  const BDesc& q = D[p];
  s.m_old = s.m;
  s.m = s.m == 0 ? min(q.m_init, q.m_max) : min(2 * s.m, q.m_max);
  s.form = s.m >= q.d ? 0 : 1;
  // nested sketches: the Cholesky form keeps G = Y^T Y and adds the new rows
  s.k_begin = s.form == 0 ? s.gram_rows : 0;
  if (s.form == 0) s.gram_rows = s.m;
  s.factorizations += 1;
  atomicMax(c.round_kmax, ((s.form == 0 ? q.d : (int)s.m) + kTile - 1) / kTile);
}

// perm[r] = pi(r) for the new sketch rows r in [m_old, m)
__global__ void b_perm_kernel(BCtl c, const BDesc* __restrict__ D, BState* S) {
  if (*c.round_kmax == 0) return;  // no problem grows this round
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    for (int64_t r = s.m_old + threadIdx.x; r < s.m; r += blockDim.x) {
      const uint32_t v = feistel_perm(c.key, (uint32_t)r, q.bits);
      q.perm[r] = v == 0xffffffffu ? 0u : v;
      if (v == 0xffffffffu) {
        S[p].status = SKS_ERR_NUMERIC;
        S[p].phase = PH_FAIL;
      }
    }
  }
}

// acc[i][j] += sum_k As[k][ty*4+i] Bs[k][tx*4+j] for one 16-deep chunk
SKS_DEV void mma_chunk(const double (*As)[kTP], const double (*Bs)[kTP], double acc[4][4], int tx, int ty) {
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const double2 a01 = *(const double2*)&As[k][ty * 4];
    const double2 a23 = *(const double2*)&As[k][ty * 4 + 2];
    const double2 b01 = *(const double2*)&Bs[k][tx * 4];
    const double2 b23 = *(const double2*)&Bs[k][tx * 4 + 2];
    const double a[4] = {a01.x, a01.y, a23.x, a23.y};
    const double b[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
  }
}

// Split of the Gram's sum (over the new sketch rows in the Cholesky form, over
// the d columns in the Woodbury form) into at most kGramSplit slices, summed in
// a fixed order by b_gram_reduce_kernel (deterministic).
constexpr int kGramSplit = 8;
constexpr int kGramSliceRows = 256;  // Cholesky form: new sketch rows per slice (at least)
constexpr int kGramSliceCols = 128;  // Woodbury form: columns of Y per slice (at least)

SKS_DEV int gram_slices(const BState& s, int d) {
  const int64_t k = s.form == 0 ? s.m - s.k_begin : d;
  const int per = s.form == 0 ? kGramSliceRows : kGramSliceCols;
  return min(kGramSplit, max(1, (int)((k + per - 1) / per)));
}

// A Gram unit's 4 x 4 outputs: the raw slice sum to the partial tiles (nks > 1),
// else G (Cholesky form, added to the rows summed before) and the matrix M.
SKS_DEV void gram_epilogue(const BDesc& q, const BState& s, int nks, int ks, int l, int i0, int j0, int N,
                           const double (&acc)[4][4], int tx, int ty) {
  if (nks > 1) {
    double* tile = q.gpart + ((size_t)ks * (size_t)q.ntri + l) * (kTile * kTile);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) tile[(ty * 4 + i) * kTile + tx * 4 + j] = acc[i][j];
    return;
  }
  const int d = q.d;
  const double scale = s.form == 0 ? 1.0 / (double)s.m : 1.0 / ((double)s.m * q.nu2);
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = i0 + ty * 4 + i, gj = j0 + tx * 4 + j;
      if (gi < N && gj < N) {
        double g = acc[i][j];
        if (s.form == 0) {
          double* gp = q.G + (int64_t)gi * d + gj;
          if (s.k_begin > 0) g += *gp;
          *gp = g;
        }
        double v = g * scale;
        if (gi == gj) v += s.form == 0 ? q.nu2 * q.lam[gi] : 1.0;
        q.M[(int64_t)gi * d + gj] = v;
      }
    }
}

// Sketched-Hessian matrix of every GROW problem, lower 64 x 64 tiles:
//   form 0: M = (1/m) G + nu^2 Lambda, G = Y^T Y (Y = rows perm[0..m) of B)
//           kept across doublings: G += Y_new^T Y_new for the rows added
//   form 1: M = I + (1/(m nu^2)) Y Lambda^{-1} Y^T
// Units are (tile, slice); with one slice the tile is written to M, else the
// raw slice sum goes to the problem's partial tiles.
__global__ void __launch_bounds__(256) b_gram_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S,
                                                     int total) {
  if (*c.round_kmax == 0) return;  // no problem grows this round
  __shared__ __align__(16) double As[16][kTP];
  __shared__ __align__(16) double Bs[16][kTP];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  tk_start(c, TK_GRAM);
  double flops = 0.0;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int tu = u / kGramSplit, ks = u - tu * kGramSplit;
    const int p = find_problem(c.pre_tri, c.P, tu);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int nks = gram_slices(s, q.d);
    if (ks >= nks) continue;
    const int l = tu - c.pre_tri[p];
    int ti, tj;
    tri_index(l, &ti, &tj);
    const int N = factor_size(s, q);
    const int i0 = ti * kTile, j0 = tj * kTile;
    if (i0 >= N) continue;
    const int d = q.d;
    const int m = (int)s.m;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    if (s.form == 0) {
      const int k_begin = (int)s.k_begin;
      const int per = ((m - k_begin + nks - 1) / nks + 15) / 16 * 16;
      const int kb = k_begin + ks * per, ke = min(m, kb + per);
      flops += 2.0 * kTile * kTile * (double)max(0, ke - kb);
      for (int k0 = kb; k0 < ke; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * kTile; e += blockDim.x) {
          const int kk = e >> 6, ii = e & 63;
          const int r = k0 + kk;
          double a = 0.0, b = 0.0;
          if (r < ke) {
            const double* y = q.B + (int64_t)q.perm[r] * d;
            if (i0 + ii < N) a = y[i0 + ii];
            if (j0 + ii < N) b = y[j0 + ii];
          }
          As[kk][ii] = a;
          Bs[kk][ii] = b;
        }
        __syncthreads();
        mma_chunk(As, Bs, acc, tx, ty);
        __syncthreads();
      }
    } else {
      const int per = ((d + nks - 1) / nks + 15) / 16 * 16;
      const int cb = ks * per, ce = min(d, cb + per);
      flops += 2.0 * kTile * kTile * (double)max(0, ce - cb);
      for (int k0 = cb; k0 < ce; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * kTile; e += blockDim.x) {
          const int ii = e >> 4, kk = e & 15;
          const int col = k0 + kk;
          double a = 0.0, b = 0.0;
          if (col < ce) {
            if (i0 + ii < N) a = q.B[(int64_t)q.perm[i0 + ii] * d + col] / q.lam[col];
            if (j0 + ii < N) b = q.B[(int64_t)q.perm[j0 + ii] * d + col];
          }
          As[kk][ii] = a;
          Bs[kk][ii] = b;
        }
        __syncthreads();
        mma_chunk(As, Bs, acc, tx, ty);
        __syncthreads();
      }
    }
    gram_epilogue(q, s, nks, ks, l, i0, j0, N, acc, tx, ty);
  }
  tk_stop(c, TK_GRAM);
  if (threadIdx.x == 0 && c.tk && flops > 0) atomicAdd(c.gram_flops, flops);
}

// (hi, lo) += a b: the product exact (TwoProd), summed by Knuth's TwoSum into
// the high part; the rounding errors go to the low part (double-float, ~2^-44
// relative after thousands of terms).  The _rn intrinsics keep the compiler
// from contracting the sums into multiply-adds.
SKS_DEV void df_mac(float a, float b, float& hi, float& lo) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float s = __fadd_rn(hi, p);
  const float z = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, z)), __fsub_rn(p, z)), e));
  hi = s;
}

constexpr int kTPf = kTile + 4;  // float shared-memory row (16-byte aligned quads)

// The Gram units of b_gram_kernel for the mixed form: float32 sketch rows (and
// 1/lambda in float32 for the Woodbury form), exact products summed in
// double-float on the float32 pipe (a float64 Gram runs at 1/64 of its rate
// on this part).
__global__ void __launch_bounds__(256) b_gram_mixed_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S,
                                                           int total) {
  if (*c.round_kmax == 0) return;  // no problem grows this round
  __shared__ __align__(16) float As[16][kTPf];
  __shared__ __align__(16) float Bs[16][kTPf];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  tk_start(c, TK_GRAM);
  double flops = 0.0;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int tu = u / kGramSplit, ks = u - tu * kGramSplit;
    const int p = find_problem(c.pre_tri, c.P, tu);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int nks = gram_slices(s, q.d);
    if (ks >= nks) continue;
    const int l = tu - c.pre_tri[p];
    int ti, tj;
    tri_index(l, &ti, &tj);
    const int N = factor_size(s, q);
    const int i0 = ti * kTile, j0 = tj * kTile;
    if (i0 >= N) continue;
    const int d = q.d;
    const int m = (int)s.m;
    float hi[4][4], lo[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
    int kb, ke;
    if (s.form == 0) {
      const int k_begin = (int)s.k_begin;
      const int per = ((m - k_begin + nks - 1) / nks + 15) / 16 * 16;
      kb = k_begin + ks * per;
      ke = min(m, kb + per);
    } else {
      const int per = ((d + nks - 1) / nks + 15) / 16 * 16;
      kb = ks * per;
      ke = min(d, kb + per);
    }
    flops += 2.0 * kTile * kTile * (double)max(0, ke - kb);
    // the next chunk's elements are loaded into registers while the current
    // one is multiplied (the gathered sketch rows' latency stays hidden)
    constexpr int kPer = 16 * kTile / 256;  // elements per thread and operand
    float pa[kPer], pb[kPer];
    auto fetch = [&](int k0) {
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = threadIdx.x + 256 * t;
        float a = 0.f, b = 0.f;
        if (s.form == 0) {
          const int kk = e >> 6, ii = e & 63;
          const int r = k0 + kk;
          if (r < ke) {
            const float* y = q.Bf + (int64_t)q.perm[r] * d;
            if (i0 + ii < N) a = y[i0 + ii];
            if (j0 + ii < N) b = y[j0 + ii];
          }
        } else {
          const int ii = e >> 4, kk = e & 15;
          const int col = k0 + kk;
          if (col < ke) {
            if (i0 + ii < N) a = __fmul_rn(q.Bf[(int64_t)q.perm[i0 + ii] * d + col], q.ilam[col]);
            if (j0 + ii < N) b = q.Bf[(int64_t)q.perm[j0 + ii] * d + col];
          }
        }
        pa[t] = a;
        pb[t] = b;
      }
    };
    if (kb < ke) fetch(kb);
    for (int k0 = kb; k0 < ke; k0 += 16) {
#pragma unroll
      for (int t = 0; t < kPer; ++t) {
        const int e = threadIdx.x + 256 * t;
        const int kk = s.form == 0 ? e >> 6 : e & 15, ii = s.form == 0 ? e & 63 : e >> 4;
        As[kk][ii] = pa[t];
        Bs[kk][ii] = pb[t];
      }
      __syncthreads();
      if (k0 + 16 < ke) fetch(k0 + 16);
#pragma unroll 4
      for (int k = 0; k < 16; ++k) {
        const float4 a4 = *(const float4*)&As[k][ty * 4];
        const float4 b4 = *(const float4*)&Bs[k][tx * 4];
        const float a[4] = {a4.x, a4.y, a4.z, a4.w};
        const float b[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) df_mac(a[i], b[j], hi[i][j], lo[i][j]);
      }
      __syncthreads();
    }
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = (double)hi[i][j] + (double)lo[i][j];
    gram_epilogue(q, s, nks, ks, l, i0, j0, N, acc, tx, ty);
  }
  tk_stop(c, TK_GRAM);
  if (threadIdx.x == 0 && c.tk && flops > 0) atomicAdd(c.gram_flops, flops);
}

// Sum of the slice partials (slice order fixed), scale and diagonal, into M.
__global__ void __launch_bounds__(256) b_gram_reduce_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S,
                                                            int total) {
  if (*c.round_kmax == 0) return;  // no problem grows this round
  tk_start(c, TK_GRAM);
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_tri, c.P, u);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int nks = gram_slices(s, q.d);
    if (nks <= 1) continue;
    const int l = u - c.pre_tri[p];
    int ti, tj;
    tri_index(l, &ti, &tj);
    const int N = factor_size(s, q);
    const int i0 = ti * kTile, j0 = tj * kTile;
    if (i0 >= N) continue;
    const int d = q.d;
    const double scale = s.form == 0 ? 1.0 / (double)s.m : 1.0 / ((double)s.m * q.nu2);
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int gi = i0 + (e >> 6), gj = j0 + (e & 63);
      if (gi >= N || gj >= N) continue;
      double t = 0.0;
      for (int ks = 0; ks < nks; ++ks) t += q.gpart[((size_t)ks * (size_t)q.ntri + l) * (kTile * kTile) + e];
      if (s.form == 0) {
        double* gp = q.G + (int64_t)gi * d + gj;
        if (s.k_begin > 0) t = *gp + t;
        *gp = t;
      }
      double v = t * scale;
      if (gi == gj) v += s.form == 0 ? q.nu2 * q.lam[gi] : 1.0;
      q.M[(int64_t)gi * d + gj] = v;
    }
  }
  tk_stop(c, TK_GRAM);
}

// Panel k, diagonal block: L_kk = chol(M_kk) in shared memory; writes L_kk
// (lower), L_kk^T (strict upper) and 1 / diag(L_kk).
__global__ void __launch_bounds__(256) b_potrf_kernel(BCtl c, const BDesc* __restrict__ D, BState* S, int k) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  tk_start(c, TK_FACTOR);
  __shared__ double L[kTile][kTile + 1];
  __shared__ int bad;
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int N = factor_size(s, q);
    const int k0 = k * kTile;
    if (k0 >= N) continue;
    const int nb = min(kTile, N - k0);
    const int d = q.d;
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int i = e >> 6, j = e & 63;
      L[i][j] = (i < nb && j <= i) ? q.M[(int64_t)(k0 + i) * d + k0 + j] : 0.0;
    }
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      if (threadIdx.x == 0) {
        const double v = L[j][j];
        if (!(v > 0.0) || !isfinite(v)) {
          bad = j + 1;
          L[j][j] = 1.0;
        } else {
          L[j][j] = sqrt(v);
        }
      }
      __syncthreads();
      if (bad) break;
      const double rjj = 1.0 / L[j][j];
      for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) L[i][j] *= rjj;
      __syncthreads();
      const int w = nb - j - 1;
      for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
        const int ii = e / w, ll = e - ii * w;
        if (ll <= ii) L[j + 1 + ii][j + 1 + ll] -= L[j + 1 + ii][j] * L[j + 1 + ll][j];
      }
      __syncthreads();
    }
    if (bad) {
      if (threadIdx.x == 0) {
        S[p].status = SKS_ERR_NOT_PD;
        S[p].phase = PH_FAIL;
      }
      __syncthreads();
      continue;
    }
    double* dinv = q.vec + (size_t)V_DINV * d;
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      const int i = e / nb, j = e - i * nb;
      if (j <= i) {
        const double v = L[i][j];
        q.M[(int64_t)(k0 + i) * d + k0 + j] = v;
        if (j < i) q.M[(int64_t)(k0 + j) * d + k0 + i] = v;
        else dinv[k0 + i] = 1.0 / v;
      }
    }
    __syncthreads();
  }
  tk_stop(c, TK_FACTOR);
}

// Panel k, blocks below the diagonal: L_ik = M_ik L_kk^{-T} (one thread per
// row, forward substitution), written to the lower part and transposed to the
// upper part.
__global__ void __launch_bounds__(64) b_trsm_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S, int k,
                                                    int total) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  tk_start(c, TK_FACTOR);
  extern __shared__ double tr_smem[];
  double (*L)[kTile + 1] = (double (*)[kTile + 1])tr_smem;                    // [64][65]
  double (*X)[kTile + 1] = (double (*)[kTile + 1])(tr_smem + kTile * (kTile + 1));  // [64][65]
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_T, c.P, u);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int N = factor_size(s, q);
    const int i = u - c.pre_T[p];
    const int k0 = k * kTile, i0 = i * kTile;
    if (i <= k || i0 >= N) continue;
    const int nb = min(kTile, N - k0), rb = min(kTile, N - i0);
    const int d = q.d;
    const double* dinv = q.vec + (size_t)V_DINV * d;
    for (int e = threadIdx.x; e < kTile * kTile; e += blockDim.x) {
      const int a = e >> 6, b = e & 63;
      L[a][b] = (a < nb && b < a) ? q.M[(int64_t)(k0 + a) * d + k0 + b] : 0.0;
      X[a][b] = (a < rb && b < nb) ? q.M[(int64_t)(i0 + a) * d + k0 + b] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x;
    if (r < rb) {
      for (int j = 0; j < nb; ++j) {
        double v = X[r][j];
        for (int l = 0; l < j; ++l) v -= X[r][l] * L[j][l];
        X[r][j] = v * dinv[k0 + j];
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < rb * nb; e += blockDim.x) {
      const int a = e / nb, b = e - a * nb;
      q.M[(int64_t)(i0 + a) * d + k0 + b] = X[a][b];
    }
    for (int e = threadIdx.x; e < rb * nb; e += blockDim.x) {
      const int b = e / rb, a = e - b * rb;
      q.M[(int64_t)(k0 + b) * d + i0 + a] = X[a][b];
    }
    __syncthreads();
  }
  tk_stop(c, TK_FACTOR);
}

// Panel k, trailing update of the lower tiles (ti >= tj > k):
// M_ij -= L_ik L_jk^T.
__global__ void __launch_bounds__(256) b_update_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S, int k,
                                                       int total) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  tk_start(c, TK_FACTOR);
  __shared__ __align__(16) double As[16][kTP];
  __shared__ __align__(16) double Bs[16][kTP];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_tri, c.P, u);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    int ti, tj;
    tri_index(u - c.pre_tri[p], &ti, &tj);
    const int N = factor_size(s, q);
    const int k0 = k * kTile, i0 = ti * kTile, j0 = tj * kTile;
    if (tj <= k || i0 >= N) continue;
    const int nb = min(kTile, N - k0);
    const int d = q.d;
    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
    for (int c0 = 0; c0 < nb; c0 += 16) {
      for (int e = threadIdx.x; e < 16 * kTile; e += blockDim.x) {
        const int ii = e >> 4, kk = e & 15;
        const int col = k0 + c0 + kk;
        double a = 0.0, b = 0.0;
        if (c0 + kk < nb) {
          if (i0 + ii < N) a = q.M[(int64_t)(i0 + ii) * d + col];
          if (j0 + ii < N) b = q.M[(int64_t)(j0 + ii) * d + col];
        }
        As[kk][ii] = a;
        Bs[kk][ii] = b;
      }
      __syncthreads();
      mma_chunk(As, Bs, acc, tx, ty);
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = i0 + ty * 4 + i, gj = j0 + tx * 4 + j;
        if (gi < N && gj < N) q.M[(int64_t)gi * d + gj] -= acc[i][j];
      }
  }
  tk_stop(c, TK_FACTOR);
}

// ---- mixed form: the factorisation in double-float arithmetic
//
// The batch's float64 factorisation is bound, along its chain of 64-column
// panels, by the float64 pipe (two FMAs per clock per SM).  The mixed form
// runs the same blocked Cholesky on the float32 pipe: every M value is split
// into a float pair by integer operations after a power-of-two scaling
// (M' = 2^(-2 sexp) M, largest diagonal entry in [1, 4), so no pair
// underflows), and written back as float64 at its true scale.  The diagonal
// block's kernel also inverts its factor, so the panel below is a product
// (L_ik = M_ik L_kk^{-T}) and the apply multiplies by the block inverses
// instead of running a substitution chain.

// float64 x 2^sh -> float pair, and back (integer operations but one float64 add)
SKS_DEV F2 to_f2(double v, int sh) { return split_f64(scale_pow2(v, sh)); }
SKS_DEV double from_f2(F2 v, int sh) { return scale_pow2(f32_to_f64_bits(v.h) + f32_to_f64_bits(v.l), sh); }

// Panel k, diagonal block, mixed form: L_kk = chol(M_kk) and X = L_kk^{-1},
// both right-looking, in registers: thread (c, g) holds column c, rows
// g + 16q (q < 4) of the block and of X (1024 threads: enough warps to hide
// the latency of the double-float chains between the step's barriers).  Step j: the pivot's owner
// publishes it; the four owners of column j scale it and publish it; every
// thread updates its trailing entries with column j, the owners of row j of
// X scale that row and publish it, and every thread updates its rows of X
// below j.  Writes L_kk (lower), L_kk^T (strict upper) and X (Li block k).
// At k = 0 the CTA first picks the problem's scaling exponent.
constexpr int kPotThreads = 1024;                    // 16 threads per column of the block
constexpr int kPotRows = kTile / (kPotThreads / kTile);  // rows per thread (4)

__global__ void __launch_bounds__(kPotThreads) b_potrf_df_kernel(BCtl c, const BDesc* __restrict__ D, BState* S,
                                                                 int k) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  __shared__ F2 colv[kTile], xrow[kTile];
  __shared__ F2 s_piv, s_r;
  __shared__ int s_bad, s_emax;
  constexpr int NGR = kPotThreads / kTile;  // row groups
  tk_start(c, TK_FACTOR);
  const int tid = threadIdx.x, cc = tid & 63, g = tid >> 6;
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    const BDesc& q = D[p];
    const int N = factor_size(s, q);
    const int k0 = k * kTile;
    if (k0 >= N) continue;
    const int nb = min(kTile, N - k0);
    const int d = q.d;
    int te;
    if (k == 0) {
      if (tid == 0) s_emax = -1100;
      __syncthreads();
      int e = -1100;
      for (int i = tid; i < N; i += blockDim.x) {
        const long long b = __double_as_longlong(q.M[(int64_t)i * d + i]);
        const int E = (int)((b >> 52) & 0x7ff);
        if (b > 0 && E > 0 && E < 0x7ff) e = max(e, E - 1023);
      }
      atomicMax(&s_emax, e);
      __syncthreads();
      const int em = s_emax > -1000 ? s_emax : 0;
      te = (em - (em & 1)) / 2;  // 2 te <= em < 2 te + 2
      if (tid == 0) S[p].sexp = te;
    } else {
      te = s.sexp;
    }
    F2 v[kPotRows], xi[kPotRows];
#pragma unroll
    for (int r = 0; r < kPotRows; ++r) {
      const int i = g + NGR * r;
      v[r] = (i < nb && cc <= i) ? to_f2(q.M[(int64_t)(k0 + i) * d + k0 + cc], -2 * te) : F2{0.f, 0.f};
      xi[r] = (i < nb && cc == i) ? F2{1.f, 0.f} : F2{0.f, 0.f};
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      const int jr = j / NGR, jg = j % NGR;
      if (cc == j && g == jg) {
#pragma unroll
        for (int r = 0; r < kPotRows; ++r)
          if (r == jr) s_piv = v[r];
      }
      __syncthreads();
      if (cc == j) {
        const F2 pv = s_piv;
        if (!(pv.h > 0.f) || !isfinite(pv.h)) {
          if (g == jg) s_bad = j + 1;
        } else {
          const F2 r = f2_rsqrt(pv);  // 1 / L_jj
#pragma unroll
          for (int rr = 0; rr < kPotRows; ++rr) {
            const int i = g + NGR * rr;
            if (i > j && i < nb) {
              v[rr] = f2_mul(v[rr], r);
              colv[i] = v[rr];
            } else if (i == j) {
              v[rr] = f2_mul(pv, r);  // L_jj = p / sqrt(p)
              s_r = r;
            }
          }
        }
      }
      __syncthreads();
      if (s_bad) break;
      if (cc > j) {
        const F2 lc = colv[cc];
#pragma unroll
        for (int rr = 0; rr < kPotRows; ++rr) {
          const int i = g + NGR * rr;
          if (i >= cc && i < nb) f2_acc<true>(v[rr].h, v[rr].l, colv[i], lc);
        }
      }
      if (g == jg && cc <= j) {
        const F2 r = s_r;
#pragma unroll
        for (int rr = 0; rr < kPotRows; ++rr)
          if (rr == jr) {
            xi[rr] = f2_mul(xi[rr], r);
            xrow[cc] = xi[rr];
          }
      }
      __syncthreads();
      if (cc <= j) {
        const F2 xj = xrow[cc];
#pragma unroll
        for (int rr = 0; rr < kPotRows; ++rr) {
          const int i = g + NGR * rr;
          if (i > j && i < nb) f2_acc<true>(xi[rr].h, xi[rr].l, colv[i], xj);
        }
      }
    }
    if (s_bad) {
      if (tid == 0) {
        S[p].status = SKS_ERR_NOT_PD;
        S[p].phase = PH_FAIL;
      }
      __syncthreads();
      continue;
    }
    float2* Lib = q.Lif + (size_t)k * (kTile * kTile);
#pragma unroll
    for (int rr = 0; rr < kPotRows; ++rr) {
      const int i = g + NGR * rr;
      if (i < nb && cc <= i) {
        const float2 val = make_float2(v[rr].h, v[rr].l);
        q.Lf[(int64_t)(k0 + i) * d + k0 + cc] = val;
        if (cc < i) q.Lf[(int64_t)(k0 + cc) * d + k0 + i] = val;
      }
      Lib[i * kTile + cc] = (i < nb && cc <= i) ? make_float2(xi[rr].h, xi[rr].l) : make_float2(0.f, 0.f);
    }
    __syncthreads();
  }
  tk_stop(c, TK_FACTOR);
}

// acc[i][j] += sum over 16 steps of a[k][ty*4+i] b[k][tx*4+j] in double-float
SKS_DEV void df_tile_chunk(const float (*Ah)[kTPf], const float (*Al)[kTPf], const float (*Bh)[kTPf],
                           const float (*Bl)[kTPf], F2 (&acc)[4][4], int tx, int ty) {
#pragma unroll 2
  for (int k = 0; k < 16; ++k) {
    const float4 ah = *(const float4*)&Ah[k][ty * 4], al = *(const float4*)&Al[k][ty * 4];
    const float4 bh = *(const float4*)&Bh[k][tx * 4], bl = *(const float4*)&Bl[k][tx * 4];
    const F2 a[4] = {{ah.x, al.x}, {ah.y, al.y}, {ah.z, al.z}, {ah.w, al.w}};
    const F2 b[4] = {{bh.x, bl.x}, {bh.y, bl.y}, {bh.z, bl.z}, {bh.w, bl.w}};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) f2_acc<false>(acc[i][j].h, acc[i][j].l, a[i], b[j]);
  }
}

// one operand element: float64 scaled by 2^sh and split, or a float pair as is
SKS_DEV F2 ld_f2(const double* p, int64_t i, int sh) { return to_f2(p[i], sh); }
SKS_DEV F2 ld_f2(const float2* p, int64_t i, int) {
  const float2 v = p[i];
  return F2{v.x, v.y};
}

// acc = A B^T for a 64 x 64 output tile: A rows ra (< na valid), B rows rb
// (< nbv valid), K columns (both row-major; float64 operands scaled by
// 2^sha / 2^shb on the way in, float-pair operands taken as they are).
template <typename TA, typename TB>
SKS_DEV void df_tile_abt(const TA* __restrict__ A, int64_t lda, int na, int sha, const TB* __restrict__ B,
                         int64_t ldb, int nbv, int shb, int K, F2 (&acc)[4][4], float (*Ah)[kTPf],
                         float (*Al)[kTPf], float (*Bh)[kTPf], float (*Bl)[kTPf]) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = F2{0.f, 0.f};
  // the next 16 columns are loaded into registers (raw values, split when
  // stored) while the current ones are multiplied; 256 threads, 4 elements
  // of each operand per thread
  constexpr int kPer = 16 * kTile / 256;
  TA ra[kPer];
  TB rb[kPer];
  auto fetch = [&](int c0) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = threadIdx.x + 256 * t;
      const int ii = e >> 4, col = c0 + (e & 15);
      ra[t] = (col < K && ii < na) ? A[(int64_t)ii * lda + col] : TA{};
      rb[t] = (col < K && ii < nbv) ? B[(int64_t)ii * ldb + col] : TB{};
    }
  };
  if (K > 0) fetch(0);
  for (int c0 = 0; c0 < K; c0 += 16) {
#pragma unroll
    for (int t = 0; t < kPer; ++t) {
      const int e = threadIdx.x + 256 * t;
      const int ii = e >> 4, kk = e & 15;
      const F2 a = ld_f2(ra + t, 0, sha), b = ld_f2(rb + t, 0, shb);
      Ah[kk][ii] = a.h;
      Al[kk][ii] = a.l;
      Bh[kk][ii] = b.h;
      Bl[kk][ii] = b.l;
    }
    __syncthreads();
    if (c0 + 16 < K) fetch(c0 + 16);
    df_tile_chunk(Ah, Al, Bh, Bl, acc, tx, ty);
    __syncthreads();
  }
}

// Panel k, blocks below the diagonal, mixed form: L_ik = M_ik L_kk^{-T}
// (a product with the block inverse), to the lower part and transposed to
// the upper part.
__global__ void __launch_bounds__(256) b_trsm_df_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S, int k,
                                                        int total) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  __shared__ __align__(16) float Ah[16][kTPf], Al[16][kTPf], Bh[16][kTPf], Bl[16][kTPf];
  tk_start(c, TK_FACTOR);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_T, c.P, u);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    const int N = factor_size(s, q);
    const int i = u - c.pre_T[p];
    const int k0 = k * kTile, i0 = i * kTile;
    if (i <= k || i0 >= N) continue;
    const int nb = min(kTile, N - k0), rb = min(kTile, N - i0);
    const int d = q.d, te = s.sexp;
    F2 acc[4][4];
    // M'_ik (2^-2te M) times (L'_kk)^{-T}: L'_ik = 2^-te L_ik
    df_tile_abt(q.M + (int64_t)i0 * d + k0, d, rb, -2 * te, q.Lif + (size_t)k * (kTile * kTile), kTile, nb, 0,
                nb, acc, Ah, Al, Bh, Bl);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int r = ty * 4 + a, cl = tx * 4 + b;
        if (r < rb && cl < nb) {
          const float2 val = make_float2(acc[a][b].h, acc[a][b].l);
          q.Lf[(int64_t)(i0 + r) * d + k0 + cl] = val;
          q.Lf[(int64_t)(k0 + cl) * d + i0 + r] = val;
        }
      }
  }
  tk_stop(c, TK_FACTOR);
}

// Panel k, trailing update of the lower tiles (ti >= tj > k), mixed form:
// M_ij -= L_ik L_jk^T with the product in double-float.
__global__ void __launch_bounds__(256) b_update_df_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S, int k,
                                                          int total) {
  if (k >= *c.round_kmax) return;  // no matrix of this round has panel k
  __shared__ __align__(16) float Ah[16][kTPf], Al[16][kTPf], Bh[16][kTPf], Bl[16][kTPf];
  tk_start(c, TK_FACTOR);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_tri, c.P, u);
    if (S[p].phase != PH_GROW) continue;
    const BState s = S[p];
    if (s.phase != PH_GROW) continue;
    const BDesc& q = D[p];
    int ti, tj;
    tri_index(u - c.pre_tri[p], &ti, &tj);
    const int N = factor_size(s, q);
    const int k0 = k * kTile, i0 = ti * kTile, j0 = tj * kTile;
    if (tj <= k || i0 >= N) continue;
    const int nb = min(kTile, N - k0);
    const int d = q.d, te = s.sexp;
    F2 acc[4][4];
    // L'_ik L'_jk^T = 2^-2te L_ik L_jk^T
    df_tile_abt(q.Lf + (int64_t)i0 * d + k0, d, min(kTile, N - i0), 0, q.Lf + (int64_t)j0 * d + k0, d,
                min(kTile, N - j0), 0, nb, acc, Ah, Al, Bh, Bl);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
        if (gi < N && gj < N) q.M[(int64_t)gi * d + gj] -= from_f2(acc[a][b], 2 * te);
      }
  }
  tk_stop(c, TK_FACTOR);
}

// One A-pass unit: rows [r0, r1) of A against v (in shared memory); warp w
// takes rows r0 + w, r0 + w + 8, ...; lane l owns columns l + 32 j (j < QC).
template <int QC>
SKS_DEV void apass_unit(const double* __restrict__ A, long long lda, int d, int64_t r0, int64_t r1,
                        const double* vs, double* red, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc[QC];
#pragma unroll
  for (int j = 0; j < QC; ++j) acc[j] = 0.0;
  for (int64_t r = r0 + warp; r < r1; r += kApWarps) {
    const double* a = A + r * lda;
    double av[QC];
    double dot = 0.0;
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const int col = lane + 32 * j;
      av[j] = col < d ? __ldg(a + col) : 0.0;
    }
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const int col = lane + 32 * j;
      if (col < d) dot = fma(av[j], vs[col], dot);
    }
    dot = warp_sum(dot);
#pragma unroll
    for (int j = 0; j < QC; ++j) acc[j] = fma(dot, av[j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < QC; ++j) {
    const int col = lane + 32 * j;
    if (col < d) red[warp * d + col] = acc[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < d; col += blockDim.x) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kApWarps; ++w) t += red[w * d + col];
    out[col] = t;
  }
  __syncthreads();
}

// A-pass of every INIT (v = x) and ITER (v = p) problem: one partial
// d-vector per unit of rows_per_unit rows.
__global__ void __launch_bounds__(kApThreads, 1) b_apass_kernel(BCtl c, const BDesc* __restrict__ D,
                                                                const BState* S, int total) {
  extern __shared__ __align__(16) double ap_smem[];
  double* vs = ap_smem;            // [d]
  double* red = ap_smem + kMaxD;   // [8][d]
  tk_start(c, TK_APASS);
  double flops = 0.0;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_ap, c.P, u);
    const int phase = S[p].phase;
    if (phase != PH_INIT && phase != PH_ITER) continue;
    if (phase == PH_INIT && S[p].xzero) continue;  // H x_0 = 0
    const BDesc& q = D[p];
    const int d = q.d;
    const double* v = phase == PH_INIT ? q.x : q.vec + (size_t)V_P * d;
    for (int j = threadIdx.x; j < d; j += blockDim.x) vs[j] = v[j];
    __syncthreads();
    const int t = u - c.pre_ap[p];
    const int64_t r0 = (int64_t)t * c.rows_per_unit;
    const int64_t r1 = min(q.n, r0 + c.rows_per_unit);
    double* out = q.part + (size_t)t * d;
    if (d <= 32) apass_unit<1>(q.A, q.lda, d, r0, r1, vs, red, out);
    else if (d <= 64) apass_unit<2>(q.A, q.lda, d, r0, r1, vs, red, out);
    else if (d <= 128) apass_unit<4>(q.A, q.lda, d, r0, r1, vs, red, out);
    else if (d <= 256) apass_unit<8>(q.A, q.lda, d, r0, r1, vs, red, out);
    else if (d <= 512) apass_unit<16>(q.A, q.lda, d, r0, r1, vs, red, out);
    else apass_unit<32>(q.A, q.lda, d, r0, r1, vs, red, out);
    flops += 4.0 * (double)(r1 - r0) * d;
  }
  tk_stop(c, TK_APASS);
  if (threadIdx.x == 0 && c.tk && flops > 0) atomicAdd(c.apass_flops, flops);
}

// ---- mixed form A-pass (float32 A)
SKS_DEV void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}
// (h, l) += (bh, bl), renormalised
SKS_DEV void df_add2(float& h, float& l, float bh, float bl) {
  float s, e;
  df_two_sum(h, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(l, bl));
  h = __fadd_rn(s, e);
  l = __fsub_rn(e, __fsub_rn(h, s));
}

// Inner iterations: rows [r0, r1) of the float32 A against p rounded to
// float32 (vs), float32 sums; the unit's d partial sums leave as float64.
// A warp takes RR rows at a time (their loads in flight together, their dot
// reductions interleaved): narrow rows need several to keep HBM busy.
template <int QC, int RR>
SKS_DEV void apass_unit_f32(const float* __restrict__ A, long long lda, int d, int64_t r0, int64_t r1,
                            const float* vs, float* red, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[QC];
  float xv[QC];
#pragma unroll
  for (int j = 0; j < QC; ++j) {
    acc[j] = 0.f;
    const int col = lane + 32 * j;
    xv[j] = col < d ? vs[col] : 0.f;
  }
  for (int64_t r = r0 + warp; r < r1; r += (int64_t)kApWarps * RR) {
    float av[RR][QC];
    float dot[RR];
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      const int64_t rk = r + (int64_t)k * kApWarps;
      const float* a = A + rk * lda;
#pragma unroll
      for (int j = 0; j < QC; ++j) {
        const int col = lane + 32 * j;
        av[k][j] = (rk < r1 && col < d) ? __ldg(a + col) : 0.f;
      }
    }
#pragma unroll
    for (int k = 0; k < RR; ++k) {
      dot[k] = 0.f;
#pragma unroll
      for (int j = 0; j < QC; ++j) dot[k] = fmaf(av[k][j], xv[j], dot[k]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < RR; ++k) dot[k] += __shfl_xor_sync(0xffffffffu, dot[k], o);
#pragma unroll
    for (int k = 0; k < RR; ++k)
#pragma unroll
      for (int j = 0; j < QC; ++j) acc[j] = fmaf(dot[k], av[k][j], acc[j]);
  }
#pragma unroll
  for (int j = 0; j < QC; ++j) {
    const int col = lane + 32 * j;
    if (col < d) red[warp * d + col] = acc[j];
  }
  __syncthreads();
  for (int col = threadIdx.x; col < d; col += blockDim.x) {
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kApWarps; ++w) t += red[w * d + col];
    out[col] = (double)t;
  }
  __syncthreads();
}

// Refinement residual: rows [r0, r1) of the float32 A against x_o split into
// two floats (xh + xl), every product exact (TwoProd) and every sum in
// double-float; the unit's partial sums leave as float64 (hi + lo).
template <int QC>
SKS_DEV void apass_unit_df(const float* __restrict__ A, long long lda, int d, int64_t r0, int64_t r1,
                           const float* xh, const float* xl, float* redh, float* redl, double* __restrict__ out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float ah[QC], al[QC];
#pragma unroll
  for (int j = 0; j < QC; ++j) ah[j] = al[j] = 0.f;
  for (int64_t r = r0 + warp; r < r1; r += kApWarps) {
    const float* a = A + r * lda;
    float av[QC];
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const int col = lane + 32 * j;
      av[j] = col < d ? __ldg(a + col) : 0.f;
    }
    float sh = 0.f, sl = 0.f;
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const int col = lane + 32 * j;
      if (col < d) {
        const float p = __fmul_rn(av[j], xh[col]);
        const float e = __fmaf_rn(av[j], xl[col], __fmaf_rn(av[j], xh[col], -p));
        float t, u;
        df_two_sum(sh, p, t, u);
        sh = t;
        sl = __fadd_rn(sl, __fadd_rn(u, e));
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
      df_add2(sh, sl, oh, ol);
    }
    // acc_j += a_j (sh + sl)
#pragma unroll
    for (int j = 0; j < QC; ++j) {
      const float p = __fmul_rn(av[j], sh);
      const float e = __fmaf_rn(av[j], sl, __fmaf_rn(av[j], sh, -p));
      float t, u;
      df_two_sum(ah[j], p, t, u);
      ah[j] = t;
      al[j] = __fadd_rn(al[j], __fadd_rn(u, e));
    }
  }
#pragma unroll
  for (int j = 0; j < QC; ++j) {
    const int col = lane + 32 * j;
    if (col < d) {
      redh[warp * d + col] = ah[j];
      redl[warp * d + col] = al[j];
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < d; col += blockDim.x) {
    float h = redh[col], l = redl[col];
#pragma unroll
    for (int w = 1; w < kApWarps; ++w) df_add2(h, l, redh[w * d + col], redl[w * d + col]);
    out[col] = (double)h + (double)l;
  }
  __syncthreads();
}

// Mixed-form A-pass: DF = true serves the INIT problems (v = x_o, double-
// float), DF = false the ITER problems (v = p, float32).  tune = 1 (unit-
// height timing only) runs every unit as ITER.
template <bool DF>
__global__ void __launch_bounds__(kApThreads) b_apass_mixed_kernel(BCtl c, const BDesc* __restrict__ D,
                                                                   const BState* S, int total, int tune) {
  extern __shared__ __align__(16) float apf_smem[];
  float* vh = apf_smem;                     // [d]
  float* vl = apf_smem + kMaxD;             // [d] (DF only)
  float* redh = apf_smem + (DF ? 2 : 1) * kMaxD;   // [8][d]
  float* redl = redh + kApWarps * kMaxD;    // [8][d] (DF only)
  tk_start(c, TK_APASS);
  double flops = 0.0;
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_ap, c.P, u);
    const int phase = S[p].phase;
    if (!tune && phase != (DF ? PH_INIT : PH_ITER)) continue;
    if (DF && !tune && S[p].xzero && S[p].outer == 0) continue;  // H x_0 = 0
    const BDesc& q = D[p];
    const int d = q.d;
    if (DF) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double x = q.x[j];
        const float h = (float)x;
        vh[j] = h;
        vl[j] = (float)(x - (double)h);
      }
    } else {
      const double* v = q.vec + (size_t)V_P * d;
      for (int j = threadIdx.x; j < d; j += blockDim.x) vh[j] = (float)v[j];
    }
    __syncthreads();
    const int t = u - c.pre_ap[p];
    const int64_t r0 = (int64_t)t * c.rows_per_unit;
    const int64_t r1 = min(q.n, r0 + c.rows_per_unit);
    double* out = q.part + (size_t)t * d;
    if (DF) {
      if (d <= 32) apass_unit_df<1>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
      else if (d <= 64) apass_unit_df<2>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
      else if (d <= 128) apass_unit_df<4>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
      else if (d <= 256) apass_unit_df<8>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
      else if (d <= 512) apass_unit_df<16>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
      else apass_unit_df<32>(q.Af, q.lda, d, r0, r1, vh, vl, redh, redl, out);
    } else {
      if (d <= 32) apass_unit_f32<1, 8>(q.Af, q.lda, d, r0, r1, vh, redh, out);
      else if (d <= 64) apass_unit_f32<2, 8>(q.Af, q.lda, d, r0, r1, vh, redh, out);
      else if (d <= 128) apass_unit_f32<4, 4>(q.Af, q.lda, d, r0, r1, vh, redh, out);
      else if (d <= 256) apass_unit_f32<8, 2>(q.Af, q.lda, d, r0, r1, vh, redh, out);
      else if (d <= 512) apass_unit_f32<16, 2>(q.Af, q.lda, d, r0, r1, vh, redh, out);
      else apass_unit_f32<32, 1>(q.Af, q.lda, d, r0, r1, vh, redh, out);
    }
    flops += 4.0 * (double)(r1 - r0) * d;
  }
  tk_stop(c, TK_APASS);
  if (threadIdx.x == 0 && c.tk && flops > 0) atomicAdd(c.apass_flops, flops);
}
constexpr size_t apass_mixed_smem(bool df) { return (size_t)(df ? 2 + 2 * kApWarps : 1 + kApWarps) * kMaxD * 4; }

// Hv = sum of the unit partials + nu^2 Lambda v, in chunks of 256 columns.
__global__ void __launch_bounds__(256) b_reduce_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S,
                                                       int total) {
  for (int u = blockIdx.x; u < total; u += gridDim.x) {
    const int p = find_problem(c.pre_red, c.P, u);
    const int phase = S[p].phase;
    if (phase != PH_INIT && phase != PH_ITER) continue;
    const BDesc& q = D[p];
    const int d = q.d;
    const int col = (u - c.pre_red[p]) * 256 + threadIdx.x;
    if (col >= d) continue;
    if (phase == PH_INIT && S[p].xzero && S[p].outer == 0) {  // H x_0 = 0: no pass was made
      q.vec[(size_t)V_HV * d + col] = 0.0;
      continue;
    }
    const int units = (int)((q.n + c.rows_per_unit - 1) / c.rows_per_unit);
    const double* v = phase == PH_INIT ? q.x : q.vec + (size_t)V_P * d;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    int t = 0;
    for (; t + 3 < units; t += 4) {
      s0 += q.part[(size_t)t * d + col];
      s1 += q.part[(size_t)(t + 1) * d + col];
      s2 += q.part[(size_t)(t + 2) * d + col];
      s3 += q.part[(size_t)(t + 3) * d + col];
    }
    for (; t < units; ++t) s0 += q.part[(size_t)t * d + col];
    q.vec[(size_t)V_HV * d + col] = ((s0 + s1) + (s2 + s3)) + q.nu2 * q.lam[col] * v[col];
  }
}

// INIT: r = b - H x.   ITER: alpha = delta~_t / p^T H p, x+ = x + alpha p, r+ = r - alpha H p.
__global__ void __launch_bounds__(256) b_step1_kernel(BCtl c, const BDesc* __restrict__ D, BState* S) {
  __shared__ double scratch[32];
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    const int phase = S[p].phase;
    if (phase != PH_INIT && phase != PH_ITER) continue;
    const BDesc& q = D[p];
    const int d = q.d;
    double* r = q.vec + (size_t)V_R * d;
    const double* Hv = q.vec + (size_t)V_HV * d;
    if (phase == PH_INIT) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) r[j] = q.b[j] - Hv[j];
      if (c.mixed) {
        // a new inner solve of H dx = r from dx = 0; b^T x_o for the stop rule
        double* xi = q.vec + (size_t)V_XI * d;
        for (int j = threadIdx.x; j < d; j += blockDim.x) xi[j] = 0.0;
        const double btx = block_dot(d, q.b, q.x, scratch);
        if (threadIdx.x == 0) {
          S[p].btx = btx;
          S[p].t = 0;
          S[p].I = 0;
        }
      }
    } else {
      const double* pv = q.vec + (size_t)V_P * d;
      const double* xc = c.mixed ? q.vec + (size_t)V_XI * d : q.x;
      const double pHp = block_dot(d, pv, Hv, scratch);
      const double alpha = S[p].dt / pHp;
      const bool bad = !(pHp > 0.0) || !isfinite(alpha);
      double* xp = q.vec + (size_t)V_XP * d;
      double* rp = q.vec + (size_t)V_RP * d;
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        xp[j] = xc[j] + alpha * pv[j];
        rp[j] = r[j] - alpha * Hv[j];
      }
      if (bad && threadIdx.x == 0) {
        S[p].status = SKS_ERR_NUMERIC;
        S[p].phase = PH_FAIL;
      }
    }
    if (threadIdx.x == 0 && !(phase == PH_INIT && S[p].xzero && S[p].outer == 0)) S[p].a_passes += 1;
    __syncthreads();
  }
}

// y = L^{-1} z (lower, forward) or U^{-1} z (upper = L^T, backward) for the
// N x N factor in M (ld), in place on the shared vector y.  Blocks of 64: the
// off-diagonal part as one warp per row, the diagonal block by warp 0.
SKS_DEV void tri_solve(const double* __restrict__ M, int ld, int N, const double* __restrict__ dinv, double* y,
                       bool upper) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nblk = (N + kTile - 1) / kTile;
  for (int bi = 0; bi < nblk; ++bi) {
    const int blk = upper ? nblk - 1 - bi : bi;
    const int b0 = blk * kTile, nb = min(kTile, N - b0);
    // y[b0 + i] -= sum over the solved part
    const int j0 = upper ? b0 + nb : 0, j1 = upper ? N : b0;
    if (j1 > j0) {
      for (int i = warp; i < nb; i += nw) {
        const double* row = M + (int64_t)(b0 + i) * ld;
        double s = 0.0;
        for (int j = j0 + lane; j < j1; j += 32) s = fma(row[j], y[j], s);
        s = warp_sum(s);
        if (lane == 0) y[b0 + i] -= s;
      }
    }
    __syncthreads();
    if (warp == 0) {
      for (int jj = 0; jj < nb; ++jj) {
        const int j = upper ? nb - 1 - jj : jj;
        const double yj = y[b0 + j] * dinv[b0 + j];
        __syncwarp();
        if (lane == 0) y[b0 + j] = yj;
        if (upper) {
          for (int i = lane; i < j; i += 32) y[b0 + i] -= M[(int64_t)(b0 + i) * ld + b0 + j] * yj;
        } else {
          for (int i = j + 1 + lane; i < nb; i += 32) y[b0 + i] -= M[(int64_t)(b0 + i) * ld + b0 + j] * yj;
        }
        __syncwarp();
      }
    }
    __syncthreads();
  }
}

// GROW: r~ = H_S^{-1} r.   ITER: r~+ = H_S^{-1} r+.
//   form 0: H_S = L L^T (two triangular solves)
//   form 1: H_S^{-1} z = u - (nu^2 Lambda)^{-1} Y_s^T K^{-1} Y_s u,  u = (nu^2 Lambda)^{-1} z,
//           Y_s = Y / sqrt(m), K = I + Y_s (nu^2 Lambda)^{-1} Y_s^T = L L^T
__global__ void __launch_bounds__(512) b_apply_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S) {
  tk_start(c, TK_APPLY);
  __shared__ double y[kMaxD];
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    const BState s = S[p];
    if (s.phase != PH_GROW && s.phase != PH_ITER && s.phase != PH_RESTART) continue;
    const BDesc& q = D[p];
    const int d = q.d;
    const bool restart = s.phase != PH_ITER;
    const double* z = q.vec + (size_t)(restart ? V_R : V_RP) * d;
    double* out = q.vec + (size_t)(restart ? V_RT : V_RTP) * d;
    const double* dinv = q.vec + (size_t)V_DINV * d;
    if (s.form == 0) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) y[j] = z[j];
      __syncthreads();
      tri_solve(q.M, d, d, dinv, y, false);
      tri_solve(q.M, d, d, dinv, y, true);
      for (int j = threadIdx.x; j < d; j += blockDim.x) out[j] = y[j];
    } else {
      const int m = (int)s.m;
      const double ism = 1.0 / sqrt((double)m);
      double* u = q.vec + (size_t)V_U * d;
      for (int j = threadIdx.x; j < d; j += blockDim.x) u[j] = z[j] / (q.nu2 * q.lam[j]);
      __syncthreads();
      const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
      for (int r = warp; r < m; r += nw) {
        const int64_t off = (int64_t)q.perm[r] * d;
        double t = 0.0;
        if (q.Bf) {
          for (int j = lane; j < d; j += 32) t = fma((double)q.Bf[off + j], u[j], t);
        } else {
          for (int j = lane; j < d; j += 32) t = fma(q.B[off + j], u[j], t);
        }
        t = warp_sum(t);
        if (lane == 0) y[r] = t * ism;
      }
      __syncthreads();
      tri_solve(q.M, d, m, dinv, y, false);
      tri_solve(q.M, d, m, dinv, y, true);
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        double t = 0.0;
        if (q.Bf) {
          for (int r = 0; r < m; ++r) t = fma((double)q.Bf[(int64_t)q.perm[r] * d + j], y[r], t);
        } else {
          for (int r = 0; r < m; ++r) t = fma(q.B[(int64_t)q.perm[r] * d + j], y[r], t);
        }
        out[j] = u[j] - t * ism / (q.nu2 * q.lam[j]);
      }
    }
    __syncthreads();
  }
  tk_stop(c, TK_APPLY);
}

// ---- mixed form: the preconditioner apply in double-float
SKS_DEV F2 f2_add(F2 a, F2 b) {
  const F2 s = f2_two_sum(a.h, b.h);
  return f2_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
SKS_DEV F2 warp_sum_f2(F2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = f2_add(v, F2{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)});
  return v;
}
// largest binary exponent of |v[0..n)| over the block (0 if every entry is 0)
SKS_DEV int block_max_exp(const double* v, int n, int* s_e) {
  if (threadIdx.x == 0) *s_e = -2000;
  __syncthreads();
  int e = -2000;
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int E = (int)((__double_as_longlong(v[j]) >> 52) & 0x7ff);
    if (E > 0 && E < 0x7ff) e = max(e, E - 1023);
  }
  atomicMax(s_e, e);
  __syncthreads();
  const int r = *s_e;
  __syncthreads();
  return r > -2000 ? r : 0;
}

// yd[0..N) <- (L L^T)^{-1} yd with the float-pair factor L' = 2^-te L of the
// problem (Lf, Lif): the vector scaled by a power of two into range, blocked
// forward and backward solves (off-diagonal part one warp per row, the
// diagonal block as a product with its inverse), scaled back.
SKS_DEV void df_chol_solve(const BDesc& q, int N, int te, double* yd, F2* yf, F2* tmpf, int* s_e) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int d = q.d;
  const int ez = block_max_exp(yd, N, s_e);
  for (int j = threadIdx.x; j < N; j += blockDim.x) yf[j] = to_f2(yd[j], -ez);
  __syncthreads();
  const int nblk = (N + kTile - 1) / kTile;
  for (int pass = 0; pass < 2; ++pass) {
    const bool upper = pass == 1;
    for (int bi = 0; bi < nblk; ++bi) {
      const int blk = upper ? nblk - 1 - bi : bi;
      const int b0 = blk * kTile, nb = min(kTile, N - b0);
      const int j0 = upper ? b0 + nb : 0, j1 = upper ? N : b0;
      if (j1 > j0) {
        for (int i = warp; i < nb; i += nw) {
          const float2* row = q.Lf + (int64_t)(b0 + i) * d;
          F2 acc = {0.f, 0.f}, acc2 = {0.f, 0.f};
          int j = j0 + lane;
          for (; j + 96 < j1; j += 128) {  // four loads in flight per lane
            const float2 a0 = row[j], a1 = row[j + 32], a2 = row[j + 64], a3 = row[j + 96];
            f2_acc<false>(acc.h, acc.l, F2{a0.x, a0.y}, yf[j]);
            f2_acc<false>(acc2.h, acc2.l, F2{a1.x, a1.y}, yf[j + 32]);
            f2_acc<false>(acc.h, acc.l, F2{a2.x, a2.y}, yf[j + 64]);
            f2_acc<false>(acc2.h, acc2.l, F2{a3.x, a3.y}, yf[j + 96]);
          }
          for (; j < j1; j += 32) {
            const float2 a = row[j];
            f2_acc<false>(acc.h, acc.l, F2{a.x, a.y}, yf[j]);
          }
          acc = warp_sum_f2(f2_add(acc, acc2));
          if (lane == 0) yf[b0 + i] = f2_add(yf[b0 + i], F2{-acc.h, -acc.l});
        }
      }
      __syncthreads();
      const float2* X = q.Lif + (size_t)blk * (kTile * kTile);
      for (int i = warp; i < nb; i += nw) {
        F2 acc = {0.f, 0.f};
        if (!upper) {
          for (int l = lane; l <= i; l += 32) {
            const float2 a = X[i * kTile + l];
            f2_acc<false>(acc.h, acc.l, F2{a.x, a.y}, yf[b0 + l]);
          }
        } else {
          for (int l = i + lane; l < nb; l += 32) {
            const float2 a = X[l * kTile + i];
            f2_acc<false>(acc.h, acc.l, F2{a.x, a.y}, yf[b0 + l]);
          }
        }
        acc = warp_sum_f2(acc);
        if (lane == 0) tmpf[i] = acc;
      }
      __syncthreads();
      if (threadIdx.x < nb) yf[b0 + threadIdx.x] = tmpf[threadIdx.x];
      __syncthreads();
    }
  }
  for (int j = threadIdx.x; j < N; j += blockDim.x) yd[j] = from_f2(yf[j], ez - 2 * te);
  __syncthreads();
}

// GROW / RESTART: r~ = H_S^{-1} r.   ITER: r~+ = H_S^{-1} r+   (mixed form,
// double-float on the float32 pipe; the same forms as b_apply_kernel).
__global__ void __launch_bounds__(512) b_apply_mixed_kernel(BCtl c, const BDesc* __restrict__ D, const BState* S) {
  __shared__ double yd[kMaxD];
  __shared__ F2 yf[kMaxD];
  __shared__ F2 tmpf[kTile];
  __shared__ int s_e;
  tk_start(c, TK_APPLY);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    const int ph = S[p].phase;
    if (ph != PH_GROW && ph != PH_ITER && ph != PH_RESTART) continue;
    const BState s = S[p];
    const BDesc& q = D[p];
    const int d = q.d;
    const bool restart = s.phase != PH_ITER;
    const double* z = q.vec + (size_t)(restart ? V_R : V_RP) * d;
    double* out = q.vec + (size_t)(restart ? V_RT : V_RTP) * d;
    if (s.form == 0) {
      for (int j = threadIdx.x; j < d; j += blockDim.x) yd[j] = z[j];
      __syncthreads();
      df_chol_solve(q, d, s.sexp, yd, yf, tmpf, &s_e);
      for (int j = threadIdx.x; j < d; j += blockDim.x) out[j] = yd[j];
    } else {
      // u = (nu^2 Lambda)^{-1} z;  t = Y_s u;  w = K^{-1} t;  out = u - (nu^2 Lambda)^{-1} Y_s^T w
      const int m = (int)s.m;
      const double ism = 1.0 / sqrt((double)m);
      const double* isc = q.vec + (size_t)V_ISC * d;
      double* u = q.vec + (size_t)V_U * d;
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        const double v = z[j] * isc[j];
        u[j] = v;
        yd[j] = v;
      }
      __syncthreads();
      const int eu = block_max_exp(yd, d, &s_e);
      for (int j = threadIdx.x; j < d; j += blockDim.x) yf[j] = to_f2(yd[j], -eu);
      __syncthreads();
      for (int r = warp; r < m; r += nw) {
        const float* row = q.Bf + (int64_t)q.perm[r] * d;
        F2 acc = {0.f, 0.f};
        for (int j = lane; j < d; j += 32) f2_acc<false>(acc.h, acc.l, F2{row[j], 0.f}, yf[j]);
        acc = warp_sum_f2(acc);
        if (lane == 0) yd[r] = from_f2(acc, eu) * ism;
      }
      __syncthreads();
      df_chol_solve(q, m, s.sexp, yd, yf, tmpf, &s_e);
      const int ew = block_max_exp(yd, m, &s_e);
      for (int r = threadIdx.x; r < m; r += blockDim.x) yf[r] = to_f2(yd[r], -ew);
      __syncthreads();
      for (int j = threadIdx.x; j < d; j += blockDim.x) {
        F2 acc = {0.f, 0.f};
        for (int r = 0; r < m; ++r) f2_acc<false>(acc.h, acc.l, F2{q.Bf[(int64_t)q.perm[r] * d + j], 0.f}, yf[r]);
        out[j] = u[j] - from_f2(acc, ew) * ism * isc[j];
      }
    }
    __syncthreads();
  }
  tk_stop(c, TK_APPLY);
}

// GROW: restart p = r~, delta~_t = delta~_I = r^T r~.
// ITER: delta~+ = r+^T r~+, the improvement test of Algorithm 2, the update.
// INIT: on to the first sketch.
// Mixed form, end of an inner solve: x_o += dx, then the next refinement step
// (or NO_CONVERGENCE after max_outer of them).
SKS_DEV void finish_inner(const BCtl& c, const BDesc& q, BState* S, int p) {
  const double* xi = q.vec + (size_t)V_XI * q.d;
  for (int j = threadIdx.x; j < q.d; j += blockDim.x) q.x[j] += xi[j];
  if (threadIdx.x == 0) {
    BState& s = S[p];
    s.outer += 1;
    if (s.outer >= c.max_outer) {
      s.status = SKS_ERR_NO_CONVERGENCE;
      s.phase = PH_FAIL;
    } else {
      s.phase = PH_INIT;
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) b_step2_kernel(BCtl c, const BDesc* __restrict__ D, BState* S) {
  __shared__ double scratch[32];
  __shared__ int s_accept, s_phase, s_inner_done;
  for (int p = blockIdx.x; p < c.P; p += gridDim.x) {
    // thread 0 changes the phase below: every thread reads it first
    __syncthreads();
    if (threadIdx.x == 0) s_phase = S[p].phase;
    __syncthreads();
    const int phase = s_phase;
    if (phase == PH_INIT) {
      if (threadIdx.x == 0) {
        // mixed form: a sketch exists after the first refinement step
        S[p].phase = (c.mixed && S[p].m > 0) ? PH_RESTART : PH_GROW;
        S[p].fresh = c.mixed;
      }
      continue;
    }
    if (phase != PH_GROW && phase != PH_ITER && phase != PH_RESTART) continue;
    const BDesc& q = D[p];
    const int d = q.d;
    double* r = q.vec + (size_t)V_R * d;
    double* rt = q.vec + (size_t)V_RT * d;
    double* pv = q.vec + (size_t)V_P * d;
    if (phase != PH_ITER) {
      const double dt = block_dot(d, r, rt, scratch);
      for (int j = threadIdx.x; j < d; j += blockDim.x) pv[j] = rt[j];
      if (threadIdx.x == 0) {
        BState& s = S[p];
        s.dt = dt;
        s.dI = dt;
        s_inner_done = 0;
        if (!isfinite(dt)) {
          s.status = SKS_ERR_NUMERIC;
          s.phase = PH_FAIL;
        } else if (!c.mixed) {
          s.phase = dt <= 0.0 ? PH_DONE : PH_ITER;
        } else if (s.fresh) {
          // first restart of an inner solve: delta~ at x_o estimates its error
          s.fresh = 0;
          s.d0 = dt;
          s.phase = (dt <= 0.0 || dt <= c.tol2 * s.btx) ? PH_DONE : PH_ITER;
        } else if (dt <= 0.0) {
          s_inner_done = 1;
        } else {
          s.phase = PH_ITER;
        }
      }
      __syncthreads();
      if (s_inner_done) finish_inner(c, q, S, p);
      continue;
    }
    const double* rp = q.vec + (size_t)V_RP * d;
    const double* rtp = q.vec + (size_t)V_RTP * d;
    const double* xp = q.vec + (size_t)V_XP * d;
    const double dp = block_dot(d, rp, rtp, scratch);
    if (threadIdx.x == 0) {
      BState& s = S[p];
      const double thr = c.c * pow(c.phi, (double)(s.t + 1 - s.I));
      const double ratio = dp / s.dI;
      const int reject = (ratio > thr) && (s.m < q.m_max);
      s_accept = 1;
      if (!isfinite(dp)) {
        s.status = SKS_ERR_NUMERIC;
        s.phase = PH_FAIL;
        s_accept = 0;
      } else if (reject) {
        s.I = s.t;
        s.rejections += 1;
        s.phase = PH_GROW;
        s_accept = 0;
      }
    }
    __syncthreads();
    if (!s_accept) continue;
    const double beta = dp / S[p].dt;
    double* xd = c.mixed ? q.vec + (size_t)V_XI * d : q.x;
    for (int j = threadIdx.x; j < d; j += blockDim.x) {
      pv[j] = rtp[j] + beta * pv[j];
      xd[j] = xp[j];
      r[j] = rp[j];
      rt[j] = rtp[j];
    }
    __syncthreads();
    if (c.mixed) {
      // inner solve: relative decrement inner_tol^2 against its first restart
      if (threadIdx.x == 0) {
        BState& s = S[p];
        s.dt = dp;
        s.t += 1;
        s.t_all += 1;
        s_inner_done = (dp <= 0.0 || dp <= c.inner2 * s.d0) ? 1 : 0;
        if (!s_inner_done && s.t_all >= c.max_iter) {
          s.status = SKS_ERR_NO_CONVERGENCE;
          s.phase = PH_FAIL;
        }
      }
      __syncthreads();
      if (s_inner_done) finish_inner(c, q, S, p);
      continue;
    }
    const double btx = block_dot(d, q.b, q.x, scratch);
    if (threadIdx.x == 0) {
      BState& s = S[p];
      s.dt = dp;
      s.t += 1;
      s.t_all = s.t;
      s.btx = btx;
      if (dp <= 0.0 || dp <= c.tol2 * btx) {
        s.phase = PH_DONE;
      } else if (s.t >= c.max_iter) {
        s.status = SKS_ERR_NO_CONVERGENCE;
        s.phase = PH_FAIL;
      }
    }
    __syncthreads();
  }
}

__global__ void b_count_kernel(BCtl c, const BState* S) {
  __shared__ int scratch[32];
  int a = 0;
  for (int p = threadIdx.x; p < c.P; p += blockDim.x) a += S[p].phase < PH_DONE ? 1 : 0;
  a = block_sum(a, scratch);
  if (threadIdx.x == 0) {
    *c.active = a;
    *c.round_kmax = 0;
    const long long r = ++*c.rounds;
    if (c.use_cond) cudaGraphSetConditional(c.cond, (a > 0 && r < c.max_rounds) ? 1u : 0u);
    if (c.tk) {
      c.tk[3 * TK_ROUND + 1] = global_ns();
      for (int i = 0; i < kTimers; ++i) {
        unsigned long long* t = c.tk + 3 * i;
        if (t[1] > t[0]) t[2] += t[1] - t[0];
        t[0] = ~0ull;
        t[1] = 0ull;
      }
    }
  }
}

// ------------------------------------------------------------------ setup kernels

// Per-solve counters: A-pass and Gram timing windows, flop sums, rounds.
__global__ void b_reset_kernel(BCtl c) {
  if (threadIdx.x != 0) return;
  for (int i = 0; i < kTimers; ++i) {
    c.tk[3 * i] = ~0ull;
    c.tk[3 * i + 1] = 0ull;
    c.tk[3 * i + 2] = 0ull;
  }
  *c.apass_flops = 0.0;
  *c.gram_flops = 0.0;
  *c.round_kmax = 0;
  *c.rounds = 0;
}

__global__ void b_check_kernel(const BDesc* __restrict__ D, int P, DevStatus* st) {
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    const BDesc& q = D[p];
    for (int j = threadIdx.x; j < q.d; j += blockDim.x)
      if (!(q.lam[j] >= 1.0 && isfinite(q.lam[j]))) raise_status(st, SKS_ERR_INVALID_ARG, 1, ((long long)p << 32) | j);
  }
}

// mixed form: 1 / lambda rounded to float32 (Woodbury Gram)
__global__ void b_prep_mixed_kernel(const BDesc* __restrict__ D, int P) {
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    const BDesc& q = D[p];
    for (int j = threadIdx.x; j < q.d; j += blockDim.x) {
      q.ilam[j] = (float)(1.0 / q.lam[j]);
      q.vec[(size_t)V_ISC * q.d + j] = 1.0 / (q.nu2 * q.lam[j]);
    }
  }
}

// x_0 = 0 (the usual start): the first r = b - H x_0 needs no pass over A.
__global__ void b_xzero_kernel(const BDesc* __restrict__ D, BState* S, int P) {
  __shared__ int any;
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const BDesc& q = D[p];
    for (int j = threadIdx.x; j < q.d; j += blockDim.x)
      if (q.x[j] != 0.0) any = 1;
    __syncthreads();
    if (threadIdx.x == 0) S[p].xzero = any ? 0 : 1;
    __syncthreads();
  }
}

__global__ void b_init_kernel(BState* S, int P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  BState s = {};
  s.phase = PH_INIT;
  s.status = SKS_OK;
  S[p] = s;
}

// ------------------------------------------------------------------ host side

struct Layout {
  BDesc* D = nullptr;
  BState* S = nullptr;
  int *pre_tri = nullptr, *pre_T = nullptr, *pre_ap = nullptr, *pre_red = nullptr, *active = nullptr;
  int* round_kmax = nullptr;
  unsigned long long* tk = nullptr;
  double* apass_flops = nullptr;
  double* gram_flops = nullptr;
  long long* rounds = nullptr;
  DevStatus* st = nullptr;
  std::vector<BDesc> host;
  size_t used = 0;
};

constexpr int kMinRowsPerUnit = 32;

int64_t m_max_of(const sks_problem& p, const sks_opts* o) {
  const int64_t n_pad = (int64_t)1 << ilog2_ceil(std::max<int64_t>(p.n, 1));
  return o->m_max <= 0 ? n_pad : std::min<int64_t>(o->m_max, n_pad);
}

sks_status check_batch(const sks_problem* probs, int count, const sks_opts* o) {
  if (!probs || count < 1) return fail(SKS_ERR_INVALID_ARG, "batch: need count >= 1 problems");
  if (!o) return fail(SKS_ERR_INVALID_ARG, "opts is NULL");
  if (!(o->rho > 0.0 && o->rho < 1.0)) return fail(SKS_ERR_INVALID_ARG, "rho must be in (0, 1)");
  if (o->m_init < 1) return fail(SKS_ERR_INVALID_ARG, "m_init must be >= 1");
  if (!(o->tol > 0.0)) return fail(SKS_ERR_INVALID_ARG, "tol must be > 0");
  if (o->stop_rule != SKS_STOP_ESTIMATE)
    return fail(SKS_ERR_UNSUPPORTED, "the batch stops by the estimate rule only");
  if (o->kind != SKS_SRHT) return fail(SKS_ERR_UNSUPPORTED, "batch: only the SRHT embedding is implemented");
  const bool mixed = o->precision == SKS_MIXED_REFINED;
  if (mixed && (o->max_outer < 1 || !(o->inner_tol > 0.0 && o->inner_tol < 1.0)))
    return fail(SKS_ERR_INVALID_ARG, "mixed form needs max_outer >= 1 and inner_tol in (0, 1)");
  for (int i = 0; i < count; ++i) {
    const sks_problem& p = probs[i];
    const sks_status v = validate_problem(&p);
    if (v != SKS_OK) return fail(v, "batch problem " + std::to_string(i) + ": " + last_error_cstr());
    if (!mixed && p.dtype != SKS_F64)
      return fail(SKS_ERR_INVALID_ARG, "batch problem " + std::to_string(i) + ": the plain form needs float64 A");
    if (mixed && p.dtype != SKS_F32)
      return fail(SKS_ERR_INVALID_ARG, "batch problem " + std::to_string(i) + ": the mixed form needs float32 A");
    if (p.k != 1) return fail(SKS_ERR_UNSUPPORTED, "batch problem " + std::to_string(i) + ": one right-hand side");
    if (p.n < 1) return fail(SKS_ERR_UNSUPPORTED, "batch problem " + std::to_string(i) + ": n >= 1");
    if (p.d > kMaxD) return fail(SKS_ERR_UNSUPPORTED, "batch problem " + std::to_string(i) + ": d <= 1024");
  }
  return SKS_OK;
}

// Carves the workspace (ws == nullptr: sizes only).
sks_status batch_layout(const sks_problem* probs, int P, const sks_opts* o, void* ws, size_t ws_bytes, Layout* L) {
  Carver c(ws, ws_bytes);
  L->D = c.take<BDesc>(P);
  L->S = c.take<BState>(P);
  L->pre_tri = c.take<int>(P + 1);
  L->pre_T = c.take<int>(P + 1);
  L->pre_ap = c.take<int>(P + 1);
  L->pre_red = c.take<int>(P + 1);
  L->active = c.take<int>(1);
  L->round_kmax = c.take<int>(1);
  L->tk = c.take<unsigned long long>(3 * kTimers);
  L->apass_flops = c.take<double>(1);
  L->gram_flops = c.take<double>(1);
  L->rounds = c.take<long long>(1);
  L->st = c.take<DevStatus>(1);
  L->host.assign(P, BDesc{});
  for (int i = 0; i < P; ++i) {
    const sks_problem& p = probs[i];
    BDesc& q = L->host[i];
    const bool mixed = o->precision == SKS_MIXED_REFINED;
    q.A = mixed ? nullptr : (const double*)p.A;
    q.Af = mixed ? (const float*)p.A : nullptr;
    q.lda = p.lda;
    q.n = p.n;
    q.d = (int)p.d;
    q.bits = ilog2_ceil(std::max<int64_t>(p.n, 1));
    q.b = (const double*)p.b;
    q.lam = p.lambda_diag;
    q.nu2 = p.nu * p.nu;
    q.m_max = m_max_of(p, o);
    q.m_init = o->m_init;
    const int64_t n_pad = (int64_t)1 << q.bits;
    if (mixed) {
      q.B = nullptr;
      q.Bf = c.take<float>((size_t)n_pad * q.d);
      q.ilam = c.take<float>((size_t)q.d);
      q.Lf = c.take<float2>((size_t)q.d * q.d);
      q.Lif = c.take<float2>((size_t)((q.d + kTile - 1) / kTile) * kTile * kTile);
    } else {
      q.Lf = nullptr;
      q.Lif = nullptr;
      q.B = c.take<double>((size_t)n_pad * q.d);
      q.Bf = nullptr;
      q.ilam = nullptr;
    }
    q.perm = c.take<uint32_t>((size_t)q.m_max);
    q.M = c.take<double>((size_t)q.d * q.d);
    q.vec = c.take<double>((size_t)kNumVec * q.d);
    q.part = c.take<double>((size_t)((p.n + kMinRowsPerUnit - 1) / kMinRowsPerUnit) * q.d);
    const int T = (q.d + kTile - 1) / kTile;
    q.ntri = T * (T + 1) / 2;
    // slices only exist when m can reach 2 kGramSliceMin rows
    q.gpart = c.take<double>((size_t)kGramSplit * q.ntri * kTile * kTile);
    q.G = c.take<double>((size_t)q.d * q.d);
  }
  L->used = c.used + 256;
  if (ws && !c.ok()) return fail(SKS_ERR_WORKSPACE, "batch: workspace too small");
  return SKS_OK;
}

std::vector<int> prefix(const std::vector<BDesc>& h, int (*units)(const BDesc&, int), int arg) {
  std::vector<int> pre(h.size() + 1, 0);
  for (size_t i = 0; i < h.size(); ++i) pre[i + 1] = pre[i] + units(h[i], arg);
  return pre;
}
int units_T(const BDesc& q, int) { return (q.d + kTile - 1) / kTile; }
int units_tri(const BDesc& q, int) {
  const int T = units_T(q, 0);
  return T * (T + 1) / 2;
}
int units_ap(const BDesc& q, int rows) { return (int)((q.n + rows - 1) / rows); }
int units_red(const BDesc& q, int) { return (q.d + 255) / 256; }

constexpr size_t kTrsmSmem = 2 * kTile * (kTile + 1) * sizeof(double);

struct Round {
  BCtl ctl;
  const BDesc* D;
  BState* S;
  int P, kmax, tot_tri, tot_T, tot_ap, tot_red;
  int g_tile, g_gram, g_trsm, g_ap, g_prob;
  size_t ap_smem;
  bool mixed;
  int g_apd;          // mixed form: grid of the double-float (residual) A-pass
};

// Enqueues one round on `stream`; returns the number of kernels.
int enqueue_round(const Round& R, cudaStream_t stream) {
  int n = 0;
  const int pb = (R.P + 127) / 128;
  b_begin_kernel<<<pb, 128, 0, stream>>>(R.ctl, R.D, R.S);
  ++n;
  b_perm_kernel<<<R.g_prob, 256, 0, stream>>>(R.ctl, R.D, R.S);
  ++n;
  if (R.mixed) b_gram_mixed_kernel<<<R.g_gram, 256, 0, stream>>>(R.ctl, R.D, R.S, R.tot_tri * kGramSplit);
  else b_gram_kernel<<<R.g_gram, 256, 0, stream>>>(R.ctl, R.D, R.S, R.tot_tri * kGramSplit);
  b_gram_reduce_kernel<<<R.g_tile, 256, 0, stream>>>(R.ctl, R.D, R.S, R.tot_tri);
  n += 2;
  for (int k = 0; k < R.kmax; ++k) {
    if (R.mixed) b_potrf_df_kernel<<<R.g_prob, kPotThreads, 0, stream>>>(R.ctl, R.D, R.S, k);
    else b_potrf_kernel<<<R.g_prob, 256, 0, stream>>>(R.ctl, R.D, R.S, k);
    ++n;
    if (k + 1 < R.kmax) {
      if (R.mixed) {
        b_trsm_df_kernel<<<R.g_trsm, 256, 0, stream>>>(R.ctl, R.D, R.S, k, R.tot_T);
        b_update_df_kernel<<<R.g_tile, 256, 0, stream>>>(R.ctl, R.D, R.S, k, R.tot_tri);
      } else {
        b_trsm_kernel<<<R.g_trsm, 64, kTrsmSmem, stream>>>(R.ctl, R.D, R.S, k, R.tot_T);
        b_update_kernel<<<R.g_tile, 256, 0, stream>>>(R.ctl, R.D, R.S, k, R.tot_tri);
      }
      n += 2;
    }
  }
  if (R.mixed) {
    b_apass_mixed_kernel<true><<<R.g_apd, kApThreads, apass_mixed_smem(true), stream>>>(R.ctl, R.D, R.S, R.tot_ap, 0);
    b_apass_mixed_kernel<false><<<R.g_ap, kApThreads, apass_mixed_smem(false), stream>>>(R.ctl, R.D, R.S, R.tot_ap,
                                                                                        0);
    ++n;
  } else {
    b_apass_kernel<<<R.g_ap, kApThreads, R.ap_smem, stream>>>(R.ctl, R.D, R.S, R.tot_ap);
  }
  b_reduce_kernel<<<R.g_tile, 256, 0, stream>>>(R.ctl, R.D, R.S, R.tot_red);
  b_step1_kernel<<<R.g_prob, 256, 0, stream>>>(R.ctl, R.D, R.S);
  if (R.mixed) b_apply_mixed_kernel<<<R.g_prob, 512, 0, stream>>>(R.ctl, R.D, R.S);
  else b_apply_kernel<<<R.g_prob, 512, 0, stream>>>(R.ctl, R.D, R.S);
  b_step2_kernel<<<R.g_prob, 256, 0, stream>>>(R.ctl, R.D, R.S);
  b_count_kernel<<<1, 256, 0, stream>>>(R.ctl, R.S);
  n += 6;
  return n;
}

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  sks_status init() {
    SKS_CUDA_TRY(cudaEventCreate(&a));
    SKS_CUDA_TRY(cudaEventCreate(&b));
    return SKS_OK;
  }
  sks_status ms(float* out) {
    SKS_CUDA_TRY(cudaEventSynchronize(b));
    SKS_CUDA_TRY(cudaEventElapsedTime(out, a, b));
    return SKS_OK;
  }
};


sks_status upload_prefix(int* dst, const std::vector<int>& pre, cudaStream_t stream) {
  SKS_CUDA_TRY(cudaMemcpyAsync(dst, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice, stream));
  return SKS_OK;
}

}  // namespace
}  // namespace sks

// A batch plan: the workspace layout, the tuned A-pass unit height and one
// instantiated graph
//     reset counters -> states INIT -> H E A_pad of every problem -> WHILE (some problem unfinished) { round }
// so that a solve is a descriptor upload and ONE graph launch: the rounds
// repeat on the device (the round's last kernel sets the loop condition)
// with no host round trip until every problem has stopped.
struct sks_batch {
  int P = 0;
  sks_opts opts;
  sks::Layout L;
  sks::Round R;
  int chosen = 0, per_round = 0;
  float ms_plan = 0.f, ms_tune = 0.f;
  cudaGraph_t g = nullptr, g_setup = nullptr;
  cudaGraphExec_t e = nullptr;
  cudaStream_t cs = nullptr;
  ~sks_batch() {
    if (e) cudaGraphExecDestroy(e);
    if (g) cudaGraphDestroy(g);
    if (g_setup) cudaGraphDestroy(g_setup);
    if (cs) cudaStreamDestroy(cs);
  }
};

namespace sks {

sks_status batch_workspace_size(const sks_problem* probs, int count, const sks_opts* o, size_t* bytes) {
  if (!bytes) return fail(SKS_ERR_INVALID_ARG, "bytes is NULL");
  SKS_TRY(check_batch(probs, count, o));
  Layout L;
  SKS_TRY(batch_layout(probs, count, o, nullptr, 0, &L));
  *bytes = L.used;
  return SKS_OK;
}

// The solve's setup: counters reset, every problem INIT, 1 / lambda (mixed
// form) and H E A_pad of every problem.
sks_status enqueue_setup(const sks_batch* B, const BCtl& c, cudaStream_t stream) {
  const Layout& L = B->L;
  const int P = B->P;
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  b_reset_kernel<<<1, 32, 0, stream>>>(c);
  b_init_kernel<<<(P + 127) / 128, 128, 0, stream>>>(L.S, P);
  b_xzero_kernel<<<std::min(P, 4 * sms), 256, 0, stream>>>(L.D, L.S, P);
  if (B->R.mixed) b_prep_mixed_kernel<<<std::min(P, 4 * sms), 256, 0, stream>>>(L.D, P);
  for (int i = 0; i < P; ++i) {
    const BDesc& q = L.host[i];
    const sks_status sr = B->R.mixed ? srht_form<float>(stream, q.Af, q.lda, q.n, q.d, q.Bf, q.d, B->opts.seed)
                                     : srht_form<double>(stream, q.A, q.lda, q.n, q.d, (double*)q.B, q.d, B->opts.seed);
    if (sr != SKS_OK) return sr;
  }
  return SKS_OK;
}

sks_status batch_create(sks_batch** out, const sks_problem* probs, int P, const sks_opts* o, int rows_per_unit,
                        void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (!out) return fail(SKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  SKS_TRY(check_batch(probs, P, o));
  if (rows_per_unit != 0 && (rows_per_unit < kMinRowsPerUnit || rows_per_unit > 65536))
    return fail(SKS_ERR_INVALID_ARG, "rows_per_unit must be 0 (autotune) or in [32, 65536]");
  if (!ws) return fail(SKS_ERR_INVALID_ARG, "workspace is NULL");
  sks_batch* B = new (std::nothrow) sks_batch;
  if (!B) return fail(SKS_ERR_INVALID_ARG, "out of host memory");
  struct Guard {
    sks_batch*& b;
    ~Guard() { delete b; }
  } guard{B};
  B->P = P;
  B->opts = *o;
  Layout& L = B->L;
  SKS_TRY(batch_layout(probs, P, o, ws, ws_bytes, &L));
  const DeviceInfo& di = device_info();
  const int sms = di.sms > 0 ? di.sms : 152;
  EventPair ev_plan, ev_tune;
  SKS_TRY(ev_plan.init());
  SKS_TRY(ev_tune.init());
  SKS_CUDA_TRY(cudaEventRecord(ev_plan.a, stream));
  // descriptors with a zeroed scratch vector standing in for x until a solve gives the real one
  std::vector<BDesc> tmp = L.host;
  for (BDesc& q : tmp) q.x = q.vec + (size_t)V_W * q.d;
  for (const BDesc& q : tmp) SKS_CUDA_TRY(cudaMemsetAsync(q.vec, 0, (size_t)kNumVec * q.d * sizeof(double), stream));
  SKS_CUDA_TRY(cudaMemsetAsync(L.st, 0, sizeof(DevStatus), stream));
  SKS_CUDA_TRY(cudaMemcpyAsync(L.D, tmp.data(), P * sizeof(BDesc), cudaMemcpyHostToDevice, stream));
  const std::vector<int> pre_tri = prefix(L.host, units_tri, 0), pre_T = prefix(L.host, units_T, 0),
                         pre_red = prefix(L.host, units_red, 0);
  SKS_TRY(upload_prefix(L.pre_tri, pre_tri, stream));
  SKS_TRY(upload_prefix(L.pre_T, pre_T, stream));
  SKS_TRY(upload_prefix(L.pre_red, pre_red, stream));
  b_check_kernel<<<std::min(P, 4 * sms), 256, 0, stream>>>(L.D, P, L.st);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  SKS_TRY(read_status(L.st, stream, "batch input check"));
  b_init_kernel<<<(P + 127) / 128, 128, 0, stream>>>(L.S, P);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());

  // ---- round description
  Round& R = B->R;
  std::memset(&R, 0, sizeof(R));
  R.P = P;
  R.D = L.D;
  R.S = L.S;
  BCtl& c = R.ctl;
  c.P = P;
  c.max_iter = o->max_iter > 0 ? o->max_iter : 1000000;
  const double rho = o->rho;
  c.phi = (1.0 - std::sqrt(1.0 - rho)) / (1.0 + std::sqrt(1.0 - rho));
  c.c = 4.0 * (1.0 + std::sqrt(rho)) / (1.0 - std::sqrt(rho));
  c.tol2 = (o->tol / 2.0) * (o->tol / 2.0);
  c.mixed = o->precision == SKS_MIXED_REFINED ? 1 : 0;
  c.max_outer = c.mixed ? o->max_outer : 1;
  c.inner2 = c.mixed ? o->inner_tol * o->inner_tol : 0.0;
  c.key = make_key(o->seed);
  c.pre_tri = L.pre_tri;
  c.pre_T = L.pre_T;
  c.pre_ap = L.pre_ap;
  c.pre_red = L.pre_red;
  c.active = L.active;
  c.round_kmax = L.round_kmax;
  c.tk = L.tk;
  c.apass_flops = L.apass_flops;
  c.gram_flops = L.gram_flops;
  c.rounds = L.rounds;
  int dmax = 0;
  int64_t mmax_all = 1;
  for (const BDesc& q : L.host) {
    dmax = std::max(dmax, q.d);
    mmax_all = std::max(mmax_all, q.m_max);
  }
  // every doubling and every refinement step (residual, restart) costs a round
  c.max_rounds = 4 + 2 * (ilog2_ceil(mmax_all) + 2) + c.max_iter + 3 * c.max_outer;
  R.kmax = (dmax + kTile - 1) / kTile;
  R.tot_tri = pre_tri[P];
  R.tot_T = pre_T[P];
  R.tot_red = pre_red[P];
  R.g_prob = std::min(P, 8 * sms);
  R.g_tile = std::max(1, std::min(R.tot_tri, 4 * sms));
  R.g_gram = std::max(1, std::min(R.tot_tri * kGramSplit, 4 * sms));
  R.g_trsm = std::max(1, std::min(R.tot_T, 8 * sms));
  R.mixed = c.mixed != 0;
  R.ap_smem = R.mixed ? apass_mixed_smem(false) : (size_t)(1 + kApWarps) * kMaxD * sizeof(double);
  SKS_CUDA_TRY(cudaFuncSetAttribute(b_trsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrsmSmem));
  int ap_occ = 1, apd_occ = 1;
  if (R.mixed) {
    SKS_CUDA_TRY(cudaFuncSetAttribute(b_apass_mixed_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)apass_mixed_smem(false)));
    SKS_CUDA_TRY(cudaFuncSetAttribute(b_apass_mixed_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)apass_mixed_smem(true)));
    SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ap_occ, b_apass_mixed_kernel<false>, kApThreads,
                                                               apass_mixed_smem(false)));
    SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&apd_occ, b_apass_mixed_kernel<true>, kApThreads,
                                                               apass_mixed_smem(true)));
  } else {
    SKS_CUDA_TRY(cudaFuncSetAttribute(b_apass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)R.ap_smem));
    SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ap_occ, b_apass_kernel, kApThreads, R.ap_smem));
  }
  const int ap_grid_max = sms * std::max(1, ap_occ);
  const int apd_grid_max = sms * std::max(1, apd_occ);

  // ---- autotune the A-pass unit height on this batch (all problems in INIT)
  SKS_CUDA_TRY(cudaEventRecord(ev_tune.a, stream));
  int chosen = rows_per_unit;
  if (chosen == 0) {
    const int cands[] = {32, 64, 128, 256, 512};
    float best = 1e30f;
    EventPair e;
    SKS_TRY(e.init());
    for (int rows : cands) {
      const std::vector<int> pa = prefix(L.host, units_ap, rows);
      SKS_TRY(upload_prefix(L.pre_ap, pa, stream));
      BCtl ct = c;
      ct.rows_per_unit = rows;
      ct.tk = nullptr;
      const int g = std::max(1, std::min(pa[P], ap_grid_max));
      // the mixed form times its float32 inner pass (every unit, v = 0)
      for (int rep = 0; rep < 4; ++rep) {
        if (rep == 1) SKS_CUDA_TRY(cudaEventRecord(e.a, stream));  // after one warm launch
        if (R.mixed) b_apass_mixed_kernel<false><<<g, kApThreads, R.ap_smem, stream>>>(ct, L.D, L.S, pa[P], 1);
        else b_apass_kernel<<<g, kApThreads, R.ap_smem, stream>>>(ct, L.D, L.S, pa[P]);
      }
      SKS_CUDA_TRY(cudaEventRecord(e.b, stream));
      note_launch(4);
      SKS_CUDA_TRY(cudaGetLastError());
      float ms = 0.f;
      SKS_TRY(e.ms(&ms));
      if (ms < best) {
        best = ms;
        chosen = rows;
      }
    }
  }
  const std::vector<int> pre_ap = prefix(L.host, units_ap, chosen);
  SKS_TRY(upload_prefix(L.pre_ap, pre_ap, stream));
  c.rows_per_unit = chosen;
  R.tot_ap = pre_ap[P];
  R.g_ap = std::max(1, std::min(R.tot_ap, ap_grid_max));
  R.g_apd = std::max(1, std::min(R.tot_ap, apd_grid_max));
  B->chosen = chosen;
  SKS_CUDA_TRY(cudaEventRecord(ev_tune.b, stream));

  // ---- the graph: setup child graph, then the while loop around one round
  SKS_CUDA_TRY(cudaStreamCreateWithFlags(&B->cs, cudaStreamNonBlocking));
  SKS_CUDA_TRY(cudaGraphCreate(&B->g, 0));
  SKS_CUDA_TRY(cudaGraphCreate(&B->g_setup, 0));
  SKS_CUDA_TRY(cudaStreamBeginCaptureToGraph(B->cs, B->g_setup, nullptr, nullptr, 0,
                                             cudaStreamCaptureModeThreadLocal));
  {
    const sks_status sr = enqueue_setup(B, c, B->cs);
    cudaGraph_t got = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(B->cs, &got);
    SKS_TRY(sr);
    SKS_CUDA_TRY(ce);
  }
  cudaGraphNode_t n_setup = nullptr, n_while = nullptr;
  SKS_CUDA_TRY(cudaGraphAddChildGraphNode(&n_setup, B->g, nullptr, 0, B->g_setup));
  SKS_CUDA_TRY(cudaGraphConditionalHandleCreate(&c.cond, B->g, 1u, cudaGraphCondAssignDefault));
  cudaGraphNodeParams np = {cudaGraphNodeTypeConditional};
  np.conditional.handle = c.cond;
  c.use_cond = 1;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  SKS_CUDA_TRY(cudaGraphAddNode(&n_while, B->g, &n_setup, nullptr, 1, &np));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  SKS_CUDA_TRY(cudaStreamBeginCaptureToGraph(B->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  B->per_round = enqueue_round(R, B->cs);
  {
    cudaGraph_t got = nullptr;
    SKS_CUDA_TRY(cudaStreamEndCapture(B->cs, &got));
  }
  SKS_CUDA_TRY(cudaGetLastError());
  SKS_CUDA_TRY(cudaGraphInstantiate(&B->e, B->g, 0));
  SKS_CUDA_TRY(cudaEventRecord(ev_plan.b, stream));
  SKS_TRY(ev_plan.ms(&B->ms_plan));
  SKS_TRY(ev_tune.ms(&B->ms_tune));
  *out = B;
  B = nullptr;  // the guard keeps nothing
  return SKS_OK;
}

sks_status batch_solve(sks_batch* B, double* const* xs, sks_stats* stats, sks_batch_info* info,
                       cudaStream_t stream) {
  if (!B) return fail(SKS_ERR_INVALID_ARG, "batch plan is NULL");
  if (!xs) return fail(SKS_ERR_INVALID_ARG, "x array is NULL");
  const int P = B->P;
  for (int i = 0; i < P; ++i)
    if (!xs[i]) return fail(SKS_ERR_INVALID_ARG, "x of batch problem " + std::to_string(i) + " is NULL");
  Layout& L = B->L;
  for (int i = 0; i < P; ++i) L.host[i].x = xs[i];
  EventPair ev_solve;
  SKS_TRY(ev_solve.init());
  SKS_CUDA_TRY(cudaMemcpyAsync(L.D, L.host.data(), P * sizeof(BDesc), cudaMemcpyHostToDevice, stream));
  SKS_CUDA_TRY(cudaEventRecord(ev_solve.a, stream));
  const char* sw = std::getenv("SKS_BATCH_STEPWISE");
  if (sw && sw[0] == '1') {
    // Profiling aid: the same setup and rounds launched one by one from the
    // host (profilers do not see the kernels of a conditional graph node);
    // the active count is read after every round.
    Round Rs = B->R;
    Rs.ctl.use_cond = 0;
    SKS_TRY(enqueue_setup(B, Rs.ctl, stream));
    for (long long r = 0; r < Rs.ctl.max_rounds; ++r) {
      enqueue_round(Rs, stream);
      SKS_CUDA_TRY(cudaGetLastError());
      int act = 0;
      SKS_CUDA_TRY(cudaMemcpyAsync(&act, L.active, sizeof(int), cudaMemcpyDeviceToHost, stream));
      SKS_CUDA_TRY(cudaStreamSynchronize(stream));
      if (act == 0) break;
    }
  } else {
    SKS_CUDA_TRY(cudaGraphLaunch(B->e, stream));
  }
  note_launch(3 + 3 * P + (B->R.mixed ? 1 : 0));  // setup kernels (counted per round below)
  SKS_CUDA_TRY(cudaEventRecord(ev_solve.b, stream));

  // ---- per-problem results (the one synchronisation of the solve)
  std::vector<BState> hs(P);
  unsigned long long h_tk[3 * kTimers] = {};
  double h_flops = 0.0, h_gflops = 0.0;
  long long rounds = 0;
  SKS_CUDA_TRY(cudaMemcpyAsync(hs.data(), L.S, P * sizeof(BState), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaMemcpyAsync(h_tk, L.tk, sizeof(h_tk), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaMemcpyAsync(&h_flops, L.apass_flops, sizeof(double), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaMemcpyAsync(&h_gflops, L.gram_flops, sizeof(double), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaMemcpyAsync(&rounds, L.rounds, sizeof(long long), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaStreamSynchronize(stream));
  note_launch((int)(rounds * B->per_round));
  float ms_solve = 0.f;
  SKS_TRY(ev_solve.ms(&ms_solve));
  sks_status result = SKS_OK;
  int first_bad = -1;
  for (int i = 0; i < P; ++i) {
    BState& s = hs[i];
    if (s.phase < PH_DONE) s.status = SKS_ERR_NO_CONVERGENCE;  // ran out of rounds
    if (s.status != SKS_OK && first_bad < 0) {
      first_bad = i;
      result = (sks_status)s.status;
    }
    if (stats) {
      sks_stats& t = stats[i];
      std::memset(&t, 0, sizeof(t));
      t.iters = s.t_all;
      t.rejections = s.rejections;
      t.final_m = s.m;
      t.a_passes = s.a_passes;
      t.sketch_passes = 1;
      t.factorizations = s.factorizations;
      t.final_delta_tilde = s.dt;
      t.est_rel_err = s.btx > 0 ? std::sqrt(std::max(0.0, s.dt / s.btx)) : 0.0;
      // mixed form: refinement residuals computed (the last one met the stop rule)
      t.outer_iters = B->R.mixed ? (int64_t)s.outer + (s.phase == PH_DONE ? 1 : 0) : 1;
      t.ms_total = ms_solve;
      t.status = (sks_status)s.status;
    }
  }
  if (info) {
    info->rounds = rounds;
    info->kernels_per_round = B->per_round;
    info->rows_per_unit = B->chosen;
    info->ms_setup = B->ms_plan;
    info->ms_autotune = B->ms_tune;
    info->ms_solve = ms_solve;
    info->ms_apass = (float)((double)h_tk[3 * TK_APASS + 2] * 1e-6);
    info->apass_flops = h_flops;
    info->ms_gram = (float)((double)h_tk[3 * TK_GRAM + 2] * 1e-6);
    info->gram_flops = h_gflops;
    info->ms_factor = (float)((double)h_tk[3 * TK_FACTOR + 2] * 1e-6);
    info->ms_apply = (float)((double)h_tk[3 * TK_APPLY + 2] * 1e-6);
    info->ms_rounds = (float)((double)h_tk[3 * TK_ROUND + 2] * 1e-6);
  }
  if (result != SKS_OK) {
    const char* what = result == SKS_ERR_NO_CONVERGENCE ? "did not converge"
                       : result == SKS_ERR_NOT_PD       ? "non-positive pivot in its factorisation"
                                                        : "non-finite value";
    return fail(result, "batch problem " + std::to_string(first_bad) + " " + what +
                            " (per-problem statuses are in stats[i].status)");
  }
  return SKS_OK;
}

void batch_destroy(sks_batch* B) { delete B; }

sks_status solve_batched(const sks_problem* probs, int P, const sks_opts* o, double* const* xs, sks_stats* stats,
                         sks_batch_info* info, int rows_per_unit, void* ws, size_t ws_bytes, cudaStream_t stream) {
  if (!xs) return fail(SKS_ERR_INVALID_ARG, "x array is NULL");
  for (int i = 0; i < P && probs; ++i)
    if (!xs[i]) return fail(SKS_ERR_INVALID_ARG, "x of batch problem " + std::to_string(i) + " is NULL");
  sks_batch* B = nullptr;
  SKS_TRY(batch_create(&B, probs, P, o, rows_per_unit, ws, ws_bytes, stream));
  const sks_status r = batch_solve(B, xs, stats, info, stream);
  const std::string msg = last_error_cstr();
  batch_destroy(B);
  if (r != SKS_OK) set_last_error(msg);
  return r;
}

}  // namespace sks
