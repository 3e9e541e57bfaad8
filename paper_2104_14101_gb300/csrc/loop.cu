// loop.cu -- the device-resident iteration of Algorithm 2 (adaptive PCG) and
// of Algorithm 1 with the IHS step (Theorem 3.2): ONE cooperative launch runs
// the iterations between two re-sketches, and every step is fused around the
// pass over A (Section 4.1.2: the O(nd) pass dominates an iteration; the
// preconditioner apply is O(min{m,d} d), the vector updates O(d)).
//
// The grid is the A-pass grid (apass_core.cuh): per CTA one producer warp
// that streams the CTA's row tiles of A into a ring of shared-memory stages
// pass after pass -- A does not change between iterations, so the next pass's
// first tiles are already in flight while the current step finishes -- and
// 8 consumer warps.  One PCG iteration, for K right-hand sides in lockstep:
//   1  A-pass on p (every CTA: partial sums of A^T A p over its tiles)
//   2  H p = sum of the partials + nu^2 Lambda p;  p^T H p (per-CTA partials)
//   3  alpha = delta~_t / p^T H p;  x+ = x + alpha p,  r+ = r - alpha H p
//   4  r~+ = H_S^{-1} r+: two row-parallel products with the inverse
//      Cholesky factor (X, X^T), or four in the Woodbury form (Y, X, X^T,
//      Y^T); delta~+ = r+^T r~+ (per-CTA partials)
//   5  the test of Algorithm 2: delta~+ / delta~_I > c phi^(t+1-I) rejects;
//      accepted columns shift (p = r~+ + beta p, x = x+, ...); b^T x
//   6  the stop rule.
// Phases are separated by a grid barrier (bounded wait: a barrier that does
// not complete within 2 s raises SKS_ERR_TIMEOUT and every CTA leaves).  The
// scalars of steps 3, 5 and 6 are reduced by every CTA from the per-CTA
// partials in the same fixed order, so all CTAs take the same decisions
// without another barrier.  The IHS iteration is the same with x+ = x - mu v
// (formed at the end of the previous step), g+ = H x+ - b and
// delta~+ = 1/2 g+^T H_S^{-1} g+.  The launch returns when a column fails its
// test (the host then grows the sketch, refactors H_S and relaunches with a
// restart prologue), when every column has stopped, or at max_iter: the host
// reads the 200-byte control block once per launch instead of once per
// iteration.
#include <algorithm>
#include <cstring>

#include "apass_core.cuh"
#include "loop.h"

namespace sks {

namespace {

using namespace apcore;

constexpr int kNW = kConsumers / 32;  // consumer warps per CTA

struct LoopShared {
  LoopCol col[kLoopMaxK];
  double sum[kLoopMaxK];
  double alpha[kLoopMaxK];
  double fin[kNW][32];
  double red[kNW][kLoopMaxK];
  int evi[kLoopMaxK];  // trace event of each column's current step (-1: none)
  int ok, quit, any_reject, all_done;
};

SKS_DEV unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
SKS_DEV void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier of the consumer threads of every CTA (the cooperative launch makes
// the grid co-resident).  Sense by generation; the wait is bounded.  Returns
// false in every CTA once one of them has given up.
SKS_DEV bool grid_sync(LoopHead* h, LoopShared* sh, DevStatus* st) {
  named_bar_sync(1, kConsumers);
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile int* abort_flag = &h->abort;
    if (*abort_flag) {
      ok = 0;
    } else {
      const unsigned g = ld_acquire_u32(&h->bar_gen);
      __threadfence();
      const unsigned arrived = atomicAdd(&h->bar_count, 1u) + 1u;
      if (arrived == gridDim.x) {
        atomicExch(&h->bar_count, 0u);
        __threadfence();
        st_release_u32(&h->bar_gen, g + 1u);
      } else {
        const uint64_t t0 = global_ns();
        while (ld_acquire_u32(&h->bar_gen) == g) {
          if (*abort_flag) {
            ok = 0;
            break;
          }
          if (global_ns() - t0 > kWaitLimitNs) {
            raise_status(st, SKS_ERR_TIMEOUT, 50, blockIdx.x);
            *abort_flag = 1;
            ok = 0;
            break;
          }
        }
      }
      __threadfence();
    }
    *(volatile int*)&sh->ok = ok;
  }
  named_bar_sync(1, kConsumers);
  return *(volatile int*)&sh->ok != 0;
}

// Per-CTA sums of v[c] (c < K) over the consumer threads into out[c] (global).
template <int K>
SKS_DEV void cta_sum_to(const double (&v)[K], LoopShared* sh, double* out, int stride) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < K; ++c) {
    const double s = warp_sum(v[c]);
    if (lane == 0) sh->red[warp][c] = s;
  }
  named_bar_sync(1, kConsumers);
  if (threadIdx.x < K) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kNW; ++w) s += sh->red[w][threadIdx.x];
    out[threadIdx.x * stride] = s;
  }
}

// sh->sum[c] = sum over CTAs of dots[b][c][slot] (fixed order: identical in
// every CTA).  Warp c handles column c.
template <int K>
SKS_DEV void grid_col_sums(const double* dots, int slot, LoopShared* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < K) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += dots[((size_t)b * K + warp) * kLoopDots + slot];
    s = warp_sum(s);
    if (lane == 0) sh->sum[warp] = s;
  }
  named_bar_sync(1, kConsumers);
}

// Row-parallel products over the whole grid (one warp per row):
//   y[c][i] = alpha sum_j M[i][j] u_c(j),  u_c(j) = x[c][j] (/ xdiv[j]),
// rows i < rows, j over the triangle (tri 1: j <= i, tri 2: j >= i), then
// mode 1: y = (z[c][i] - y) / (nu2 lam_i).  With w: dotv[c] += y[c][i] w[c][i].
template <int K>
SKS_DEV void gemv_phase(int kc, int rows, int cols, const double* __restrict__ M, long long ldm, int tri,
                        const double* x, long long ldx, const double* __restrict__ xdiv, double alpha, double* y,
                        long long ldy, int mode, const double* z, long long ldz, const double* __restrict__ lam,
                        double nu2, const double* w, long long ldw, double (&dotv)[K]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * kNW + warp, nw = gridDim.x * kNW;
  for (int i = gw; i < rows; i += nw) {
    int jlo = 0, jhi = cols;
    if (tri == 1) jhi = min(cols, i + 1);
    if (tri == 2) jlo = i;
    const double* row = M + (long long)i * ldm;
    double s[K];
#pragma unroll
    for (int c = 0; c < K; ++c) s[c] = 0.0;
    for (int j = jlo + lane; j < jhi; j += 32) {
      const double mv = row[j];
#pragma unroll
      for (int c = 0; c < K; ++c)
        if (c < kc) {
          const double xv = xdiv ? x[(long long)c * ldx + j] / xdiv[j] : x[(long long)c * ldx + j];
          s[c] = fma(mv, xv, s[c]);
        }
    }
#pragma unroll
    for (int c = 0; c < K; ++c) s[c] = warp_sum(s[c]);
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (c >= kc) break;
        const double v = alpha * s[c];
        const double out = mode == 0 ? v : (z[(long long)c * ldz + i] - v) / (nu2 * lam[i]);
        y[(long long)c * ldy + i] = out;
        if (w) dotv[c] = fma(out, w[(long long)c * ldw + i], dotv[c]);
      }
    }
  }
}

// v = H_S^{-1} z for the columns (precond_apply1's products, fused): dotv[c]
// receives this CTA's share of z_c^T v_c.  One grid barrier between products.
template <int K>
SKS_DEV bool apply_phase(const LoopTask& T, int d, const double* z, double* v, double (&dotv)[K], LoopShared* sh) {
  const LoopPrecond& P = T.P;
  double none[K];
#pragma unroll
  for (int c = 0; c < K; ++c) none[c] = 0.0;
  if (!P.woodbury) {
    gemv_phase<K>(T.kc, d, d, P.X, d, 1, z, d, nullptr, 1.0, T.t1, T.ld_t, 0, nullptr, 0, nullptr, 0.0, nullptr, 0,
                  none);
    if (!grid_sync(T.head, sh, T.st)) return false;
    gemv_phase<K>(T.kc, d, d, P.Xt, d, 2, T.t1, T.ld_t, nullptr, 1.0, v, d, 0, nullptr, 0, nullptr, 0.0, z, d, dotv);
    return true;
  }
  const int m = P.m;
  gemv_phase<K>(T.kc, m, d, P.Y, P.ldy, 0, z, d, T.lam, P.c, T.t1, T.ld_t, 0, nullptr, 0, nullptr, 0.0, nullptr, 0,
                none);
  if (!grid_sync(T.head, sh, T.st)) return false;
  gemv_phase<K>(T.kc, m, m, P.X, m, 1, T.t1, T.ld_t, nullptr, 1.0, T.t2, T.ld_t, 0, nullptr, 0, nullptr, 0.0, nullptr,
                0, none);
  if (!grid_sync(T.head, sh, T.st)) return false;
  gemv_phase<K>(T.kc, m, m, P.Xt, m, 2, T.t2, T.ld_t, nullptr, 1.0, T.t1, T.ld_t, 0, nullptr, 0, nullptr, 0.0,
                nullptr, 0, none);
  if (!grid_sync(T.head, sh, T.st)) return false;
  gemv_phase<K>(T.kc, d, m, P.Yt, m, 0, T.t1, T.ld_t, nullptr, P.c, v, d, 1, z, d, T.lam, T.nu2, z, d, dotv);
  return true;
}

// y[c][j] = sgn (sum over the pass's partials + nu^2 lam_j u[c][j]) + addc addv[c][j]
// for every element (c < kc, j < d), partials summed by the 8 warps of a CTA
// over 32 consecutive elements (coalesced; a fixed order); dotv[c] +=
// y[c][j] w[c][j] with w.  u: the pass vector (float32 copy in the float32 pass).
template <typename TX, int K>
SKS_DEV void reduce_phase(const LoopTask& T, int d, int nparts, const double* u, double sgn, const double* addv,
                          double addc, double* y, const double* w, double (&dotv)[K], LoopShared* sh) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const TX* part = (const TX*)T.partials;
  const long long total = (long long)K * d, used = (long long)T.kc * d;
  for (long long e0 = (long long)blockIdx.x * 32; e0 < used; e0 += (long long)gridDim.x * 32) {
    const long long e = e0 + lane;
    double s = 0.0;
    if (e < used)
      for (int p = warp; p < nparts; p += kNW) s += (double)part[(size_t)p * total + e];
    sh->fin[warp][lane] = s;
    named_bar_sync(1, kConsumers);
    if (warp == 0 && e < used) {
      double t = 0.0;
#pragma unroll
      for (int w8 = 0; w8 < kNW; ++w8) t += sh->fin[w8][lane];
      const int c = (int)(e / d), j = (int)(e - (long long)c * d);
      const double uv = sizeof(TX) == 4 ? (double)T.v32[e] : u[e];
      double v = sgn * (t + T.nu2 * T.lam[j] * uv);
      if (addv) v += addc * addv[e];
      y[e] = v;
      if (w) {
#pragma unroll
        for (int cc = 0; cc < K; ++cc)
          if (cc == c) dotv[cc] = fma(v, w[e], dotv[cc]);
      }
    }
    named_bar_sync(1, kConsumers);
  }
}

template <typename TA, typename TX, int G, int QMAX, int K>
__global__ void __launch_bounds__(kThreads,
                                  (sizeof(TA) == 4 && sizeof(TX) == 4 && QMAX <= 4 && !(K == 8 && QMAX > 1)) ? 2 : 1)
    solve_loop_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                 ApassArgs ap, LoopTask T) {
  extern __shared__ __align__(128) unsigned char smem[];
  using Core = ApassCore<TA, TX, G, QMAX, K, false>;
  Core core;
  core.carve(smem, ap);
  LoopShared* sh = (LoopShared*)align_up((size_t)(core.empty + ap.stages), 16);
  const int tid = threadIdx.x;
  if (tid == 0) {
    core.init(ap);
    sh->quit = 0;
    sh->any_reject = 0;
  }
  if (tid < K) sh->col[tid] = T.cols[tid];
  __syncthreads();
  if (tid >= kConsumers) {
    if (tid == kConsumers) core.produce(&tmap, ap, -1, &sh->quit);
    return;
  }
  // ---------------------------------------------------------------- consumers
  const int d = ap.d;
  const int gt = blockIdx.x * kConsumers + tid, GT = gridDim.x * kConsumers;
  const int nparts = gridDim.x * Core::NG;
  const bool pcg = T.method == 0;
  const bool f32v = sizeof(TX) == 4;
  double* dots = T.dots + (size_t)blockIdx.x * K * kLoopDots;
  int it = 0;
  long long apass_ns = 0, passes = 0, iters = 0;
  bool ok = true;
  auto live = [&](int c) {
    const LoopCol& s = sh->col[c];
    return c < T.kc && s.active && !s.stop && !s.numeric && s.t < T.max_iter;
  };
  auto zero = [](double (&v)[K]) {
#pragma unroll
    for (int c = 0; c < K; ++c) v[c] = 0.0;
  };
  // float32 copy of the pass vector (float32 pass only)
  auto to32 = [&](const double* src, bool all) {
    if constexpr (sizeof(TX) == 4) {
#pragma unroll
      for (int c = 0; c < K; ++c)
        if (c < T.kc && (all || live(c)))
          for (int j = gt; j < d; j += GT) T.v32[(size_t)c * d + j] = (float)src[(size_t)c * d + j];
    }
  };
  // one pass over A with the vector src (float64, or its float32 copy), then a grid barrier
  auto apass = [&](const double* src) -> bool {
    const uint64_t t0 = global_ns();
    const bool r = core.consume(ap, f32v ? (const void*)T.v32 : (const void*)src, T.partials, it);
    apass_ns += (long long)(global_ns() - t0);
    ++passes;
    if (!r) *(volatile int*)&T.head->abort = 1;
    return grid_sync(T.head, sh, T.st) && r;
  };
  double dv[K];

  // ---------------------------------------------------------------- prologue
  if (T.resid) {
    // PCG: r = b - H x;  IHS: g = H x - b
    to32(T.x, true);
    ok = grid_sync(T.head, sh, T.st);
    if (ok) ok = apass(T.x);
    zero(dv);
    if (ok) reduce_phase<TX, K>(T, d, nparts, T.x, pcg ? -1.0 : 1.0, T.b, pcg ? 1.0 : -1.0, T.r, nullptr, dv, sh);
    if (ok) ok = grid_sync(T.head, sh, T.st);
  }
  const double dsgn = pcg ? 1.0 : -1.0;  // r = b - H x (PCG) or g = H x - b (IHS)
  double dz[K];
  if (ok && T.restart) {
    zero(dv);
    ok = apply_phase<K>(T, d, T.r, T.rt, dv, sh);
    if (ok) cta_sum_to<K>(dv, sh, dots + 3, kLoopDots);
    if (ok && T.xstar && T.first) {
      // trace mode: delta_0 = 1/2 (x* - x_0)^T r_0
      zero(dz);
#pragma unroll
      for (int c = 0; c < K; ++c)
        if (c < T.kc)
          for (int j = gt; j < d; j += GT) {
            const size_t e = (size_t)c * d + j;
            dz[c] = fma(T.xstar[e] - T.x[e], T.r[e], dz[c]);
          }
      named_bar_sync(1, kConsumers);
      cta_sum_to<K>(dz, sh, dots + 4, kLoopDots);
    }
    if (ok) ok = grid_sync(T.head, sh, T.st);
    if (ok) {
      if (T.xstar && T.first) {
        grid_col_sums<K>(T.dots, 4, sh);
        if (tid == 0)
          for (int c = 0; c < T.kc; ++c) sh->col[c].delta = sh->col[c].delta0 = 0.5 * dsgn * sh->sum[c];
        named_bar_sync(1, kConsumers);
      }
      grid_col_sums<K>(T.dots, 3, sh);
      if (tid == 0) {
        for (int c = 0; c < T.kc; ++c) {
          LoopCol& s = sh->col[c];
          if (!s.active || s.stop) continue;
          const double dt = (pcg ? 1.0 : 0.5) * sh->sum[c];
          s.dt = dt;
          s.dI = dt;
          s.I = s.t;
          s.accept = 1;
          s.rejected = 0;
          if (!isfinite(dt)) s.numeric = 1;
          if (dt <= 0.0) s.stop = 1;
          if (T.first) {
            s.dt0 = dt;
            s.stop_abs = T.rel2 > 0.0 ? T.rel2 * dt : 0.0;
            if (T.outer_tol2 > 0.0) {
              // refinement: the decrement at the outer iterate estimates its error
              const double est2 = s.btx_outer > 0.0 ? T.fac * dt / s.btx_outer : (dt <= 0.0 ? 0.0 : 1.0);
              if (est2 <= T.outer_tol2 || dt <= 0.0) {
                s.outer_done = 1;
                s.stop = 1;
              }
            }
          }
          if (s.stop_abs > 0.0 && dt <= s.stop_abs) s.stop = 1;
        }
      }
      named_bar_sync(1, kConsumers);
      // PCG: p = r~;  IHS: x+ = x - mu v
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (!live(c)) continue;
        for (int j = gt; j < d; j += GT) {
          const size_t e = (size_t)c * d + j;
          if (pcg) T.p[e] = T.rt[e];
          else T.xp[e] = T.x[e] - T.mu * T.rt[e];
        }
      }
      to32(pcg ? T.p : T.xp, false);
      ok = grid_sync(T.head, sh, T.st);
    }
  }

  // ---------------------------------------------------------------- iterations
  while (ok) {
    bool any = false;
#pragma unroll
    for (int c = 0; c < K; ++c) any = any || live(c);
    if (!any) break;
    // 1-2: the pass over A and its reduction
    if (!(ok = apass(pcg ? T.p : T.xp))) break;
    zero(dv);
    if (pcg) reduce_phase<TX, K>(T, d, nparts, T.p, 1.0, nullptr, 0.0, T.Hp, T.p, dv, sh);
    else reduce_phase<TX, K>(T, d, nparts, T.xp, 1.0, T.b, -1.0, T.rp, nullptr, dv, sh);
    if (pcg) {
      cta_sum_to<K>(dv, sh, dots + 0, kLoopDots);
      if (!(ok = grid_sync(T.head, sh, T.st))) break;
      // 3: alpha, x+ and r+
      grid_col_sums<K>(T.dots, 0, sh);
      if (tid == 0)
        for (int c = 0; c < T.kc; ++c) {
          LoopCol& s = sh->col[c];
          const double pHp = sh->sum[c];
          const double alpha = s.dt / pHp;
          sh->alpha[c] = alpha;
          if (live(c) && (!(pHp > 0.0) || !isfinite(alpha))) s.numeric = 1;
        }
      named_bar_sync(1, kConsumers);
#pragma unroll
      for (int c = 0; c < K; ++c) {
        if (!live(c)) continue;
        const double alpha = sh->alpha[c];
        for (int j = gt; j < d; j += GT) {
          const size_t e = (size_t)c * d + j;
          T.xp[e] = T.x[e] + alpha * T.p[e];
          T.rp[e] = T.r[e] - alpha * T.Hp[e];
        }
      }
    }
    if (!(ok = grid_sync(T.head, sh, T.st))) break;
    // 4: r~+ = H_S^{-1} r+ (IHS: v+ = H_S^{-1} g+) and the decrement
    zero(dv);
    if (!(ok = apply_phase<K>(T, d, T.rp, T.rtp, dv, sh))) break;
    cta_sum_to<K>(dv, sh, dots + 1, kLoopDots);
    if (!(ok = grid_sync(T.head, sh, T.st))) break;
    grid_col_sums<K>(T.dots, 1, sh);
    // 5: the improvement test of Algorithm 2 / Algorithm 1
    if (tid == 0) {
      int anyrej = 0;
      for (int c = 0; c < T.kc; ++c) {
        LoopCol& s = sh->col[c];
        if (!live(c)) continue;
        const double dp = (pcg ? 1.0 : 0.5) * sh->sum[c];
        const double thr = T.c * pow(T.phi, (double)(s.t + 1 - s.I));
        const double ratio = dp / s.dI;
        s.dp = dp;
        s.ratio = ratio;
        s.thr = thr;
        if (!isfinite(dp)) s.numeric = 1;
        const int reject = (ratio > thr) && T.can_double;
        s.accept = !reject;
        s.rejected = reject;
        anyrej |= reject;
        sh->evi[c] = -1;
        if (blockIdx.x == 0 && T.trace && T.head->trace_len < T.trace_cap) {
          sh->evi[c] = T.head->trace_len;
          LoopTraceEv& ev = T.trace[T.head->trace_len++];
          ev.t = s.t;
          ev.m = T.m;
          ev.ratio = ratio;
          ev.thr = thr;
          ev.accepted = !reject;
          ev.column = c;
          ev.delta = s.delta;  // the kept iterate's; accepted steps are updated below
          ev.delta0 = s.delta0;
        }
      }
      sh->any_reject = anyrej;
    }
    named_bar_sync(1, kConsumers);
    // accepted columns shift; b^T x (and, in trace mode, (x* - x+)^T r+)
    zero(dv);
    zero(dz);
#pragma unroll
    for (int c = 0; c < K; ++c) {
      if (!live(c) || !sh->col[c].accept) continue;
      const double beta = sh->col[c].dp / sh->col[c].dt;
      for (int j = gt; j < d; j += GT) {
        const size_t e = (size_t)c * d + j;
        const double xn = T.xp[e];
        T.x[e] = xn;
        T.r[e] = T.rp[e];
        T.rt[e] = T.rtp[e];
        if (pcg) T.p[e] = T.rtp[e] + beta * T.p[e];
        else T.xp[e] = xn - T.mu * T.rtp[e];  // the next proposal
        dv[c] = fma(T.b[e], xn, dv[c]);
        if (T.xstar) dz[c] = fma(T.xstar[e] - xn, T.rp[e], dz[c]);
        if (f32v) T.v32[e] = (float)(pcg ? T.p[e] : T.xp[e]);
      }
    }
    cta_sum_to<K>(dv, sh, dots + 2, kLoopDots);
    if (T.xstar) {
      named_bar_sync(1, kConsumers);
      cta_sum_to<K>(dz, sh, dots + 4, kLoopDots);
    }
    if (!(ok = grid_sync(T.head, sh, T.st))) break;
    if (T.xstar) {
      grid_col_sums<K>(T.dots, 4, sh);
      if (tid == 0)
        for (int c = 0; c < T.kc; ++c) {
          if (!live(c) || !sh->col[c].accept) continue;
          sh->col[c].delta = 0.5 * dsgn * sh->sum[c];
          if (blockIdx.x == 0 && sh->evi[c] >= 0) T.trace[sh->evi[c]].delta = sh->col[c].delta;
        }
      named_bar_sync(1, kConsumers);
    }
    grid_col_sums<K>(T.dots, 2, sh);
    // 6: the stop rule
    if (tid == 0) {
      for (int c = 0; c < T.kc; ++c) {
        LoopCol& s = sh->col[c];
        if (!live(c) || !s.accept) continue;
        const double dp = s.dp, btx = sh->sum[c];
        s.btx = btx;
        s.dt = dp;
        s.t += 1;
        s.stop = (dp <= 0.0) || ((pcg ? dp : 2.0 * dp) <= T.tol2 * btx) || (dp <= s.stop_abs);
      }
    }
    ++iters;
    named_bar_sync(1, kConsumers);
    if (sh->any_reject) break;
  }

  // ---------------------------------------------------------------- leave
  if (tid == 0) *(volatile int*)&sh->quit = 1;
  named_bar_sync(1, kConsumers);
  core.release(ap, it);
  if (tid == 0) {
    atomicMax((unsigned long long*)&T.head->apass_ns, (unsigned long long)apass_ns);
    if (blockIdx.x == 0) {
      for (int c = 0; c < K; ++c) T.cols[c] = sh->col[c];
      T.head->any_reject = sh->any_reject;
      T.head->iters = iters;
      T.head->apasses = passes;
    }
  }
}

template <typename TA, typename TX, int G, int QMAX, int K>
sks_status launch_loop_t(const ApassPlan& pl, const CUtensorMap* tmap, int64_t n, int64_t d, const LoopTask& task,
                         cudaStream_t stream, bool query_only) {
  auto kern = solve_loop_kernel<TA, TX, G, QMAX, K>;
  const size_t smem = pl.smem + sizeof(LoopShared) + 16;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  if (per_sm < 1) return fail(SKS_ERR_UNSUPPORTED, "solver loop: the kernel does not fit an SM");
  // the partial sums are laid out for the plan's grid: never launch more CTAs
  const int grid = std::min(pl.grid, per_sm * sms);
  if (query_only) return SKS_OK;
  ApassArgs a;
  a.d = (int)d;
  a.dp = pl.dp;
  a.boxw = pl.boxw;
  a.nbox = pl.nbox;
  a.rows = pl.rows_per_stage;
  a.stages = pl.stages;
  a.q = pl.q;
  a.ntiles = (int)((std::max<int64_t>(n, 1) + pl.rows_per_stage - 1) / pl.rows_per_stage);
  a.x = nullptr;
  a.partials = nullptr;
  a.st = task.st;
  a.bulk = pl.bulk;
  a.n = n;
  a.A = (const char*)pl.A;
  a.lda_bytes = pl.lda_bytes;
  CUtensorMap map = *tmap;
  LoopTask t = task;
  void* args[] = {(void*)&map, (void*)&a, (void*)&t};
  SKS_CUDA_TRY(cudaLaunchCooperativeKernel((const void*)kern, dim3((unsigned)grid), dim3(kThreads), args, smem,
                                           stream));
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

sks_status dispatch(const ApassPlan& pl, const CUtensorMap* tmap, int64_t n, int64_t d, int K, bool a_f32,
                    bool vec_f32, const LoopTask& task, cudaStream_t stream, bool query_only) {
  if (pl.wide) return fail(SKS_ERR_UNSUPPORTED, "solver loop: rows wider than 4096 columns");
  if (!(K == 1 || K == 8)) return fail(SKS_ERR_UNSUPPORTED, "solver loop: K must be 1 or 8");
#define SKS_LOOP(TA, TX, G, Q, KK) return launch_loop_t<TA, TX, G, Q, KK>(pl, tmap, n, d, task, stream, query_only)
  if (!a_f32) {
    if (vec_f32) return fail(SKS_ERR_UNSUPPORTED, "solver loop: float64 A with float32 vectors");
    if (K == 8) SKS_LOOP(double, double, 256, 2, 8);
    if (pl.group == 32) SKS_LOOP(double, double, 32, 8, 1);
    if (pl.group == 128) SKS_LOOP(double, double, 128, 8, 1);
    SKS_LOOP(double, double, 256, 8, 1);
  }
  if (!vec_f32) return fail(SKS_ERR_UNSUPPORTED, "solver loop: float32 A needs the float32 pass");
  if (K == 8 && pl.group == 128) SKS_LOOP(float, float, 128, 2, 8);
  if (K == 8) SKS_LOOP(float, float, 256, 1, 8);
  if (pl.group == 32) SKS_LOOP(float, float, 32, 4, 1);
  if (pl.group == 128) SKS_LOOP(float, float, 128, 4, 1);
  SKS_LOOP(float, float, 256, 4, 1);
#undef SKS_LOOP
}

}  // namespace

sks_status loop_supported(const ApassPlan& plan, int64_t d, int K, bool a_f32, bool vec_f32) {
  const DeviceInfo& di = device_info();
  int coop = 0;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, di.device >= 0 ? di.device : 0) != cudaSuccess ||
      !coop) {
    cudaGetLastError();
    return fail(SKS_ERR_UNSUPPORTED, "solver loop: no cooperative launch on this device");
  }
  LoopTask none;
  std::memset(&none, 0, sizeof(none));
  return dispatch(plan, nullptr, 1, d, K, a_f32, vec_f32, none, nullptr, true);
}

sks_status loop_launch(const ApassPlan& plan, const CUtensorMap* tmap, int64_t n, int64_t d, bool a_f32, bool vec_f32,
                       const LoopTask& task, cudaStream_t stream) {
  return dispatch(plan, tmap, n, d, task.K, a_f32, vec_f32, task, stream, false);
}

size_t loop_partial_bytes(const ApassPlan& plan, int64_t d, int K, bool vec_f32) {
  return (size_t)plan.grid * (kConsumers / plan.group) * (size_t)K * (size_t)d * (vec_f32 ? 4 : 8) + 256;
}

size_t loop_dots_bytes(const ApassPlan& plan, int K) {
  return (size_t)plan.grid * K * kLoopDots * sizeof(double) + 256;
}

void loop_adjust_plan(ApassPlan* pl, bool a_f32, bool vec_f32) {
  const DeviceInfo& di = device_info();
  const int ctas = (a_f32 && vec_f32 && !pl->wide) ? 2 : 1;
  const size_t optin = di.smem_optin ? di.smem_optin : 232448;
  const size_t budget = optin / ctas - (ctas > 1 ? 1024 : 0);
  const size_t stage_bytes = (size_t)pl->rows_per_stage * pl->dp * (a_f32 ? 4 : 8);
  const size_t extra = sizeof(LoopShared) + 16;
  while (pl->smem + extra > budget && pl->stages > 2) {
    pl->stages -= 1;
    pl->smem -= stage_bytes + 16;
  }
}

}  // namespace sks
