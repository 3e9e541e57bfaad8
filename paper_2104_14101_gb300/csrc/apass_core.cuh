// apass_core.cuh -- the machinery of K1, the Hessian pass
//     y = A^T (A x) + nu^2 Lambda x   in ONE read of A
// (Section 4.1.2: the O(nd) cost of every iteration of the IHS and of PCG),
// shared by the stand-alone pass (apass.cu) and the device-resident solver
// loop (loop.cu), which runs one pass per iteration inside one launch.
//
// A CTA is 8 consumer warps plus one producer warp.  The producer streams the
// CTA's row tiles of A (tiles blockIdx.x, blockIdx.x + gridDim.x, ...) into a
// ring of shared-memory stages (2-D tensor copies, or whole-row 1-D bulk
// copies when rows are 16-byte multiples) with mbarrier completion; in the
// loop it keeps streaming the same tile sequence pass after pass, since A does
// not change.  Every consumer thread owns a fixed set of 16-byte column
// vectors of a row, so the running sum  sum_i (a_i^T x) a_i  stays in its
// registers for the whole pass; the row dots a_i^T x are reduced over the
// group of threads sharing the row (a warp for narrow rows, the 256 consumers
// for wide rows).  Each warp group writes one partial d-vector per pass.
// Rows and columns past the edge of A are zero-filled by the tensor copy, so
// the inner loop has no tail handling.  All waits are bounded (SKS_ERR_TIMEOUT).
#pragma once

#include <type_traits>

#include "internal.h"

namespace sks {
namespace apcore {

template <typename TA>
struct Vec;
template <>
struct Vec<double> {
  using T = double2;
  static constexpr int N = 2;
  static SKS_DEV void load(const double* p, double* o) {
    const double2 v = *(const double2*)p;
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct Vec<float> {
  using T = float4;
  static constexpr int N = 4;
  static SKS_DEV void load(const float* p, float* o) {
    const float4 v = *(const float4*)p;
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};

// ------------------------------------------------------------ accumulator arithmetic
// float / double: plain arithmetic.  df32: double-float (an unevaluated sum of
// two floats, ~44-48 significant bits) built from float32 operations --
// TwoProd via fmaf and Knuth's TwoSum -- for the refinement residual, whose
// float64 version is bound by the float64 FMA rate on this part.
struct df32 {
  float h, l;
};

template <typename TX>
struct Acc {
  using T = TX;
  using In = TX;   // type of x in global memory
  using Out = TX;  // type of the partial sums
  static SKS_DEV T zero() { return T(0); }
  static SKS_DEV T from_in(In x) { return x; }
  template <typename TA>
  static SKS_DEV void mac(T& acc, TA a, const T& x) { acc += (T)a * x; }
  static SKS_DEV void add(T& a, const T& b) { a += b; }
  static SKS_DEV T wsum(T v) { return warp_sum(v); }
  static SKS_DEV Out out(const T& v) { return v; }
};

SKS_DEV void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bp = s - a;
  e = (a - (s - bp)) + (b - bp);
}

template <>
struct Acc<df32> {
  using T = df32;
  using In = double;
  using Out = double;
  static SKS_DEV T zero() { return df32{0.f, 0.f}; }
  static SKS_DEV T from_in(double x) {
    const float h = (float)x;
    return df32{h, (float)(x - (double)h)};
  }
  // acc += a * x  (a float, x double-float)
  static SKS_DEV void mac(T& acc, float a, const T& x) {
    const float ph = a * x.h;
    const float pl = fmaf(a, x.l, fmaf(a, x.h, -ph));
    float s, e;
    two_sum(acc.h, ph, s, e);
    acc.h = s;
    acc.l += e + pl;
  }
  static SKS_DEV void add(T& a, const T& b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    e += a.l + b.l;
    a.h = s + e;
    a.l = e - (a.h - s);
  }
  static SKS_DEV T wsum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const df32 w{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
      add(v, w);
    }
    return v;
  }
  static SKS_DEV Out out(const T& v) { return (double)v.h + (double)v.l; }
};


constexpr int kConsumers = 256;
constexpr int kThreads = kConsumers + 32;
constexpr int kRC = 2;  // rows reduced together
// wide rows (d > 4096): column vectors per thread (16 x 4 floats, 28 x 2 doubles)
constexpr int kWideQF32 = 16;
constexpr int kWideQF64 = 28;
constexpr int kApassMaxD(bool a_f32) { return a_f32 ? 256 * kWideQF32 * 4 : 256 * kWideQF64 * 2; }

struct ApassArgs {
  int d, dp, boxw, nbox, rows, stages, q, ntiles;
  int bulk;            // 1: whole rows by 1-D bulk copies (row-major [rows][d] stages)
  int64_t n;           // rows of A (bulk mode: rows past n are skipped)
  const char* A;       // bulk mode source
  long long lda_bytes;
  const void* x;       // d x K column-major, vector type (stand-alone pass)
  void* partials;      // [grid * NG][K][d] (stand-alone pass)
  DevStatus* st;
};

SKS_HD size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Shared memory of the pass: the stages, the row-dot exchange of wide groups
// and the 2 x stages mbarriers (bytes past `base`).
template <typename TA, typename TX>
SKS_HD size_t apass_smem_bytes(int stages, size_t stage_bytes, int K) {
  return align_up((size_t)stages * stage_bytes, 128) + align_up((size_t)2 * 8 * kRC * K * sizeof(TX), 128) +
         (size_t)2 * 8 * stages;
}

// XG: wide rows -- the thread's slice of x is read through L1 at each use
// instead of being held in registers (the accumulators need them).
template <typename TA, typename TX, int G, int QMAX, int K, bool XG = false>
struct ApassCore {
  static constexpr int VEC = Vec<TA>::N;
  static constexpr int NG = kConsumers / G;
  using AT = Acc<TX>;
  TA* stage0;
  TX* red;
  uint64_t* full;
  uint64_t* empty;
  size_t stage_elems;

  SKS_DEV void carve(unsigned char* smem, const ApassArgs& a) {
    stage_elems = (size_t)a.rows * a.dp;
    stage0 = (TA*)smem;
    size_t off = align_up((size_t)a.stages * stage_elems * sizeof(TA), 128);
    red = (TX*)(smem + off);
    off += align_up((size_t)2 * 8 * kRC * K * sizeof(TX), 128);
    full = (uint64_t*)(smem + off);
    empty = full + a.stages;
  }

  // one thread, before a __syncthreads
  SKS_DEV void init(const ApassArgs& a) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers / 32);
    }
    fence_mbar_init();
    fence_proxy_async();
  }

  // Producer thread: the CTA's tiles, `passes` times over (passes < 0: until
  // *quit is set, checked after every wait for a free stage), then waits
  // until every issued copy has landed.
  SKS_DEV void produce(const CUtensorMap* tmap, const ApassArgs& a, int passes, volatile int* quit) {
    const uint32_t stage_bytes = (uint32_t)(stage_elems * sizeof(TA));
    int it = 0;
    bool go = true;
    for (int pass = 0; go && (passes < 0 || pass < passes); ++pass) {
      for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        const int s = it % a.stages;
        const uint32_t ph = (uint32_t)(it / a.stages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, a.st, 12) || (quit && *quit)) {
          go = false;
          break;
        }
        TA* dst = stage0 + (size_t)s * stage_elems;
        if (a.bulk) {
          const int64_t r0 = (int64_t)tile * a.rows;
          const int valid = (int)min((int64_t)a.rows, a.n - r0);
          const uint32_t row_bytes = (uint32_t)(a.d * sizeof(TA));
          mbar_arrive_expect_tx(&full[s], (uint32_t)valid * row_bytes);
          for (int r = 0; r < valid; ++r)
            bulk_load(dst + (size_t)r * a.d, a.A + (r0 + r) * a.lda_bytes, row_bytes, &full[s]);
        } else {
          mbar_arrive_expect_tx(&full[s], stage_bytes);
          for (int b = 0; b < a.nbox; ++b)
            tma_load_2d(dst + (size_t)b * a.rows * a.boxw, tmap, &full[s], b * a.boxw, tile * a.rows);
        }
      }
    }
    // drain: every issued copy has landed before the CTA may exit
    const int first = it > a.stages ? it - a.stages : 0;
    for (int k = first; k < it; ++k) mbar_wait(&full[k % a.stages], (uint32_t)(k / a.stages) & 1u, a.st, 13);
  }

  // Consumers leaving a loop: once *quit is set, one more arrival of every
  // warp on the stage after the last consumed tile frees a producer that waits
  // for it (it then sees *quit and stops).
  SKS_DEV void release(const ApassArgs& a, int it) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[it % a.stages]);
  }

  // Consumer threads (tid < kConsumers): one pass over the CTA's tiles with
  // vector x (d x K, Acc<TX>::In), partial sums to `partials`; `it` counts
  // the tiles consumed so far (it is advanced).  Returns false after a
  // timed-out wait.
  SKS_DEV bool consume(const ApassArgs& a, const void* x, void* partials, int& it) {
    const int tid = threadIdx.x;
    const int g = tid / G, l = tid % G;
    const int warp = tid >> 5, lane = tid & 31;
    const int nvec = a.dp / VEC;
    const int rg = a.rows / NG;  // rows of a stage handled by this group
    TX acc[QMAX][VEC][K];
#pragma unroll
    for (int q = 0; q < QMAX; ++q)
#pragma unroll
      for (int e = 0; e < VEC; ++e)
#pragma unroll
        for (int c = 0; c < K; ++c) acc[q][e][c] = AT::zero();

    // the thread's slice of x (zero past column d) stays in registers for the whole pass
    const typename AT::In* xg = (const typename AT::In*)x;
    constexpr int QX = XG ? 1 : QMAX;
    TX xr[QX][VEC][K];
    if constexpr (!XG) {
#pragma unroll
      for (int q = 0; q < QMAX; ++q) {
        const int vi = l + q * G;
#pragma unroll
        for (int e = 0; e < VEC; ++e)
#pragma unroll
          for (int c = 0; c < K; ++c) {
            const int col = vi * VEC + e;
            xr[q][e][c] = (q < a.q && vi < nvec && col < a.d) ? AT::from_in(xg[(size_t)c * a.d + col]) : AT::zero();
          }
      }
    }

    // shared-memory offset of each of the thread's column vectors within a stage
    // row (the row stride is boxw in both stage layouts), hoisted out of the loops
    int soff[QMAX];
    bool qv[QMAX];
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int vi = l + q * G;
      qv[q] = q < a.q && vi < nvec;
      const int col = vi * VEC;
      const int b = col / a.boxw;
      soff[q] = b * a.rows * a.boxw + (col - b * a.boxw);
    }
    const int rstride = a.boxw;

    int buf = 0;
    bool all_ok = true;
    for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
      const int s = it % a.stages;
      const uint32_t ph = (uint32_t)(it / a.stages) & 1u;
      const bool ok = mbar_wait_warp(&full[s], ph, a.st, 11);
      // narrow rows: the warp is the group and leaves on its own.  Wide rows: a
      // timed-out warp reads the (stale) stage like the others and the group
      // leaves together at the reduction barrier below.
      if (!ok) all_ok = false;
      if (G <= 32 && !ok) break;
      const int valid = a.bulk ? (int)min((int64_t)a.rows, a.n - (int64_t)tile * a.rows) : a.rows;
      const TA* S = stage0 + (size_t)s * stage_elems;
      bool stop = false;
      for (int j0 = 0; j0 < rg; j0 += kRC) {
        // partial dots: one chain per column vector for a single right-hand
        // side (kRC * QMAX independent chains), one per (row, column) otherwise;
        // float64 keeps one chain per row (bound by the float64 pipe, where the
        // extra adds of the split would cost more than the latency it hides)
        constexpr int QD =
            QMAX <= 8 && ((K == 1 && std::is_same<TX, float>::value) || (K == 1 && !XG && !std::is_same<TX, double>::value))
                ? QMAX
                : 1;
        TX dq[kRC][QD][K];
#pragma unroll
        for (int rc = 0; rc < kRC; ++rc) {
          const int r = g + NG * (j0 + rc);
          const bool rok = (j0 + rc) < rg && r < valid;
          const TA* row = S + r * rstride;
#pragma unroll
          for (int q = 0; q < QD; ++q)
#pragma unroll
            for (int c = 0; c < K; ++c) dq[rc][q][c] = AT::zero();
#pragma unroll
          for (int q = 0; q < QMAX; ++q) {
            if (rok && qv[q]) {
              TA v[VEC];
              Vec<TA>::load(row + soff[q], v);
#pragma unroll
              for (int e = 0; e < VEC; ++e)
#pragma unroll
                for (int c = 0; c < K; ++c) {
                  if constexpr (XG) {
                    const int col = (l + q * G) * VEC + e;  // past d: A's staged value there is 0
                    const TX xv = col < a.d ? AT::from_in(__ldg(xg + (size_t)c * a.d + col)) : AT::zero();
                    AT::mac(dq[rc][QD > 1 ? q : 0][c], v[e], xv);
                  } else {
                    AT::mac(dq[rc][QD > 1 ? q : 0][c], v[e], xr[q][e][c]);
                  }
                }
            }
          }
        }
        TX dot[kRC][K];
#pragma unroll
        for (int rc = 0; rc < kRC; ++rc)
#pragma unroll
          for (int c = 0; c < K; ++c) {
#pragma unroll
            for (int w = 1; w < QD; w <<= 1)
#pragma unroll
              for (int q = 0; q + w < QD; q += 2 * w) AT::add(dq[rc][q][c], dq[rc][q + w][c]);
            dot[rc][c] = AT::wsum(dq[rc][0][c]);
          }
        if (G > 32) {
          TX* rb = red + buf * (8 * kRC * K);
          if (lane == 0) {
#pragma unroll
            for (int rc = 0; rc < kRC; ++rc)
#pragma unroll
              for (int c = 0; c < K; ++c) rb[warp * kRC * K + rc * K + c] = dot[rc][c];
          }
          if (named_bar_or(2 + g, G, !ok)) {
            stop = true;
            break;
          }
          constexpr int WPG = G / 32;  // warps per group
          const int w0 = g * WPG;
#pragma unroll
          for (int rc = 0; rc < kRC; ++rc)
#pragma unroll
            for (int c = 0; c < K; ++c) {
              TX t = AT::zero();
#pragma unroll
              for (int w = 0; w < WPG; ++w) AT::add(t, rb[(w0 + w) * kRC * K + rc * K + c]);
              dot[rc][c] = t;
            }
          buf ^= 1;
        }
        // rank-one updates  acc += (a_r^T x) a_r  (row re-read from shared memory)
#pragma unroll
        for (int rc = 0; rc < kRC; ++rc) {
          const int r = g + NG * (j0 + rc);
          if ((j0 + rc) < rg && r < valid) {
            const TA* row = S + r * rstride;
#pragma unroll
            for (int q = 0; q < QMAX; ++q) {
              if (qv[q]) {
                TA v[VEC];
                Vec<TA>::load(row + soff[q], v);
#pragma unroll
                for (int e = 0; e < VEC; ++e)
#pragma unroll
                  for (int c = 0; c < K; ++c) AT::mac(acc[q][e][c], v[e], dot[rc][c]);
              }
            }
          }
        }
      }
      if (stop) {
        all_ok = false;
        break;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }

    typename AT::Out* out = (typename AT::Out*)partials + (size_t)(blockIdx.x * NG + g) * K * a.d;
#pragma unroll
    for (int q = 0; q < QMAX; ++q) {
      const int vi = l + q * G;
      if (q < a.q && vi < nvec) {
#pragma unroll
        for (int e = 0; e < VEC; ++e) {
          const int col = vi * VEC + e;
          if (col < a.d)
#pragma unroll
            for (int c = 0; c < K; ++c) out[(size_t)c * a.d + col] = AT::out(acc[q][e][c]);
        }
      }
    }
    return all_ok;
  }
};

}  // namespace apcore
}  // namespace sks
