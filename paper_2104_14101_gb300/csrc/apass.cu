// apass.cu -- K1: the Hessian pass  y = A^T (A x) + nu^2 Lambda x  in ONE read
// of A (Section 4.1.2: the O(nd) gradient / H p cost that dominates every
// iteration of the IHS and of PCG).
//
// Design (GB300): a persistent grid, one CTA per SM.  Warp 8 is a producer
// that streams row tiles of A into a ring of shared-memory stages with 2-D
// bulk tensor copies (TMA, mbarrier completion); warps 0-7 consume.  Every
// consumer thread owns a fixed set of 16-byte column vectors of the row, so
// the running sum  sum_i (a_i^T x) a_i  stays in its registers for the whole
// pass.  Per row, the dot a_i^T x is reduced over the group of threads that
// shares the row (a warp for narrow rows, the 256 consumers for wide rows).
// Each CTA (or warp group) writes one partial d-vector; a second small kernel
// sums the partials in float64 and adds nu^2 lambda .* x.
// Rows and columns past the edge of A are zero-filled by the tensor copy, so
// there is no tail handling in the inner loop.
#include <algorithm>
#include <type_traits>

#include "internal.h"

namespace sks {

namespace {

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
  const void* x;  // d x K column-major, vector type
  void* partials; // [grid * NG][K][d]
  DevStatus* st;
};

SKS_HD size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// XG: wide rows -- the thread's slice of x is read through L1 at each use
// instead of being held in registers (the accumulators need them).
template <typename TA, typename TX, int G, int QMAX, int K, bool XG = false>
__global__ void __launch_bounds__(kThreads, (sizeof(TA) == 4 && sizeof(TX) == 4 && QMAX <= 4) ? 2 : 1)
    apass_kernel(const __grid_constant__ CUtensorMap tmap, ApassArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  constexpr int VEC = Vec<TA>::N;
  constexpr int NG = kConsumers / G;
  const int tid = threadIdx.x;
  const size_t stage_elems = (size_t)a.rows * a.dp;
  TA* stage0 = (TA*)smem;
  size_t off = align_up((size_t)a.stages * stage_elems * sizeof(TA), 128);
  using AT = Acc<TX>;
  TX* red = (TX*)(smem + off);
  off += align_up((size_t)2 * 8 * kRC * K * sizeof(TX), 128);
  uint64_t* full = (uint64_t*)(smem + off);
  uint64_t* empty = full + a.stages;
  if (tid == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumers / 32);
    }
    fence_mbar_init();
    fence_proxy_async();
  }
  __syncthreads();

  const uint32_t stage_bytes = (uint32_t)(stage_elems * sizeof(TA));

  if (tid >= kConsumers) {
    // ------------------------------------------------------------ producer
    if (tid == kConsumers) {
      int it = 0;
      for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
        const int s = it % a.stages;
        const uint32_t ph = (uint32_t)(it / a.stages) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, a.st, 12)) break;
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
            tma_load_2d(dst + (size_t)b * a.rows * a.boxw, &tmap, &full[s], b * a.boxw, tile * a.rows);
        }
      }
      // drain: every issued copy has landed before the CTA may exit
      const int first = it > a.stages ? it - a.stages : 0;
      for (int k = first; k < it; ++k) mbar_wait(&full[k % a.stages], (uint32_t)(k / a.stages) & 1u, a.st, 13);
    }
    return;
  }

  // -------------------------------------------------------------- consumers
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
  const typename AT::In* xg = (const typename AT::In*)a.x;
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
  int it = 0;
  for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
    const int s = it % a.stages;
    const uint32_t ph = (uint32_t)(it / a.stages) & 1u;
    const bool ok = mbar_wait_warp(&full[s], ph, a.st, 11);
    // narrow rows: the warp is the group and leaves on its own.  Wide rows: a
    // timed-out warp reads the (stale) stage like the others and the group
    // leaves together at the reduction barrier below.
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
    if (stop) break;
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  typename AT::Out* out = (typename AT::Out*)a.partials + (size_t)(blockIdx.x * NG + g) * K * a.d;
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
}

// y[c][j] = sum_p partials[p][c][j] + nu2 * lambda[j] * x[c][j]   (float64 sum)
// (y = sgn * H x + addc * addv when addv is given: residuals b - H x, gradients H x - b)
template <typename TX>
__global__ void apass_finalize(int nparts, int d, int k, const TX* __restrict__ partials, const TX* __restrict__ x,
                               TX* __restrict__ y, double nu2, const double* __restrict__ lambda, double sgn,
                               const TX* __restrict__ addv, double addc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (j >= d) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int p = 0;
  for (; p + 3 < nparts; p += 4) {
    s0 += (double)partials[((size_t)(p + 0) * k + c) * d + j];
    s1 += (double)partials[((size_t)(p + 1) * k + c) * d + j];
    s2 += (double)partials[((size_t)(p + 2) * k + c) * d + j];
    s3 += (double)partials[((size_t)(p + 3) * k + c) * d + j];
  }
  for (; p < nparts; ++p) s0 += (double)partials[((size_t)p * k + c) * d + j];
  const double xv = (double)x[(size_t)c * d + j];
  double v = sgn * ((s0 + s1) + (s2 + s3) + nu2 * lambda[j] * xv);
  if (addv) v += addc * (double)addv[(size_t)c * d + j];
  y[(size_t)c * d + j] = (TX)v;
}

template <typename TA, typename TX, int G, int QMAX, int K, bool XG = false>
sks_status launch_t(const ApassPlan& pl, const CUtensorMap* tmap, int64_t n, int64_t d, const void* x,
                    void* y, double nu2, const double* lambda, void* partials, DevStatus* st, cudaStream_t stream,
                    double sgn, const void* addv, double addc, cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  auto kern = apass_kernel<TA, TX, G, QMAX, K, XG>;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pl.smem));
  const int nparts = pl.grid * (kConsumers / G);
  if (n > 0) {
    ApassArgs a;
    a.d = (int)d;
    a.dp = pl.dp;
    a.boxw = pl.boxw;
    a.nbox = pl.nbox;
    a.rows = pl.rows_per_stage;
    a.stages = pl.stages;
    a.q = pl.q;
    a.ntiles = (int)((n + pl.rows_per_stage - 1) / pl.rows_per_stage);
    a.x = x;
    a.partials = partials;
    a.st = st;
    a.bulk = pl.bulk;
    a.n = n;
    a.A = (const char*)pl.A;
    a.lda_bytes = pl.lda_bytes;
    if (ev_begin) SKS_CUDA_TRY(cudaEventRecord(ev_begin, stream));
    kern<<<pl.grid, kThreads, pl.smem, stream>>>(*tmap, a);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    if (ev_end) SKS_CUDA_TRY(cudaEventRecord(ev_end, stream));
  } else if (ev_begin && ev_end) {
    SKS_CUDA_TRY(cudaEventRecord(ev_begin, stream));
    SKS_CUDA_TRY(cudaEventRecord(ev_end, stream));
  }
  dim3 fg((unsigned)((d + 127) / 128), (unsigned)K);
  using TO = typename Acc<TX>::Out;
  apass_finalize<TO><<<fg, 128, 0, stream>>>(n > 0 ? nparts : 0, (int)d, K, (const TO*)partials, (const TO*)x,
                                               (TO*)y, nu2, lambda, sgn, (const TO*)addv, addc);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

int vec_of(bool a_f32) { return a_f32 ? 4 : 2; }

}  // namespace

sks_status apass_plan(int64_t n, int64_t d, int64_t k, bool a_f32, bool vec_f32, ApassPlan* pl) {
  if (d < 1 || d > kApassMaxD(a_f32))
    return fail(SKS_ERR_UNSUPPORTED, a_f32 ? "A-pass supports 1 <= d <= 16384 (float32 A)"
                                           : "A-pass supports 1 <= d <= 14336 (float64 A)");
  if (d > 4096 && k != 1) return fail(SKS_ERR_UNSUPPORTED, "A-pass: d > 4096 with one right-hand side only");
  if (!(k == 1 || k == 8)) return fail(SKS_ERR_UNSUPPORTED, "A-pass kernel instantiated for k in {1, 8}");
  const int vec = vec_of(a_f32);
  const size_t esz = a_f32 ? 4 : 8, xsz = vec_f32 ? 4 : 8;
  const int boxw = (int)std::min<int64_t>(256, (d + vec - 1) / vec * vec);
  const int nbox = (int)((d + boxw - 1) / boxw);
  const int dp = nbox * boxw;
  const int nvec = dp / vec;
  // narrow rows: one warp per row; wide rows: all 256 consumers per row.
  // Per-thread column vectors: 8 (float64 A, 2 per vector) or 4 (float32 A,
  // 4 per vector), i.e. 16 register-resident accumulators per right-hand side.
  const int qcap = a_f32 ? 4 : 8;
  int group = 256;
  if (k == 1) {
    if (nvec <= 32 * qcap) group = 32;
    else if (nvec <= 128 * qcap) group = 128;
  }
  int qmax = (k == 8) ? (a_f32 ? 1 : 2) : qcap;
  const bool wide = d > 4096;  // more column vectors per thread, one CTA per SM (float64 / double-float: x through L1)
  if (wide) qmax = a_f32 ? kWideQF32 : kWideQF64;
  const int q = (nvec + group - 1) / group;
  if (q > qmax) return fail(SKS_ERR_UNSUPPORTED, "A-pass: row too wide for this instantiation");
  const int ng = kConsumers / group;
  const size_t row_bytes = (size_t)dp * esz;
  // stages of ~32 KB; wide rows: ~64 KB, so that a stage holds the kRC rows
  // reduced together by the 256 consumers (one barrier per kRC rows)
  int rows = (int)std::max<size_t>(1, (wide ? 64 * 1024 : 32 * 1024) / row_bytes);
  rows = std::max(rows, ng);
  rows = std::min(rows, 256);
  rows = rows / ng * ng;
  const DeviceInfo& di = device_info();
  // the float32 pass (HBM-bound, latency-limited at one CTA per SM) runs two
  // CTAs per SM, each with half the shared memory
  const int ctas_per_sm = (a_f32 && vec_f32 && !wide) ? 2 : 1;
  const size_t budget = (di.smem_optin ? di.smem_optin : 232448) / ctas_per_sm - (ctas_per_sm > 1 ? 1024 : 0);
  const size_t fixed = ((size_t)2 * 8 * kRC * k * xsz + 127) / 128 * 128;
  const size_t stage_bytes = ((size_t)rows * row_bytes);
  int stages = (int)std::min<size_t>(8, (budget - fixed - 1024) / stage_bytes);
  if (stages < 2) return fail(SKS_ERR_UNSUPPORTED, "A-pass: shared memory too small");
  const int64_t ntiles = (n + rows - 1) / rows;
  const int sms = di.sms > 0 ? di.sms : 152;
  pl->grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, (int64_t)sms * ctas_per_sm));
  pl->wide = wide ? 1 : 0;
  pl->group = group;
  pl->q = q;
  pl->rows_per_stage = rows;
  pl->stages = stages;
  pl->boxw = boxw;
  pl->nbox = nbox;
  pl->dp = dp;
  pl->smem = (size_t)stages * stage_bytes + fixed + 2 * 8 * stages + 256;
  pl->partial_elems = (size_t)pl->grid * ng * k * d;
  return SKS_OK;
}

void apass_use_bulk(ApassPlan* pl, const void* A, int64_t d, int64_t lda, bool a_f32) {
  const size_t esz = a_f32 ? 4 : 8;
  if ((d * esz) % 16 != 0 || (lda * esz) % 16 != 0 || ((uintptr_t)A & 15) != 0) return;
  // stage layout [rows][d]: same byte budget, no padding (d <= dp)
  pl->bulk = 1;
  pl->boxw = (int)d;
  pl->nbox = 1;
  pl->dp = (int)d;
  pl->A = A;
  pl->lda_bytes = (long long)(lda * esz);
}

size_t apass_workspace_bytes(int64_t n, int64_t d, int64_t k, bool a_f32, bool vec_f32) {
  ApassPlan pl;
  if (apass_plan(n, d, k, a_f32, vec_f32, &pl) != SKS_OK) return 0;
  return pl.partial_elems * (vec_f32 ? 4 : 8) + 256;
}

sks_status apass_launch(const ApassPlan& pl, const CUtensorMap* tmap, int64_t n, int64_t d, int64_t k, bool a_f32,
                        bool vec_f32, const void* x, void* y, double nu2, const double* lambda, void* partials,
                        DevStatus* st, cudaStream_t stream, double sgn, const void* addv, double addc,
                        cudaEvent_t ev_begin, cudaEvent_t ev_end) {
  if (!a_f32 && vec_f32) return fail(SKS_ERR_UNSUPPORTED, "float64 A with float32 vectors");
#define SKS_APASS_ARGS pl, tmap, n, d, x, y, nu2, lambda, partials, st, stream, sgn, addv, addc, ev_begin, ev_end
  if (pl.wide) {
    if (!a_f32) return launch_t<double, double, 256, kWideQF64, 1, true>(SKS_APASS_ARGS);
    // float32 inner pass: the thread's slice of x in registers (8 or 16 column vectors)
    if (vec_f32 && pl.q <= 8) return launch_t<float, float, 256, 8, 1, false>(SKS_APASS_ARGS);
    if (vec_f32) return launch_t<float, float, 256, kWideQF32, 1, false>(SKS_APASS_ARGS);
    return launch_t<float, df32, 256, kWideQF32, 1, true>(SKS_APASS_ARGS);
  }
  if (!a_f32) {
    if (k == 8) return launch_t<double, double, 256, 2, 8>(SKS_APASS_ARGS);
    if (pl.group == 32) return launch_t<double, double, 32, 8, 1>(SKS_APASS_ARGS);
    if (pl.group == 128) return launch_t<double, double, 128, 8, 1>(SKS_APASS_ARGS);
    return launch_t<double, double, 256, 8, 1>(SKS_APASS_ARGS);
  }
  if (vec_f32) {
    if (k == 8) return launch_t<float, float, 256, 1, 8>(SKS_APASS_ARGS);
    if (pl.group == 32) return launch_t<float, float, 32, 4, 1>(SKS_APASS_ARGS);
    if (pl.group == 128) return launch_t<float, float, 128, 4, 1>(SKS_APASS_ARGS);
    return launch_t<float, float, 256, 4, 1>(SKS_APASS_ARGS);
  }
  // float32 A, float64 vectors: double-float arithmetic (~2^-44 relative)
  if (k == 8) return launch_t<float, df32, 256, 1, 8>(SKS_APASS_ARGS);
  if (pl.group == 32) return launch_t<float, df32, 32, 4, 1>(SKS_APASS_ARGS);
  if (pl.group == 128) return launch_t<float, df32, 128, 4, 1>(SKS_APASS_ARGS);
  return launch_t<float, df32, 256, 4, 1>(SKS_APASS_ARGS);
#undef SKS_APASS_ARGS
}

}  // namespace sks
