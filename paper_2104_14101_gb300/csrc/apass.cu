// apass.cu -- K1 as a stand-alone launch: the Hessian pass
//     y = A^T (A x) + nu^2 Lambda x   in ONE read of A
// (Section 4.1.2: the O(nd) gradient / H p cost that dominates every
// iteration of the IHS and of PCG).  The pass itself (a persistent grid of
// CTAs, one producer warp streaming row tiles of A by tensor copies, eight
// consumer warps keeping sum_i (a_i^T x) a_i in registers) is apass_core.cuh;
// here one launch makes one pass and apass_finalize sums the partial vectors
// in float64 and adds nu^2 lambda .* x.  The plan (grid, stage geometry,
// group size) is shared with the device-resident solver loop (loop.cu).
#include <algorithm>
#include <type_traits>

#include "apass_core.cuh"

namespace sks {

namespace {

using namespace apcore;

// The stand-alone pass: one pass per launch; partial sums summed by apass_finalize.
template <typename TA, typename TX, int G, int QMAX, int K, bool XG = false>
__global__ void __launch_bounds__(kThreads, (sizeof(TA) == 4 && QMAX <= 4 && !(K == 8 && QMAX > 1) &&
                                             (sizeof(TX) == 4 || (!XG && K == 1)))
                                                ? 2
                                                : 1)
    apass_kernel(const __grid_constant__ CUtensorMap tmap, ApassArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  ApassCore<TA, TX, G, QMAX, K, XG> core;
  core.carve(smem, a);
  if (threadIdx.x == 0) core.init(a);
  __syncthreads();
  if (threadIdx.x >= kConsumers) {
    if (threadIdx.x == kConsumers) core.produce(&tmap, a, 1, nullptr);
    return;
  }
  int it = 0;
  core.consume(a, a.x, a.partials, it);
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
  // eight float32 right-hand sides: four warps per row, two column vectors each (half the
  // cross-warp reductions per element of a whole-CTA row)
  if (k == 8 && a_f32 && vec_f32 && nvec <= 128 * 2) {
    group = 128;
    qmax = 2;
  }
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
  // the float32 pass (HBM-bound, latency-limited at one CTA per SM) and the
  // double-float pass with one right-hand side (bound by its float32 operation
  // chains) run two CTAs per SM, each with half the shared memory
  const int ctas_per_sm = (a_f32 && !wide && (vec_f32 || k == 1) && !(k == 8 && qmax > 1)) ? 2 : 1;
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
    if (k == 8 && pl.group == 128) return launch_t<float, float, 128, 2, 8>(SKS_APASS_ARGS);
    if (k == 8) return launch_t<float, float, 256, 1, 8>(SKS_APASS_ARGS);
    if (pl.group == 32) return launch_t<float, float, 32, 4, 1>(SKS_APASS_ARGS);
    if (pl.group == 128) return launch_t<float, float, 128, 4, 1>(SKS_APASS_ARGS);
    return launch_t<float, float, 256, 4, 1>(SKS_APASS_ARGS);
  }
  // float32 A, float64 vectors: double-float arithmetic (~2^-44 relative)
  if (k == 8) {
    // two passes of four columns each: the eight double-float accumulators and
    // vectors of one pass do not fit a thread's registers (spills); the second
    // read of A costs less than the spills
    const size_t h = (size_t)4 * d;
    const double* xd = (const double*)x;
    const double* ad = (const double*)addv;
    double* yd = (double*)y;
    SKS_TRY((launch_t<float, df32, 256, 1, 4>(pl, tmap, n, d, xd, yd, nu2, lambda, partials, st, stream, sgn, ad,
                                               addc, ev_begin, nullptr)));
    return launch_t<float, df32, 256, 1, 4>(pl, tmap, n, d, xd + h, yd + h, nu2, lambda, partials, st, stream, sgn,
                                            ad ? ad + h : nullptr, addc, nullptr, ev_end);
  }
  if (pl.group == 32) return launch_t<float, df32, 32, 4, 1>(SKS_APASS_ARGS);
  if (pl.group == 128) return launch_t<float, df32, 128, 4, 1>(SKS_APASS_ARGS);
  return launch_t<float, df32, 256, 4, 1>(SKS_APASS_ARGS);
#undef SKS_APASS_ARGS
}

}  // namespace sks
