// solver.cu -- sketches, preconditioners and the adaptive solvers behind the
// C ABI (include/sks.h).
//
// Algorithm 2 (adaptive PCG) and Algorithm 1 with the IHS step (Theorem 3.2)
// run as a host loop that only queues work: every iteration is one A-pass
// (K1) plus three small kernels (the step, the preconditioner apply, the
// improvement test).  The test's verdict lives in a device control block;
// the host reads that 96-byte block once per iteration to decide whether to
// grow the sketch (the rare, variable-size branch).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dense.h"
#include "internal.h"
#include "loop.h"
#include "sketch.h"
#include "tc_gram.h"

// ============================================================================ handles

struct sks_sketch {
  sks_problem p;
  sks_kind kind;
  int64_t m = 0, m_max = 0, n_pad = 1;
  int s = 1, d = 0;
  uint64_t seed = 0;
  bool f32 = false;
  void* B = nullptr;  // SRHT: n_pad x d
  void* Y = nullptr;  // m_max x d, unscaled sketch
  long long ldy = 0;
  void* gbuf = nullptr;
  size_t gbuf_elems = 0;
  void* split = nullptr;
  size_t split_elems = 0;
  // float32 Gaussian sketch on the tensor cores: split A^T, column maxima, slice partials
  void* tch = nullptr;
  void* tcl = nullptr;
  float* tcpart = nullptr;
  size_t tcpart_elems = 0;
  bool tc_ready = false;
  // 8-bit Gaussian sketch: e4m3 operand A^T, its (slice, column) scales, the
  // column maxima scratch and ||A||_F^2
  unsigned char* a8 = nullptr;
  float* a8s = nullptr;
  unsigned* a8max = nullptr;
  double* frob2 = nullptr;
  bool a8_ready = false;
  uint32_t* sj = nullptr;  // SJLT buckets for the gathering kernel (larger m)
  size_t sj_elems = 0;
  sks::DevStatus* st = nullptr;
  double scale2() const { return kind == SKS_SJLT ? 1.0 : 1.0 / (double)m; }
};

struct sks_precond {
  int d = 0;
  int64_t m = 0;
  bool woodbury = false;
  double nu2 = 0, c2 = 0;
  const double* lam = nullptr;
  double* H = nullptr;   // d x d (or m x m) matrix being factored
  double* X = nullptr;   // inverse triangular factor
  double* Xt = nullptr;  // its transpose
  double* Y64 = nullptr; // float64 sketch (copy when the sketch is float32)
  long long ldy64 = 0;
  double* Yt = nullptr;  // d x m transpose of Y64 (Woodbury)
  double* Ys = nullptr;  // Y64 Lambda^{-1} (Woodbury build)
  double* chol_ws = nullptr;
  double* split = nullptr;
  size_t split_elems = 0;
  double* t1 = nullptr;  // m-vectors
  double* t2 = nullptr;
  __nv_bfloat16* bf[4] = {nullptr, nullptr, nullptr, nullptr};  // split-bf16 operands (float32 sketches)
  size_t bf_elems = 0;
  unsigned* rmax = nullptr;  // per-row maximum scratch of the split
  float* inv32 = nullptr;    // float32 inverse-factor scratch (float32 problems)
  sks::DevStatus* st = nullptr;
};

namespace sks {

sks_status validate_operator(const sks_problem* p) {
  if (!p) return fail(SKS_ERR_INVALID_ARG, "problem is NULL");
  if (p->n < 0 || p->d < 1 || p->k < 1) return fail(SKS_ERR_INVALID_ARG, "need n >= 0, d >= 1, k >= 1");
  if (p->lda < p->d) return fail(SKS_ERR_INVALID_ARG, "lda < d");
  if (p->n > 0 && !p->A) return fail(SKS_ERR_INVALID_ARG, "A is NULL");
  if (!p->lambda_diag) return fail(SKS_ERR_INVALID_ARG, "lambda is NULL");
  if (!(p->nu > 0.0) || !std::isfinite(p->nu)) return fail(SKS_ERR_INVALID_ARG, "nu must be > 0");
  if (p->dtype != SKS_F64 && p->dtype != SKS_F32) return fail(SKS_ERR_INVALID_ARG, "bad dtype");
  if (p->dtype == SKS_F32 && p->d > 16384) return fail(SKS_ERR_UNSUPPORTED, "d > 16384 (float32 A)");
  if (p->dtype == SKS_F64 && p->d > 14336) return fail(SKS_ERR_UNSUPPORTED, "d > 14336 (float64 A)");
  if (p->n > (int64_t)1 << 31) return fail(SKS_ERR_UNSUPPORTED, "n > 2^31");
  const size_t esz = p->dtype == SKS_F32 ? 4 : 8;
  if (p->n > 0 && (((uintptr_t)p->A & 15) || (p->lda * esz) % 16))
    return fail(SKS_ERR_INVALID_ARG, "A must be 16-byte aligned with lda * element size a multiple of 16");
  return SKS_OK;
}

sks_status validate_problem(const sks_problem* p) {
  SKS_TRY(validate_operator(p));
  if (!p->b) return fail(SKS_ERR_INVALID_ARG, "b is NULL");
  return SKS_OK;
}

sks_status read_status(DevStatus* st, cudaStream_t stream, const char* what) {
  DevStatus h;
  SKS_CUDA_TRY(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaStreamSynchronize(stream));
  if (h.code != 0) {
    std::string msg = std::string(what) + ": device status " + std::to_string(h.code) + " (site " +
                      std::to_string(h.where) + ", detail " + std::to_string(h.aux) + ")";
    if (h.code == SKS_ERR_INVALID_ARG && h.where == 1) msg = "lambda_i must be >= 1 (index " + std::to_string(h.aux) + ")";
    if (h.code == SKS_ERR_NOT_PD) msg = "non-positive pivot in Cholesky at column " + std::to_string(h.aux);
    if (h.code == SKS_ERR_TIMEOUT) msg = std::string(what) + ": bounded device wait ran out (site " + std::to_string(h.where) + ")";
    return fail((sks_status)h.code, msg);
  }
  return SKS_OK;
}

__global__ void f64_to_f32_kernel(long long count, const double* a, float* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void f32_to_f64_kernel(long long count, const float* a, double* b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

unsigned blocks_for(long long n, int t) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + t - 1) / t, 65535ll * 16));
}

namespace {

// ---------------------------------------------------------------- validation
__global__ void check_lambda_kernel(int d, const double* lam, DevStatus* st) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < d && !(lam[i] >= 1.0 && isfinite(lam[i]))) raise_status(st, SKS_ERR_INVALID_ARG, 1, i);
}


sks_status map_for(const sks_problem* p, CUtensorMap* map, const ApassPlan& pl) {
  const bool f32 = p->dtype == SKS_F32;
  return make_tmap_2d(map, p->A, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                      f32 ? 4 : 8, (uint64_t)p->n, (uint64_t)p->d, (uint64_t)p->lda, (uint32_t)pl.boxw,
                      (uint32_t)pl.rows_per_stage);
}

__global__ void f32_to_f64_2d_kernel(int rows, int cols, const float* a, long long lda, double* b, long long ldb) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  b[(long long)r * ldb + c] = (double)a[(long long)r * lda + c];
}
__global__ void scale_cols_kernel(int rows, int cols, const double* a, long long lda, const double* lam, double* b,
                                  long long ldb) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  b[(long long)r * ldb + c] = a[(long long)r * lda + c] / lam[c];
}
// Dual data matrix of eq. (2): D = Lambda^{-1/2} A^T (d x n row-major, ldd), by
// 32 x 32 shared-memory tiles (coalesced reads of A's rows and writes of D's rows).
template <typename T>
__global__ void dual_transpose_kernel(int64_t n, int d, const T* __restrict__ A, long long lda,
                                      const double* __restrict__ lam, T* __restrict__ D, long long ldd) {
  __shared__ T tile[32][33];
  const int64_t i0 = (int64_t)blockIdx.x * 32;
  const int j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t i = i0 + r;
    const int j = j0 + threadIdx.x;
    tile[r][threadIdx.x] = (i < n && j < d) ? A[i * lda + j] : T(0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int j = j0 + r;
    const int64_t i = i0 + threadIdx.x;
    if (j < d && i < n) D[(long long)j * ldd + i] = (T)((double)tile[threadIdx.x][r] / sqrt(lam[j]));
  }
}
__global__ void fill_kernel(int64_t count, double v, double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = v;
}
// primal solution from the dual one: x = Lambda^{-1} (b - A^T w) / nu^2, with
// t = D w = Lambda^{-1/2} A^T w, so (A^T w)_j = sqrt(lambda_j) t_j
__global__ void dual_recover_kernel(int d, const double* __restrict__ b, const double* __restrict__ t,
                                    const double* __restrict__ lam, double nu2, double* __restrict__ x) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) x[j] = (b[j] - sqrt(lam[j]) * t[j]) / (nu2 * lam[j]);
}
__global__ void scale_rows_out_kernel(int rows, int cols, const void* Y, int f32, long long ldy, double scale,
                                      double* out) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  const double v = f32 ? (double)((const float*)Y)[(long long)r * ldy + c] : ((const double*)Y)[(long long)r * ldy + c];
  out[e] = scale * v;
}


// ---------------------------------------------------------------- sketch
struct SketchSizes {
  size_t b_elems = 0, y_elems = 0, g_elems = 0, split_elems = 0;
  size_t sj_elems = 0;  // SJLT buckets (counts, offsets, entries) of the gathering kernel
  size_t tc_elems = 0, tcpart_elems = 0;  // float32 Gaussian (tensor cores)
  size_t a8_elems = 0, a8s_elems = 0;     // 8-bit Gaussian: d x Kp bytes, slices x d scales
};

SketchSizes sketch_sizes(const sks_problem* p, sks_kind kind, int64_t m_max, int sjlt_s) {
  SketchSizes z;
  if (kind == SKS_SJLT && p->dtype == SKS_F64) z.sj_elems = sjlt_gather_ws_elems(p->n, m_max, std::max(1, sjlt_s));
  if (kind == SKS_SJLT && p->dtype == SKS_F32) z.sj_elems = (sjlt_table_bytes(p->n) + 3) / 4 + 16;
  const int64_t n_pad = (int64_t)1 << ilog2_ceil(std::max<int64_t>(p->n, 1));
  if (kind == SKS_SRHT) z.b_elems = (size_t)n_pad * p->d;
  z.y_elems = (size_t)m_max * p->d;
  // S drawn entry by entry; the 8-bit kind keeps the bfloat16 operands too (the
  // solver falls back to them when the noise estimate rules 8 bits out)
  const bool dense_kind = kind == SKS_GAUSSIAN || kind == SKS_RADEMACHER || kind == SKS_GAUSSIAN_E4M3;
  if (dense_kind && p->dtype == SKS_F32) {
    z.tc_elems = (size_t)p->d * (size_t)tc_gauss_kp(p->n);
    z.tcpart_elems = tc_gauss_part_elems(p->n, (int)p->d, (int)std::min<int64_t>(m_max, 1 << 30));
    if (kind == SKS_GAUSSIAN_E4M3) {
      z.a8_elems = (size_t)p->d * (size_t)tc_gauss_kp(p->n);
      z.a8s_elems = (size_t)tc_gauss_slices(p->n) * (size_t)p->d;
    }
  } else if (dense_kind) {
    z.g_elems = (size_t)std::min<int64_t>((int64_t)m_max * std::max<int64_t>(p->n, 1), (int64_t)1 << 24);
    z.g_elems = std::max<size_t>(z.g_elems, (size_t)m_max * 64);
    z.split_elems = std::min<size_t>((size_t)8 * m_max * p->d, (size_t)1 << 24);
  }
  return z;
}

int64_t resolve_m_max(const sks_problem* p, sks_kind kind, int64_t m_max) {
  const int64_t n_pad = (int64_t)1 << ilog2_ceil(std::max<int64_t>(p->n, 1));
  const int64_t cap = kind == SKS_SRHT ? n_pad : std::max<int64_t>(p->n, 1);
  if (m_max <= 0) return cap;
  return std::min(m_max, cap);
}

size_t sketch_ws_bytes(const sks_problem* p, sks_kind kind, int64_t m_max, int sjlt_s) {
  const SketchSizes z = sketch_sizes(p, kind, m_max, sjlt_s);
  const size_t esz = p->dtype == SKS_F32 ? 4 : 8;
  Carver c(nullptr, 0);
  c.take<DevStatus>(1);
  c.take<char>(z.b_elems * esz);
  c.take<char>(z.y_elems * esz);
  c.take<__nv_bfloat16>(z.tc_elems);
  c.take<__nv_bfloat16>(z.tc_elems);
  c.take<float>(z.tcpart_elems);
  c.take<char>(z.g_elems * esz);
  c.take<char>(z.split_elems * esz);
  c.take<uint32_t>(z.sj_elems);
  c.take<unsigned char>(z.a8_elems);
  c.take<float>(z.a8s_elems);
  c.take<unsigned>(z.a8s_elems);
  c.take<double>(1);
  return c.used + 256;
}

sks_status sketch_init(sks_sketch* s, const sks_problem* p, sks_kind kind, int64_t m_max, int sjlt_s, uint64_t seed,
                       void* ws, size_t ws_bytes, DevStatus* shared_st) {
  s->p = *p;
  s->kind = kind;
  s->m = 0;
  s->m_max = m_max;
  s->s = std::max(1, sjlt_s);
  s->seed = seed;
  s->d = (int)p->d;
  s->f32 = p->dtype == SKS_F32;
  s->n_pad = (int64_t)1 << ilog2_ceil(std::max<int64_t>(p->n, 1));
  const SketchSizes z = sketch_sizes(p, kind, m_max, sjlt_s);
  const size_t esz = s->f32 ? 4 : 8;
  Carver c(ws, ws_bytes);
  DevStatus* own = c.take<DevStatus>(1);
  s->st = shared_st ? shared_st : own;
  s->B = c.take<char>(z.b_elems * esz);
  s->Y = c.take<char>(z.y_elems * esz);
  s->ldy = p->d;
  s->gbuf = c.take<char>(z.g_elems * esz);
  s->gbuf_elems = z.g_elems;
  s->split = c.take<char>(z.split_elems * esz);
  s->split_elems = z.split_elems;
  s->tch = c.take<__nv_bfloat16>(z.tc_elems);
  s->tcl = c.take<__nv_bfloat16>(z.tc_elems);
  s->tcpart = c.take<float>(z.tcpart_elems);
  s->tcpart_elems = z.tcpart_elems;
  s->sj = c.take<uint32_t>(z.sj_elems);
  s->sj_elems = z.sj_elems;
  s->a8 = c.take<unsigned char>(z.a8_elems);
  s->a8s = c.take<float>(z.a8s_elems);
  s->a8max = c.take<unsigned>(z.a8s_elems);
  s->frob2 = c.take<double>(1);
  s->a8_ready = false;
  s->tc_ready = false;
  if (!c.ok()) return fail(SKS_ERR_WORKSPACE, "sketch workspace too small");
  if (z.b_elems == 0) s->B = nullptr;
  return SKS_OK;
}

template <typename T>
sks_status sketch_to_t(sks_sketch* s, int64_t new_m, cudaStream_t stream) {
  const sks_problem& p = s->p;
  const T* A = (const T*)p.A;
  T* Y = (T*)s->Y;
  const int d = s->d;
  if (s->kind == SKS_SRHT) {
    if (s->m == 0) SKS_TRY(srht_form<T>(stream, A, p.lda, p.n, d, (T*)s->B, d, s->seed));
    SKS_TRY(srht_gather<T, T>(stream, (const T*)s->B, d, d, s->n_pad, s->seed, (int)s->m, (int)new_m, Y, s->ldy, s->st));
  } else if (s->kind == SKS_GAUSSIAN_E4M3) {
    if (!s->f32) return fail(SKS_ERR_UNSUPPORTED, "the 8-bit Gaussian sketch needs a float32 A");
    // e4m3(G) times e4m3(A / scale) on the tensor cores; the operand is made once per sketch
    if (!s->a8_ready) {
      SKS_TRY(tc_split8_t(stream, (const float*)A, p.lda, p.n, d, s->a8, s->a8s, s->a8max, s->frob2));
      s->a8_ready = true;
    }
    SKS_TRY(tc_gauss_sketch(stream, nullptr, nullptr, p.n, d, s->seed, (int)s->m, (int)(new_m - s->m), s->tcpart,
                            s->tcpart_elems, (float*)Y, s->ldy, s->st, false, s->a8, s->a8s));
  } else if ((s->kind == SKS_GAUSSIAN || s->kind == SKS_RADEMACHER) && s->f32) {
    // bf16(G) times the split A^T on the tensor cores; the split is made once per sketch
    if (!s->tc_ready) {
      SKS_TRY(tc_split_t(stream, (const float*)A, p.lda, p.n, d, (__nv_bfloat16*)s->tch, (__nv_bfloat16*)s->tcl));
      s->tc_ready = true;
    }
    SKS_TRY(tc_gauss_sketch(stream, (const __nv_bfloat16*)s->tch, (const __nv_bfloat16*)s->tcl, p.n, d, s->seed,
                            (int)s->m, (int)(new_m - s->m), s->tcpart, s->tcpart_elems, (float*)Y, s->ldy, s->st,
                            s->kind == SKS_RADEMACHER));
  } else if (s->kind == SKS_GAUSSIAN || s->kind == SKS_RADEMACHER) {
    SKS_TRY(gaussian_extend<T>(stream, A, p.lda, p.n, d, s->seed, (int)s->m, (int)(new_m - s->m), Y, s->ldy,
                               (T*)s->gbuf, s->gbuf_elems, (T*)s->split, s->split_elems, s->kind == SKS_RADEMACHER));
  } else {
    SKS_TRY(sjlt_form<T, T>(stream, A, p.lda, p.n, d, (int)new_m, s->s, s->seed, Y, s->ldy, s->sj, s->sj_elems,
                            s->st));
  }
  s->m = new_m;
  return SKS_OK;
}

sks_status sketch_to(sks_sketch* s, int64_t new_m, cudaStream_t stream) {
  if (new_m < s->m) return fail(SKS_ERR_INVALID_ARG, "sketch can only grow");
  if (new_m > s->m_max) return fail(SKS_ERR_INVALID_ARG, "sketch size above m_max");
  if (new_m == s->m) return SKS_OK;
  if (s->f32) return sketch_to_t<float>(s, new_m, stream);
  return sketch_to_t<double>(s, new_m, stream);
}

// ---------------------------------------------------------------- preconditioner
size_t precond_ws_bytes(const sks_problem* p, int64_t m_max) {
  const size_t d = (size_t)p->d;
  Carver c(nullptr, 0);
  c.take<DevStatus>(1);
  c.take<double>(d * d);  // H
  c.take<double>(d * d);  // X
  c.take<double>(d * d);  // Xt
  c.take<double>(d * d);  // Yt  (Woodbury only when m < d)
  c.take<double>(d * d);  // Ys
  if (p->dtype == SKS_F32) c.take<double>((size_t)m_max * d);  // Y64
  c.take<double>(cholesky_ws_elems((int)d));
  c.take<double>(std::min<size_t>(4 * d * d, (size_t)1 << 24));
  c.take<double>(std::max<size_t>(2 * d, (size_t)m_max));  // t1 (also 2 d column factors during a build)
  c.take<double>(std::max<size_t>(d, (size_t)m_max));      // t2
  if (p->dtype == SKS_F32) {
    const size_t e = std::max(tc_gram_split_elems((int)m_max, (int)d), tc_gram_split_elems((int)d, (int)m_max));
    for (int i = 0; i < 4; ++i) c.take<__nv_bfloat16>(e + 64);
    c.take<unsigned>(std::max<size_t>(d, (size_t)m_max));
    c.take<float>(cholesky_ws32_elems((int)d));
  }
  return c.used + 256;
}

sks_status precond_init(sks_precond* P, const sks_problem* p, int64_t m_max, void* ws, size_t ws_bytes,
                        DevStatus* shared_st, bool f32_inverse = false) {
  const size_t d = (size_t)p->d;
  Carver c(ws, ws_bytes);
  DevStatus* own = c.take<DevStatus>(1);
  P->st = shared_st ? shared_st : own;
  P->d = (int)d;
  P->H = c.take<double>(d * d);
  P->X = c.take<double>(d * d);
  P->Xt = c.take<double>(d * d);
  P->Yt = c.take<double>(d * d);
  P->Ys = c.take<double>(d * d);
  P->Y64 = p->dtype == SKS_F32 ? c.take<double>((size_t)m_max * d) : nullptr;
  P->chol_ws = c.take<double>(cholesky_ws_elems((int)d));
  P->split_elems = std::min<size_t>(4 * d * d, (size_t)1 << 24);
  P->split = c.take<double>(P->split_elems);
  P->t1 = c.take<double>(std::max<size_t>(2 * d, (size_t)m_max));
  P->t2 = c.take<double>(std::max<size_t>(d, (size_t)m_max));
  if (p->dtype == SKS_F32) {
    P->bf_elems = std::max(tc_gram_split_elems((int)m_max, (int)d), tc_gram_split_elems((int)d, (int)m_max));
    for (int i = 0; i < 4; ++i) P->bf[i] = c.take<__nv_bfloat16>(P->bf_elems + 64);
    P->rmax = c.take<unsigned>(std::max<size_t>(d, (size_t)m_max));
    float* w32 = c.take<float>(cholesky_ws32_elems((int)d));
    P->inv32 = f32_inverse ? w32 : nullptr;
  }
  if (!c.ok()) return fail(SKS_ERR_WORKSPACE, "preconditioner workspace too small");
  return SKS_OK;
}

// H_S = c2 Y^T Y + nu^2 Lambda (m >= d) or W_S = c2 Y Lambda^{-1} Y^T + nu^2 I (m < d).
sks_status precond_factor(sks_precond* P, const sks_sketch* s, double nu, const double* lam, cudaStream_t stream) {
  const int d = s->d;
  const int m = (int)s->m;
  P->m = m;
  P->woodbury = m < d;
  P->nu2 = nu * nu;
  P->c2 = s->scale2();
  P->lam = lam;
  const double* Y64;
  long long ldy;
  // Float32 sketches form the Gram matrix on the tensor cores from a
  // split-bfloat16 copy (tc_gram.cu); float64 sketches use float64 GEMMs.
  const bool tc = s->f32 && P->bf[0] != nullptr;
  if (s->f32 && !(tc && m < d)) {
    f32_to_f64_2d_kernel<<<blocks_for((long long)m * d), 256, 0, stream>>>(m, d, (const float*)s->Y, s->ldy, P->Y64, d);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  if (s->f32) {
    Y64 = P->Y64;
    ldy = d;
  } else {
    Y64 = (const double*)s->Y;
    ldy = s->ldy;
  }
  P->ldy64 = ldy;
  if (!P->woodbury) {
    if (tc) {
      int Kp = 0;
      SKS_TRY(tc_split(stream, (const float*)s->Y, s->ldy, m, d, true, nullptr, P->bf[0], P->bf[1], P->rmax, &Kp));
      SKS_TRY(tc_gram(stream, d, d, Kp, P->bf[0], P->bf[1], P->bf[0], P->bf[1], P->c2, 0.0, P->H, d, true, P->st));
    } else {
      SKS_TRY(gemm<double>(stream, d, d, m, Y64, ldy, true, Y64, ldy, false, P->H, d, P->c2, 0.0, true, 1, 0, 0, 0,
                           P->split, P->split_elems));
    }
    SKS_TRY(add_diagonal(stream, d, P->H, d, 0.0, lam, P->nu2));
    // Cholesky form: the apply is X^T X, positive definite for any nonsingular
    // X, so the mixed form (inv32 marks it) merges the inverse factor in
    // float32 after a double-float factorisation.
    SKS_TRY(cholesky_and_inverse(stream, d, P->H, d, P->X, d, P->chol_ws, P->st, P->inv32,
                                 P->inv32 != nullptr ? kCholDf32InvF32 : kCholF64));
    SKS_TRY(transpose<double>(stream, d, d, P->X, d, P->Xt, d));
  } else {
    if (tc) {
      // W = c^2 Z' Z'^T with Z' the split of Z = Y Lambda^{-1/2}; the apply then
      // uses Y_eff = Z' Lambda^{1/2}, so the preconditioner is exactly the
      // inverse of c^2 Y_eff^T Y_eff + nu^2 Lambda.
      int Kp = 0;
      // colfac: 1/sqrt(lambda) and sqrt(lambda) in the two apply vectors (free during a build)
      SKS_TRY(tc_split(stream, (const float*)s->Y, s->ldy, m, d, false, lam, P->bf[0], P->bf[1], P->rmax, &Kp,
                       P->t1));
      SKS_TRY(tc_gram(stream, m, m, Kp, P->bf[0], P->bf[1], P->bf[0], P->bf[1], P->c2, 0.0, P->H, m, true, P->st));
      SKS_TRY(tc_unsplit(stream, P->bf[0], P->bf[1], m, d, Kp, P->t1 + d, P->Y64, d));
    } else {
      scale_cols_kernel<<<blocks_for((long long)m * d), 256, 0, stream>>>(m, d, Y64, ldy, lam, P->Ys, d);
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
      SKS_TRY(gemm<double>(stream, m, m, d, P->Ys, d, false, Y64, ldy, true, P->H, m, P->c2, 0.0, true, 1, 0, 0, 0,
                           P->split, P->split_elems));
    }
    SKS_TRY(add_diagonal(stream, m, P->H, m, P->nu2, nullptr, 0.0));
    // Woodbury form: the apply subtracts two terms of size ~1/nu^2, so W^{-1}
    // must be accurate: float64, or double-float in the mixed form.
    SKS_TRY(cholesky_and_inverse(stream, m, P->H, m, P->X, m, P->chol_ws, P->st, P->inv32,
                                 P->inv32 != nullptr ? kCholDf32 : kCholF64));
    SKS_TRY(transpose<double>(stream, m, m, P->X, m, P->Xt, m));
    SKS_TRY(transpose<double>(stream, m, d, Y64, ldy, P->Yt, m));
  }
  // keep the float64 sketch pointer for the apply
  P->Y64 = const_cast<double*>(Y64);
  return SKS_OK;
}

// v = H_S^{-1} z (one column)
sks_status precond_apply1(const sks_precond* P, const double* z, double* v, cudaStream_t stream) {
  const int d = P->d;
  if (!P->woodbury) {
    SKS_TRY(gemv_rows<double>(stream, d, d, P->X, d, 1, z, nullptr, 1.0, P->t1, 0, nullptr, nullptr, 0.0));
    SKS_TRY(gemv_rows<double>(stream, d, d, P->Xt, d, 2, P->t1, nullptr, 1.0, v, 0, nullptr, nullptr, 0.0));
    return SKS_OK;
  }
  const int m = (int)P->m;
  const double c = std::sqrt(P->c2);
  SKS_TRY(gemv_rows<double>(stream, m, d, P->Y64, P->ldy64, 0, z, P->lam, c, P->t1, 0, nullptr, nullptr, 0.0));
  SKS_TRY(gemv_rows<double>(stream, m, m, P->X, m, 1, P->t1, nullptr, 1.0, P->t2, 0, nullptr, nullptr, 0.0));
  SKS_TRY(gemv_rows<double>(stream, m, m, P->Xt, m, 2, P->t2, nullptr, 1.0, P->t1, 0, nullptr, nullptr, 0.0));
  SKS_TRY(gemv_rows<double>(stream, d, m, P->Yt, m, 0, P->t1, nullptr, c, v, 1, z, P->lam, P->nu2));
  return SKS_OK;
}

// ---------------------------------------------------------------- iteration kernels
struct Ctl {
  double dt, dI, dp, alpha, ratio, thr, btx;
  double delta, delta0;  // trace mode: 1/2 ||x - x*||_H^2 now and at x_0
  long long t, I;
  int accept, stop, numeric, pad;
};

constexpr int kStepThreads = 1024;

__device__ double block_dot(int d, const double* a, const double* b) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s += a[j] * b[j];
  return block_sum(s, scratch);
}

// PCG, first half of a step: alpha = delta~_t / p^T H p, x+ = x + alpha p, r+ = r - alpha H p.
// *flag = 1 if any x[j] != 0 (one CTA)
__global__ void any_nonzero_kernel(int d, const double* __restrict__ x, int* flag) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  int mine = 0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) mine |= (x[j] != 0.0) ? 1 : 0;
  if (mine) any = 1;
  __syncthreads();
  if (threadIdx.x == 0) *flag = any;
}

__global__ void __launch_bounds__(kStepThreads) pcg_step1_kernel(int d, const double* x, const double* r,
                                                                 const double* p, const double* Hp, double* xp,
                                                                 double* rp, Ctl* ctl) {
  const double pHp = block_dot(d, p, Hp);
  const double alpha = ctl->dt / pHp;
  const bool bad = !(pHp > 0.0) || !isfinite(alpha);
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    xp[j] = x[j] + alpha * p[j];
    rp[j] = r[j] - alpha * Hp[j];
  }
  if (threadIdx.x == 0) {
    ctl->alpha = alpha;
    ctl->numeric = bad ? 1 : 0;
  }
}

// PCG, second half: delta~+ = r+^T r~+, the improvement test of Algorithm 2,
// and on acceptance p+ = r~+ + (delta~+/delta~_t) p and the state shift.
__global__ void __launch_bounds__(kStepThreads) pcg_step2_kernel(int d, const double* b, double* x, double* r,
                                                                 double* rt, double* p, const double* xp,
                                                                 const double* rp, const double* rtp, Ctl* ctl,
                                                                 double c, double phi, int can_double, double tol2,
                                                                 double stop_abs) {
  __shared__ int s_accept;
  const double dp = block_dot(d, rp, rtp);
  if (threadIdx.x == 0) {
    const long long t = ctl->t, I = ctl->I;
    const double thr = c * pow(phi, (double)(t + 1 - I));
    const double ratio = dp / ctl->dI;
    ctl->dp = dp;
    ctl->ratio = ratio;
    ctl->thr = thr;
    if (!isfinite(dp)) ctl->numeric = 1;
    const int reject = (ratio > thr) && can_double;
    s_accept = !reject;
    ctl->accept = s_accept;
    if (reject) ctl->I = t;
  }
  __syncthreads();
  if (!s_accept) return;
  const double beta = dp / ctl->dt;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    p[j] = rtp[j] + beta * p[j];
    x[j] = xp[j];
    r[j] = rp[j];
    rt[j] = rtp[j];
  }
  __syncthreads();
  const double btx = block_dot(d, b, x);
  if (threadIdx.x == 0) {
    ctl->dt = dp;
    ctl->t += 1;
    ctl->btx = btx;
    ctl->stop = (dp <= 0.0) || (dp <= tol2 * btx) || (dp <= stop_abs);
  }
}

// PCG restart at x_t with the current preconditioner: p = r~, delta~_t = delta~_I = r^T r~.
__global__ void __launch_bounds__(kStepThreads) pcg_restart_kernel(int d, const double* r, const double* rt,
                                                                   double* p, Ctl* ctl) {
  const double dt = block_dot(d, r, rt);
  for (int j = threadIdx.x; j < d; j += blockDim.x) p[j] = rt[j];
  if (threadIdx.x == 0) {
    ctl->dt = dt;
    ctl->dI = dt;
    ctl->accept = 1;
    ctl->stop = (dt <= 0.0);
    if (!isfinite(dt)) ctl->numeric = 1;
  }
}

// IHS proposal x+ = x - mu v (eq. 4); with xprev != NULL the Polyak-IHS
// (heavy-ball) proposal x+ = x - mu v + beta (x - x_prev) (Appendix A, eq. A.1).
__global__ void ihs_prop_kernel(int d, const double* x, const double* xprev, const double* v, double mu, double beta,
                                double* xp) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d) return;
  double y = x[j] - mu * v[j];
  if (xprev) y += beta * (x[j] - xprev[j]);
  xp[j] = y;
}

// IHS test: delta~+ = 1/2 g+^T v+, reject iff delta~+/delta~_I > c rho^(t+1-I).
// xprev != NULL (Polyak-IHS): the accepted step also shifts x_t into x_{t-1}.
__global__ void __launch_bounds__(kStepThreads) ihs_step2_kernel(int d, const double* b, double* x, double* g,
                                                                 double* v, const double* xp, const double* gp,
                                                                 const double* vp, Ctl* ctl, double c, double phi,
                                                                 int can_double, double tol2, double stop_abs,
                                                                 double* xprev) {
  __shared__ int s_accept;
  const double dp = 0.5 * block_dot(d, gp, vp);
  if (threadIdx.x == 0) {
    const long long t = ctl->t, I = ctl->I;
    const double thr = c * pow(phi, (double)(t + 1 - I));
    const double ratio = dp / ctl->dI;
    ctl->dp = dp;
    ctl->ratio = ratio;
    ctl->thr = thr;
    if (!isfinite(dp)) ctl->numeric = 1;
    const int reject = (ratio > thr) && can_double;
    s_accept = !reject;
    ctl->accept = s_accept;
    if (reject) ctl->I = t;
  }
  __syncthreads();
  if (!s_accept) return;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    if (xprev) xprev[j] = x[j];
    x[j] = xp[j];
    g[j] = gp[j];
    v[j] = vp[j];
  }
  __syncthreads();
  const double btx = block_dot(d, b, x);
  if (threadIdx.x == 0) {
    ctl->dt = dp;
    ctl->t += 1;
    ctl->btx = btx;
    ctl->stop = (dp <= 0.0) || (2.0 * dp <= tol2 * btx) || (dp <= stop_abs);
  }
}

// IHS restart: delta~_t = delta~_I = 1/2 g^T v with v = H_S^{-1} g.
__global__ void __launch_bounds__(kStepThreads) ihs_restart_kernel(int d, const double* g, const double* v, Ctl* ctl) {
  const double dt = 0.5 * block_dot(d, g, v);
  if (threadIdx.x == 0) {
    ctl->dt = dt;
    ctl->dI = dt;
    ctl->accept = 1;
    ctl->stop = (dt <= 0.0);
    if (!isfinite(dt)) ctl->numeric = 1;
  }
}

__global__ void ctl_init_kernel(Ctl* ctl) {
  memset(ctl, 0, sizeof(Ctl));
}

// Trace mode: delta = 1/2 ||x - x*||_H^2 = 1/2 sgn (x* - x)^T r, with r the
// residual b - H x (PCG, sgn = 1) or the gradient H x - b (IHS, sgn = -1);
// first: also delta0.
__global__ void __launch_bounds__(kStepThreads) delta_kernel(int d, const double* xs, const double* x,
                                                             const double* r, double sgn, Ctl* ctl, int first) {
  __shared__ double scratch[32];
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s += (xs[j] - x[j]) * r[j];
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) {
    ctl->delta = 0.5 * sgn * s;
    if (first) ctl->delta0 = ctl->delta;
  }
}

// Small vector kernels of the refinement loop.
__global__ void f64_to_f32_vec(int d, const double* a, float* b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) b[j] = (float)a[j];
}
__global__ void f32_to_f64_vec(int d, const float* a, double* b) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) b[j] = (double)a[j];
}
__global__ void axpy_kernel(int d, double a, const double* x, double* y) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < d) y[j] += a * x[j];
}
__global__ void __launch_bounds__(kStepThreads) dot_kernel(int d, const double* a, const double* b, double* out) {
  const double v = block_dot(d, a, b);
  if (threadIdx.x == 0) *out = v;
}

// ---------------------------------------------------------------- solve workspace
// Record left at the head of a solve workspace so that a later call on the
// same workspace (the adjoint solve) can reuse the sketch and preconditioner.
struct SolveState {
  uint64_t magic;
  int64_t n, d, m;
  int dtype, precision, kind, sjlt_s;
  uint64_t seed;
};
constexpr uint64_t kStateMagic = 0x736b73737461746full;

struct SolveWs {
  SolveState* state;
  DevStatus* st;
  Ctl* ctl;
  double* scal;  // [0] = b^T x of the outer iterate
  double *x, *r, *rt, *p, *Hp, *xp, *rp, *rtp;
  double *xo, *bo;  // refinement: outer iterate and the inner right-hand side
  float *p32, *h32;
  void* partials;    // A-pass partial sums in the iteration's precision
  void* partials64;  // float64-arithmetic A-pass (refinement residual)
  void* sketch_ws;
  size_t sketch_bytes;
  void* precond_ws;
  size_t precond_bytes;
  // device-resident loop (loop.cu): lw right-hand sides in lockstep (0: not available)
  int lw;
  long long lt_ld;                       // leading dimension of lt1, lt2
  double *lx, *lr, *lrt, *lp, *lHp, *lxp, *lrp, *lrtp, *lxo, *lbo, *lb, *lxs, *lt1, *lt2;
  float* lv32;
  void* lpart;      // loop A-pass partial sums
  void* lres;       // double-float residual partial sums (mixed form), lw columns
  double* ldots;
  LoopHead* lhead;  // followed by lw LoopCol
  LoopCol* lcols;
  LoopTraceEv* ltrace;
  int ltrace_cap;
};

// Lockstep width of the device-resident loop: 8 right-hand sides share each
// pass over A where the 8-column pass exists (d <= 1024), else one.
int loop_width(const sks_problem* p) { return (p->k > 1 && p->d <= 1024) ? 8 : 1; }

sks_status solve_layout(const sks_problem* p, const sks_opts* o, void* ws, size_t ws_bytes, SolveWs* L,
                        size_t* total) {
  const size_t d = (size_t)p->d;
  const int64_t m_max = resolve_m_max(p, o->kind, o->m_max);
  const bool f32 = p->dtype == SKS_F32;
  const bool mixed = o->precision == SKS_MIXED_REFINED;
  Carver c(ws, ws_bytes);
  SolveWs w;
  w.state = c.take<SolveState>(1);
  w.st = c.take<DevStatus>(1);
  w.ctl = c.take<Ctl>(1);
  w.scal = c.take<double>(4);
  w.x = c.take<double>(d);
  w.r = c.take<double>(d);
  w.rt = c.take<double>(d);
  w.p = c.take<double>(d);
  w.Hp = c.take<double>(d);
  w.xp = c.take<double>(d);
  w.rp = c.take<double>(d);
  w.rtp = c.take<double>(d);
  w.xo = c.take<double>(d);
  w.bo = c.take<double>(d);
  w.p32 = c.take<float>(d);
  w.h32 = c.take<float>(d);
  const int64_t n1 = std::max<int64_t>(p->n, 1);
  w.partials = c.take<char>(apass_workspace_bytes(n1, p->d, 1, f32, mixed));
  w.partials64 = c.take<char>(mixed ? apass_workspace_bytes(n1, p->d, 1, f32, false) : 0);
  w.sketch_bytes = sketch_ws_bytes(p, o->kind, m_max, o->sjlt_s);
  w.sketch_ws = c.take<char>(w.sketch_bytes);
  w.precond_bytes = precond_ws_bytes(p, m_max);
  w.precond_ws = c.take<char>(w.precond_bytes);
  w.lw = 0;
  ApassPlan lpl;
  if (p->d <= 4096 && apass_plan(n1, p->d, loop_width(p), f32, mixed, &lpl) == SKS_OK) {
    const int lw = loop_width(p);
    w.lw = lw;
    const size_t dk = d * (size_t)lw;
    w.lt_ld = (long long)std::max<size_t>(d, (size_t)m_max);
    double** vecs[] = {&w.lx, &w.lr, &w.lrt, &w.lp, &w.lHp, &w.lxp, &w.lrp, &w.lrtp, &w.lxo, &w.lbo, &w.lb, &w.lxs};
    for (double** v : vecs) *v = c.take<double>(dk);
    w.lt1 = c.take<double>((size_t)w.lt_ld * lw);
    w.lt2 = c.take<double>((size_t)w.lt_ld * lw);
    w.lv32 = c.take<float>(dk);
    w.lpart = c.take<char>(loop_partial_bytes(lpl, p->d, lw, mixed));
    w.lres = c.take<char>(mixed ? apass_workspace_bytes(n1, p->d, lw, f32, false) : 0);
    w.ldots = (double*)c.take<char>(loop_dots_bytes(lpl, lw));
    w.lhead = (LoopHead*)c.take<char>(sizeof(LoopHead) + lw * sizeof(LoopCol));
    w.lcols = w.lhead ? (LoopCol*)(w.lhead + 1) : nullptr;
    w.ltrace_cap = (o->trace && o->trace_cap > 0) ? (int)std::min<int64_t>(o->trace_cap, 1 << 16) : 0;
    w.ltrace = c.take<LoopTraceEv>((size_t)w.ltrace_cap);
  }
  if (total) *total = c.used + 256;
  if (L) *L = w;
  if (ws && !c.ok()) return fail(SKS_ERR_WORKSPACE, "solve workspace too small");
  return SKS_OK;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t s;
  float acc = 0.f;
  explicit Timer(cudaStream_t st) : s(st) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
  }
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
  void start() { cudaEventRecord(a, s); }
  void stop() {
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    acc += ms;
  }
};

// PCG: eq. (5); IHS: eq. (4) with mu = 1 - rho (Theorem 3.2); POLYAK: the
// heavy-ball IHS of Appendix A with mu_rho, beta_rho (Corollary A.2); CG: the
// unpreconditioned conjugate gradient baseline of Section 6 (PCG with H_S = I).
enum Method { PCG, IHS, POLYAK, CG };

// One adaptive solve engine shared by the plain float64 form and the inner
// solves of the mixed form.  The iteration A-pass runs in the precision of A
// (float64 A: float64; float32 A: float32 with the d-vectors converted on the
// fly); the d-vector algebra of Algorithms 1 and 2 stays in float64.
struct Engine {
  Method method;
  const sks_problem* prob;
  const sks_opts* o;
  cudaStream_t stream;
  SolveWs W;
  int d;
  int64_t m = 0, m_max = 0;
  double nu2 = 0, phi = 0, c = 0;
  bool f32 = false, mixed = false;
  ApassPlan plan, plan64;
  CUtensorMap tmap, tmap64;
  sks_sketch sk;
  sks_precond P;
  sks_stats S;
  cudaEvent_t ev_a0 = nullptr, ev_a1 = nullptr;
  bool apass_pending = false;
  Timer *t_sketch = nullptr, *t_factor = nullptr;
  int outer = 0;
  bool fixed = false;         // non-adaptive: m stays at m_init, every step is accepted
  bool fused = false;         // the device-resident loop (loop.cu) serves this solve
  int cur_col = 0;            // right-hand side being solved (host-driven iteration)
  ApassPlan lplan, lresplan;  // its A-pass plan (lw columns) and the refinement residual's
  CUtensorMap ltmap, lrtmap;
  double mu = 0, beta = 0;    // IHS / Polyak-IHS step size and momentum
  double cg_bb = 0;           // b^T b of the current right-hand side (CG stop rule)

  ~Engine() {
    if (ev_a0) cudaEventDestroy(ev_a0);
    if (ev_a1) cudaEventDestroy(ev_a1);
  }

  sks_status init(Method mth, const sks_problem* pr, const sks_opts* op, void* ws, size_t ws_bytes,
                  cudaStream_t st) {
    method = mth;
    prob = pr;
    o = op;
    stream = st;
    d = (int)pr->d;
    f32 = pr->dtype == SKS_F32;
    mixed = op->precision == SKS_MIXED_REFINED;
    std::memset(&S, 0, sizeof(S));
    SKS_TRY(solve_layout(pr, op, ws, ws_bytes, &W, nullptr));
    m_max = resolve_m_max(pr, op->kind, op->m_max);
    nu2 = pr->nu * pr->nu;
    const double rho = op->rho;
    if (method == PCG || method == CG) {
      phi = (1.0 - std::sqrt(1.0 - rho)) / (1.0 + std::sqrt(1.0 - rho));
      c = 4.0 * (1.0 + std::sqrt(rho)) / (1.0 - std::sqrt(rho));
    } else {
      phi = rho;
      c = (1.0 + std::sqrt(rho)) / (1.0 - std::sqrt(rho));
    }
    mu = 1.0 - rho;
    beta = 0.0;
    if (method == POLYAK) {
      const double s1 = std::sqrt(1.0 - rho);
      mu = 2.0 * (1.0 - rho) / (1.0 + s1);
      beta = (1.0 - s1) / (1.0 + s1);
    }
    SKS_CUDA_TRY(cudaEventCreate(&ev_a0));
    SKS_CUDA_TRY(cudaEventCreate(&ev_a1));
    const int64_t n1 = std::max<int64_t>(pr->n, 1);
    SKS_TRY(apass_plan(n1, d, 1, f32, mixed, &plan));
    if (pr->n > 0) SKS_TRY(map_for(pr, &tmap, plan));
    apass_use_bulk(&plan, pr->A, d, pr->lda, f32);
    if (mixed) {
      SKS_TRY(apass_plan(n1, d, 1, f32, false, &plan64));
      if (pr->n > 0) SKS_TRY(map_for(pr, &tmap64, plan64));
      apass_use_bulk(&plan64, pr->A, d, pr->lda, f32);
    }
    if (W.lw > 0 && (method == PCG || method == IHS)) {
      // the device-resident loop: same pass geometry, lw columns, a stage less if needed
      if (apass_plan(n1, d, W.lw, f32, mixed, &lplan) == SKS_OK) {
        loop_adjust_plan(&lplan, f32, mixed);
        if (pr->n > 0) SKS_TRY(map_for(pr, &ltmap, lplan));
        apass_use_bulk(&lplan, pr->A, d, pr->lda, f32);
        fused = pr->n > 0 && loop_supported(lplan, d, W.lw, f32, mixed) == SKS_OK;
        if (fused && mixed) {
          SKS_TRY(apass_plan(n1, d, W.lw, f32, false, &lresplan));
          if (pr->n > 0) SKS_TRY(map_for(pr, &lrtmap, lresplan));
          apass_use_bulk(&lresplan, pr->A, d, pr->lda, f32);
        }
      }
      set_last_error("");  // an unavailable loop falls back to the host-driven iteration silently
    }
    SKS_TRY(sketch_init(&sk, pr, op->kind, m_max, op->sjlt_s, op->seed, W.sketch_ws, W.sketch_bytes, W.st));
    // the mixed form forms the inverse Cholesky factor in float32
    SKS_TRY(precond_init(&P, pr, m_max, W.precond_ws, W.precond_bytes, W.st, mixed));
    return SKS_OK;
  }

  // Re-attach the sketch (m rows) and the factored preconditioner that a
  // previous solve left in this workspace.
  void restore(int64_t m_prev) {
    m = m_prev;
    sk.m = m_prev;
    P.m = m_prev;
    P.woodbury = m_prev < d;
    P.nu2 = nu2;
    P.c2 = sk.scale2();
    P.lam = prob->lambda_diag;
    if (sk.f32) {
      P.ldy64 = d;
    } else {
      P.Y64 = (double*)sk.Y;
      P.ldy64 = sk.ldy;
    }
  }

  // y = sgn * H x + addc * addv in the iteration's precision (one pass over A).
  sks_status hess(const double* x, double* y, double sgn, const double* addv, double addc) {
    S.a_passes += 1;
    apass_pending = true;
    if (!mixed)
      return apass_launch(plan, &tmap, prob->n, d, 1, f32, false, x, y, nu2, prob->lambda_diag, W.partials, W.st,
                          stream, sgn, addv, addc, ev_a0, ev_a1);
    f64_to_f32_vec<<<(d + 255) / 256, 256, 0, stream>>>(d, x, W.p32);
    note_launch();
    SKS_TRY(apass_launch(plan, &tmap, prob->n, d, 1, true, true, W.p32, W.h32, nu2, prob->lambda_diag, W.partials,
                         W.st, stream, 1.0, nullptr, 0.0, ev_a0, ev_a1));
    f32_to_f64_vec<<<(d + 255) / 256, 256, 0, stream>>>(d, W.h32, y);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    if (addv || sgn != 1.0) {
      // y = sgn * y + addc * addv  (rare: restarts only)
      return fail(SKS_ERR_UNSUPPORTED, "internal: mixed inner residual form");
    }
    return SKS_OK;
  }

  // float64-arithmetic pass over A (refinement residual): y = sgn H x + addc addv
  sks_status hess64(const double* x, double* y, double sgn, const double* addv, double addc) {
    S.a_passes += 1;
    return apass_launch(plan64, &tmap64, prob->n, d, 1, f32, false, x, y, nu2, prob->lambda_diag, W.partials64, W.st,
                        stream, sgn, addv, addc);
  }

  // v = H_S^{-1} z; the unpreconditioned CG takes H_S = I.
  sks_status apply(const double* z, double* v) {
    if (method == CG) {
      SKS_CUDA_TRY(cudaMemcpyAsync(v, z, (size_t)d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      return SKS_OK;
    }
    return precond_apply1(&P, z, v, stream);
  }

  sks_status sync_point(const char* what) {
    SKS_TRY(read_status(W.st, stream, what));
    if (apass_pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev_a0, ev_a1) == cudaSuccess) {
        S.ms_apass += ms;
        S.apass_timed += 1;
      }
      apass_pending = false;
    }
    return SKS_OK;
  }

  sks_status first_sketch() {
    if (method == CG) {  // no sketch, no preconditioner
      m = 0;
      return SKS_OK;
    }
    m = std::min<int64_t>(o->m_init, m_max);
    t_sketch->start();
    if (sk.kind == SKS_GAUSSIAN_E4M3) {
      // 8 bits only when the rounding noise of A stays well under the
      // regulariser: (2^-4)^2 / 3 ||A||_F^2 / d <= 0.1 nu^2 min lambda (the
      // e4m3 rounding of each entry is up to 2^-4 relative, the noise spreads
      // over the d directions); else the bfloat16 split serves the same G
      SKS_TRY(tc_split8_t(stream, (const float*)prob->A, prob->lda, prob->n, d, sk.a8, sk.a8s, sk.a8max, sk.frob2));
      sk.a8_ready = true;
      double frob2 = 0.0;
      std::vector<double> lam((size_t)d);
      SKS_CUDA_TRY(cudaMemcpyAsync(&frob2, sk.frob2, sizeof(double), cudaMemcpyDeviceToHost, stream));
      SKS_CUDA_TRY(cudaMemcpyAsync(lam.data(), prob->lambda_diag, (size_t)d * sizeof(double), cudaMemcpyDeviceToHost,
                                   stream));
      SKS_CUDA_TRY(cudaStreamSynchronize(stream));
      const double lam_min = *std::min_element(lam.begin(), lam.end());
      const double noise = std::ldexp(1.0, -8) / 3.0 * frob2 / (double)d;
      S.sketch_e4m3 = noise <= 0.1 * nu2 * lam_min ? 1 : 0;
      if (!S.sketch_e4m3) sk.kind = SKS_GAUSSIAN;
    }
    SKS_TRY(sketch_to(&sk, m, stream));
    t_sketch->stop();
    S.sketch_passes = 1;
    t_factor->start();
    SKS_TRY(precond_factor(&P, &sk, prob->nu, prob->lambda_diag, stream));
    t_factor->stop();
    S.factorizations = 1;
    return read_status(W.st, stream, "first preconditioner");
  }

  sks_status grow() {
    m = std::min<int64_t>(2 * m, m_max);
    t_sketch->start();
    SKS_TRY(sketch_to(&sk, m, stream));
    t_sketch->stop();
    S.sketch_passes += 1;
    t_factor->start();
    SKS_TRY(precond_factor(&P, &sk, prob->nu, prob->lambda_diag, stream));
    t_factor->stop();
    S.factorizations += 1;
    return SKS_OK;
  }

  // Adaptive solve of H x = b (Algorithm 2 or Algorithm 1) from the x already
  // in W.x.  Stops when delta~ <= tol2 * b^T x (tol2 > 0) or delta~ <=
  // rel2 * delta~_0 (rel2 > 0).  On return W.x holds the last accepted iterate;
  // *dt0 receives the decrement at the start, *h the final control block.
  sks_status inner(const double* b, double tol2, double rel2, int64_t max_iter, bool* converged, double* dt0,
                   Ctl* hout, const double* btx_dev = nullptr, double outer_tol2 = 0.0, double fac = 1.0,
                   bool* outer_done = nullptr) {
    ctl_init_kernel<<<1, 1, 0, stream>>>(W.ctl);
    note_launch();
    const bool mixed_inner = mixed;
    const bool pcg_like = method == PCG || method == CG;
    double* xprev = method == POLYAK ? W.p : nullptr;  // x_{t-1} of the heavy-ball step (p is unused by IHS)
    // PCG: r = b - H x, r~ = H_S^{-1} r.   IHS: g = H x - b (in r), v = H_S^{-1} g (in rt).
    if (mixed_inner) {
      // the inner right-hand side is the refinement residual and x starts at 0
      SKS_CUDA_TRY(cudaMemsetAsync(W.x, 0, d * sizeof(double), stream));
      if (pcg_like) SKS_CUDA_TRY(cudaMemcpyAsync(W.r, b, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      else {
        SKS_CUDA_TRY(cudaMemsetAsync(W.r, 0, d * sizeof(double), stream));
        axpy_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, -1.0, b, W.r);
        note_launch();
      }
    } else {
      if (pcg_like) SKS_TRY(hess(W.x, W.r, -1.0, b, 1.0));
      else SKS_TRY(hess(W.x, W.r, 1.0, b, -1.0));
    }
    SKS_TRY(apply(W.r, W.rt));
    if (pcg_like) pcg_restart_kernel<<<1, kStepThreads, 0, stream>>>(d, W.r, W.rt, W.p, W.ctl);
    else ihs_restart_kernel<<<1, kStepThreads, 0, stream>>>(d, W.r, W.rt, W.ctl);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    if (xprev) SKS_CUDA_TRY(cudaMemcpyAsync(xprev, W.x, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
    const double* xstar = (o->x_star && !mixed_inner) ? o->x_star + (size_t)cur_col * d : nullptr;
    if (xstar) {
      delta_kernel<<<1, kStepThreads, 0, stream>>>(d, xstar, W.x, W.r, pcg_like ? 1.0 : -1.0, W.ctl, 1);
      note_launch();
    }
    if (method == CG) {
      // CG stop rule: ||r||_2 <= tol ||b||_2 (no preconditioner, so no estimate of the H-norm error)
      dot_kernel<<<1, kStepThreads, 0, stream>>>(d, b, b, W.scal + 2);
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
      SKS_CUDA_TRY(cudaMemcpyAsync(&cg_bb, W.scal + 2, sizeof(double), cudaMemcpyDeviceToHost, stream));
    }
    Ctl h;
    SKS_CUDA_TRY(cudaMemcpyAsync(&h, W.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
    SKS_TRY(sync_point("initial residual"));
    if (h.numeric) return fail(SKS_ERR_NUMERIC, "non-finite initial decrement");
    *dt0 = h.dt;
    if (btx_dev && outer_done) {
      // refinement: the decrement of the residual at the outer iterate
      // estimates its error; stop before iterating when it meets the target.
      double btx = 0.0;
      SKS_CUDA_TRY(cudaMemcpy(&btx, btx_dev, sizeof(double), cudaMemcpyDeviceToHost));
      const double est2 = btx > 0 ? fac * h.dt / btx : (h.dt <= 0 ? 0.0 : 1.0);
      S.est_rel_err = std::sqrt(std::max(0.0, est2));
      if (est2 <= outer_tol2 || h.dt <= 0) {
        *outer_done = true;
        *converged = true;
        if (hout) *hout = h;
        return SKS_OK;
      }
    }
    double stop_abs = rel2 > 0 ? rel2 * h.dt : 0.0;
    if (method == CG) {
      stop_abs = std::max(stop_abs, o->tol * o->tol * cg_bb);
      tol2 = 0.0;
    }
    bool conv = h.stop != 0 || (stop_abs > 0 && h.dt <= stop_abs);
    if (hout) *hout = h;
    if (rel2 > 0 && *dt0 <= 0) conv = true;
    int64_t guard = 0;
    while (!conv && h.t < max_iter && guard++ < max_iter + 64) {
      const int can_double = (!fixed && m < m_max) ? 1 : 0;
      if (pcg_like) {
        SKS_TRY(hess(W.p, W.Hp, 1.0, nullptr, 0.0));
        pcg_step1_kernel<<<1, kStepThreads, 0, stream>>>(d, W.x, W.r, W.p, W.Hp, W.xp, W.rp, W.ctl);
        note_launch();
        SKS_CUDA_TRY(cudaGetLastError());
        SKS_TRY(apply(W.rp, W.rtp));
        pcg_step2_kernel<<<1, kStepThreads, 0, stream>>>(d, b, W.x, W.r, W.rt, W.p, W.xp, W.rp, W.rtp, W.ctl, c, phi,
                                                         can_double, tol2, stop_abs);
        note_launch();
      } else {
        ihs_prop_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, W.x, xprev, W.rt, mu, beta, W.xp);
        note_launch();
        if (mixed_inner) {
          SKS_TRY(hess(W.xp, W.rp, 1.0, nullptr, 0.0));
          axpy_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, -1.0, b, W.rp);
          note_launch();
        } else {
          SKS_TRY(hess(W.xp, W.rp, 1.0, b, -1.0));
        }
        SKS_TRY(apply(W.rp, W.rtp));
        ihs_step2_kernel<<<1, kStepThreads, 0, stream>>>(d, b, W.x, W.r, W.rt, W.xp, W.rp, W.rtp, W.ctl, c, phi,
                                                         can_double, tol2, stop_abs, xprev);
        note_launch();
      }
      SKS_CUDA_TRY(cudaGetLastError());
      if (xstar) {
        delta_kernel<<<1, kStepThreads, 0, stream>>>(d, xstar, W.x, W.r, pcg_like ? 1.0 : -1.0, W.ctl, 0);
        note_launch();
      }
      const long long t_before = h.t;
      SKS_CUDA_TRY(cudaMemcpyAsync(&h, W.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
      SKS_TRY(sync_point("iteration"));
      if (o->trace && S.trace_len < o->trace_cap) {
        sks_trace_event& e = o->trace[S.trace_len++];
        e.t = t_before;
        e.m = m;
        e.ratio = h.ratio;
        e.threshold = h.thr;
        e.accepted = h.accept;
        e.outer = outer;
        e.column = cur_col;
        e.reserved = 0;
        e.delta = h.delta;
        e.delta0 = h.delta0;
      }
      if (h.numeric) return fail(SKS_ERR_NUMERIC, "non-finite value in the iteration");
      if (!h.accept) {
        S.rejections += 1;
        SKS_TRY(grow());
        if (pcg_like) {
          if (!o->reuse_residual && !mixed_inner) SKS_TRY(hess(W.x, W.r, -1.0, b, 1.0));
          SKS_TRY(apply(W.r, W.rt));
          pcg_restart_kernel<<<1, kStepThreads, 0, stream>>>(d, W.r, W.rt, W.p, W.ctl);
        } else {
          SKS_TRY(apply(W.r, W.rt));
          ihs_restart_kernel<<<1, kStepThreads, 0, stream>>>(d, W.r, W.rt, W.ctl);
        }
        note_launch();
        SKS_CUDA_TRY(cudaGetLastError());
        SKS_CUDA_TRY(cudaMemcpyAsync(&h, W.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, stream));
        SKS_TRY(sync_point("restart"));
        if (h.numeric) return fail(SKS_ERR_NUMERIC, "non-finite decrement at restart");
        conv = h.stop != 0 || (stop_abs > 0 && h.dt <= stop_abs);
        continue;
      }
      conv = h.stop != 0;
    }
    S.iters += h.t;
    S.final_delta_tilde = h.dt;
    *converged = conv;
    if (hout) *hout = h;
    return SKS_OK;
  }
};

sks_status check_opts(const sks_problem* prob, const sks_opts* o, const double* x_io) {
  SKS_TRY(validate_problem(prob));
  if (!o) return fail(SKS_ERR_INVALID_ARG, "opts is NULL");
  if (!x_io) return fail(SKS_ERR_INVALID_ARG, "x is NULL");
  if (!(o->rho > 0.0 && o->rho < 1.0)) return fail(SKS_ERR_INVALID_ARG, "rho must be in (0, 1)");
  if (o->m_init < 1) return fail(SKS_ERR_INVALID_ARG, "m_init must be >= 1");
  if (!(o->tol > 0.0)) return fail(SKS_ERR_INVALID_ARG, "tol must be > 0");
  if (o->kind != SKS_SRHT && o->kind != SKS_GAUSSIAN && o->kind != SKS_SJLT && o->kind != SKS_RADEMACHER &&
      o->kind != SKS_GAUSSIAN_E4M3)
    return fail(SKS_ERR_INVALID_ARG, "bad embedding kind");
  if (o->kind == SKS_GAUSSIAN_E4M3 && prob->dtype != SKS_F32)
    return fail(SKS_ERR_UNSUPPORTED, "the 8-bit Gaussian sketch needs a float32 A (mixed form)");
  if (o->sjlt_s < 1 || o->sjlt_s > kSjltMaxS) return fail(SKS_ERR_INVALID_ARG, "sjlt_s must be in [1, 16]");
  if (o->precision == SKS_PLAIN_F64 && prob->dtype != SKS_F64)
    return fail(SKS_ERR_INVALID_ARG, "the plain float64 form needs a float64 A");
  if (o->precision == SKS_MIXED_REFINED && prob->dtype != SKS_F32)
    return fail(SKS_ERR_INVALID_ARG, "the mixed form needs a float32 A");
  if (o->precision == SKS_MIXED_REFINED && (o->max_outer < 1 || !(o->inner_tol > 0.0 && o->inner_tol < 1.0)))
    return fail(SKS_ERR_INVALID_ARG, "mixed form needs max_outer >= 1 and inner_tol in (0, 1)");
  if (o->stop_rule != SKS_STOP_ESTIMATE && o->stop_rule != SKS_STOP_CERTIFIED)
    return fail(SKS_ERR_INVALID_ARG, "bad stop rule");
  if (o->stop_rule == SKS_STOP_CERTIFIED &&
      (!(o->cert_delta > 0.0 && o->cert_delta < 1.0) || !(o->cert_de >= 0.0) || !std::isfinite(o->cert_de)))
    return fail(SKS_ERR_INVALID_ARG, "certified stop rule needs cert_delta in (0, 1) and cert_de >= 0");
  return SKS_OK;
}

// Critical sketch size m_delta of the embedding (Theorem 5.1 for the SRHT;
// Theorem 5.2 with omega(C)^2 <= d_e for the Gaussian and sub-Gaussian
// embeddings; the order d_e^2/delta of Table 1, constant 1, for the SJLT).
double critical_sketch_size(sks_kind kind, int64_t n, double d_e, double delta) {
  switch (kind) {
    case SKS_SRHT: {
      const double a = std::sqrt(d_e) + std::sqrt(8.0 * std::log(2.0 * (double)n / delta));
      return 16.0 * std::log(16.0 * d_e / delta) * a * a;
    }
    case SKS_SJLT:
      return d_e * d_e / delta;
    default: {
      const double a = std::sqrt(d_e) + std::sqrt(8.0 * std::log(16.0 / delta));
      return a * a;
    }
  }
}

// Coefficient tol2 of the stop tests "PCG: delta~ <= tol2 b^T x" and "IHS:
// 2 delta~ <= tol2 b^T x": (tol/2)^2 for the estimate rule; tol^2/(m_delta+1)
// for Remark 4.2 (delta~_t <= eps/(m_delta+1) with eps = 1/2 tol^2 b^T x_t; the
// PCG decrement of Algorithm 2 carries no 1/2).
double stop_coefficient(const sks_problem* p, const sks_opts* o) {
  if (o->stop_rule != SKS_STOP_CERTIFIED) return (o->tol / 2.0) * (o->tol / 2.0);
  const double d_e = o->cert_de > 0.0 ? o->cert_de : (double)p->d;
  return o->tol * o->tol / (critical_sketch_size(o->kind, std::max<int64_t>(p->n, 1), d_e, o->cert_delta) + 1.0);
}

// ---------------------------------------------------------------- device-resident solve
// Refinement step of the mixed form, per column c < kc: b^T x_o into the
// column's state, reset of the inner solve (t = I = 0), x = 0 and the inner
// right-hand side (r = b_o for PCG, the gradient g = -b_o for the IHS).
__global__ void __launch_bounds__(1024) loop_prep_kernel(int d, int kc, int pcg, const double* __restrict__ b,
                                                         const double* __restrict__ xo, const double* __restrict__ bo,
                                                         double* __restrict__ x, double* __restrict__ r,
                                                         LoopCol* cols) {
  __shared__ double scratch[32];
  const int c = blockIdx.x;
  if (c >= kc) return;
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const size_t e = (size_t)c * d + j;
    s += b[e] * xo[e];
    x[e] = 0.0;
    r[e] = pcg ? bo[e] : -bo[e];
  }
  s = block_sum(s, scratch);
  if (threadIdx.x == 0) {
    LoopCol& q = cols[c];
    q.btx_outer = s;
    q.t = 0;
    q.I = 0;
    q.numeric = 0;
    q.rejected = 0;
    q.stop = (!q.active || q.outer_done) ? 1 : 0;
  }
}

// x_o += x for the columns whose refinement goes on.
__global__ void loop_outer_add_kernel(int d, int kc, const LoopCol* cols, const double* __restrict__ x,
                                      double* __restrict__ xo) {
  const int c = blockIdx.y;
  if (c >= kc || !cols[c].active || cols[c].outer_done) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < d; j += gridDim.x * blockDim.x)
    xo[(size_t)c * d + j] += x[(size_t)c * d + j];
}

struct LoopHostCtl {
  LoopHead head;
  LoopCol cols[kLoopMaxK];
};

// Launches the loop until no column asks for a larger sketch: after a failed
// test the host grows the sketch, refactors H_S and relaunches with the restart
// prologue (every column restarts at its current iterate with the new
// preconditioner; see reading R17).  Reads the control block once per launch.
sks_status loop_run(Engine& E, LoopTask& T, LoopHostCtl* h) {
  const int lw = E.W.lw;
  const size_t ctl_bytes = sizeof(LoopHead) + lw * sizeof(LoopCol);
  while (true) {
    SKS_CUDA_TRY(cudaMemsetAsync(E.W.lhead, 0, sizeof(LoopHead), E.stream));
    T.m = E.m;
    T.can_double = (!E.fixed && E.m < E.m_max) ? 1 : 0;
    T.P.woodbury = E.P.woodbury ? 1 : 0;
    T.P.m = (int)E.P.m;
    T.P.X = E.P.X;
    T.P.Xt = E.P.Xt;
    T.P.Y = E.P.Y64;
    T.P.ldy = E.P.ldy64;
    T.P.Yt = E.P.Yt;
    T.P.c = std::sqrt(E.P.c2);
    SKS_TRY(loop_launch(E.lplan, &E.ltmap, E.prob->n, E.d, E.f32, E.mixed, T, E.stream));
    SKS_CUDA_TRY(cudaMemcpyAsync(h, E.W.lhead, ctl_bytes, cudaMemcpyDeviceToHost, E.stream));
    SKS_TRY(read_status(E.W.st, E.stream, "solver loop"));
    E.S.a_passes += h->head.apasses;
    E.S.ms_apass += (float)(h->head.apass_ns * 1e-6);
    E.S.apass_timed += h->head.apasses;
    if (E.o->trace && h->head.trace_len > 0) {
      std::vector<LoopTraceEv> ev((size_t)h->head.trace_len);
      SKS_CUDA_TRY(cudaMemcpy(ev.data(), E.W.ltrace, ev.size() * sizeof(LoopTraceEv), cudaMemcpyDeviceToHost));
      for (const LoopTraceEv& v : ev) {
        if (E.S.trace_len >= E.o->trace_cap) break;
        sks_trace_event& e = E.o->trace[E.S.trace_len++];
        e.t = v.t;
        e.m = v.m;
        e.ratio = v.ratio;
        e.threshold = v.thr;
        e.accepted = v.accepted;
        e.outer = E.outer;
        e.column = v.column + E.cur_col;
        e.reserved = 0;
        e.delta = v.delta;
        e.delta0 = v.delta0;
      }
    }
    for (int c = 0; c < T.kc; ++c)
      if (h->cols[c].numeric) return fail(SKS_ERR_NUMERIC, "non-finite value in the iteration");
    if (!h->head.any_reject) return SKS_OK;
    E.S.rejections += 1;
    SKS_TRY(E.grow());
    T.resid = (T.method == 0 && !E.o->reuse_residual && !E.mixed) ? 1 : 0;
    T.restart = 1;
    T.first = 0;
  }
}

// Solve H X = B for the k columns with the device-resident loop, lw columns
// in lockstep sharing every pass over A (X holds x_0 on entry).  Plain form:
// one adaptive solve per batch.  Mixed form: refinement -- r = b - H x_o by
// the double-float pass, an inner adaptive solve of H dx = r from dx = 0 in
// float32 (relative accuracy inner_tol), x_o += dx -- until the decrement at
// x_o meets the stop rule; a column whose refinement has converged rests
// while the others go on.
sks_status solve_columns_fused(Engine& E, const double* B, double* X_io) {
  const sks_problem* prob = E.prob;
  const sks_opts* o = E.o;
  cudaStream_t stream = E.stream;
  const int d = E.d, lw = E.W.lw;
  const bool pcg = E.method == PCG;
  const double fac = pcg ? 1.0 : 2.0;
  const double tol2 = stop_coefficient(prob, o);
  sks_status result = SKS_OK;
  LoopHostCtl h;
  for (int64_t c0 = 0; c0 < prob->k; c0 += lw) {
    const int kc = (int)std::min<int64_t>(lw, prob->k - c0);
    const size_t dk = (size_t)d * lw;
    E.cur_col = (int)c0;
    // padded right-hand sides and iterate (columns past kc are zero and inert)
    SKS_CUDA_TRY(cudaMemsetAsync(E.W.lb, 0, dk * sizeof(double), stream));
    SKS_CUDA_TRY(cudaMemcpyAsync(E.W.lb, B + c0 * d, (size_t)d * kc * sizeof(double), cudaMemcpyDeviceToDevice,
                                 stream));
    double* X0 = E.mixed ? E.W.lxo : E.W.lx;
    SKS_CUDA_TRY(cudaMemsetAsync(X0, 0, dk * sizeof(double), stream));
    SKS_CUDA_TRY(cudaMemcpyAsync(X0, X_io + c0 * d, (size_t)d * kc * sizeof(double), cudaMemcpyDeviceToDevice,
                                 stream));
    std::memset(&h, 0, sizeof(h));
    for (int c = 0; c < lw; ++c) h.cols[c].active = c < kc ? 1 : 0;
    SKS_CUDA_TRY(cudaMemcpyAsync(E.W.lcols, h.cols, lw * sizeof(LoopCol), cudaMemcpyHostToDevice, stream));
    LoopTask T;
    std::memset(&T, 0, sizeof(T));
    T.method = pcg ? 0 : 1;
    T.K = lw;
    T.kc = kc;
    T.c = E.c;
    T.phi = E.phi;
    T.mu = E.mu;
    T.fac = fac;
    T.nu2 = E.nu2;
    T.lam = prob->lambda_diag;
    T.x = E.W.lx;
    T.r = E.W.lr;
    T.rt = E.W.lrt;
    T.p = E.W.lp;
    T.Hp = E.W.lHp;
    T.xp = E.W.lxp;
    T.rp = E.W.lrp;
    T.rtp = E.W.lrtp;
    T.t1 = E.W.lt1;
    T.t2 = E.W.lt2;
    T.ld_t = E.W.lt_ld;
    T.v32 = E.W.lv32;
    T.partials = E.W.lpart;
    T.dots = E.W.ldots;
    T.cols = E.W.lcols;
    T.head = E.W.lhead;
    T.trace = E.W.ltrace_cap > 0 ? E.W.ltrace : nullptr;
    T.trace_cap = E.W.ltrace_cap;
    T.st = E.W.st;
    // trace mode (plain form): the solution columns of this batch, padded like b
    if (o->x_star && !E.mixed) {
      SKS_CUDA_TRY(cudaMemsetAsync(E.W.lxs, 0, dk * sizeof(double), stream));
      SKS_CUDA_TRY(cudaMemcpyAsync(E.W.lxs, o->x_star + c0 * d, (size_t)d * kc * sizeof(double),
                                   cudaMemcpyDeviceToDevice, stream));
      T.xstar = E.W.lxs;
    }
    bool converged = false;
    if (!E.mixed) {
      T.b = E.W.lb;
      T.resid = 1;
      T.restart = 1;
      T.first = 1;
      T.tol2 = tol2;
      T.max_iter = o->max_iter;
      SKS_TRY(loop_run(E, T, &h));
      converged = true;
      double est = 0.0, dtmax = 0.0;
      for (int c = 0; c < kc; ++c) {
        const LoopCol& q = h.cols[c];
        E.S.iters += q.t;
        converged = converged && q.stop;
        est = std::max(est, q.btx > 0 ? std::sqrt(std::max(0.0, fac * q.dt / q.btx)) : 0.0);
        dtmax = std::max(dtmax, q.dt);
      }
      E.S.est_rel_err = est;
      E.S.final_delta_tilde = dtmax;
    } else {
      // refinement: the outer iterate x_o lives in lxo, the inner right-hand side in lbo
      int64_t inner_budget = o->max_iter;
      for (int64_t k = 0; k < o->max_outer; ++k) {
        E.outer = (int)k + 1;
        if (k == 0) {
          // r = b - H x_o (r = b exactly when x_o = 0, without a pass over A)
          int* flag = (int*)(E.W.scal + 3);
          any_nonzero_kernel<<<1, 256, 0, stream>>>((int)dk, X0, flag);
          note_launch();
          int hf = 1;
          SKS_CUDA_TRY(cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
          SKS_CUDA_TRY(cudaStreamSynchronize(stream));
          if (hf == 0) {
            SKS_CUDA_TRY(cudaMemcpyAsync(E.W.lbo, E.W.lb, dk * sizeof(double), cudaMemcpyDeviceToDevice, stream));
          } else {
            E.S.a_passes += 1;
            SKS_TRY(apass_launch(E.lresplan, &E.lrtmap, prob->n, d, lw, true, false, E.W.lxo, E.W.lbo, E.nu2,
                                 prob->lambda_diag, E.W.lres, E.W.st, stream, -1.0, E.W.lb, 1.0));
          }
        } else {
          E.S.a_passes += 1;
          SKS_TRY(apass_launch(E.lresplan, &E.lrtmap, prob->n, d, lw, true, false, E.W.lxo, E.W.lbo, E.nu2,
                               prob->lambda_diag, E.W.lres, E.W.st, stream, -1.0, E.W.lb, 1.0));
        }
        loop_prep_kernel<<<lw, 1024, 0, stream>>>(d, kc, pcg ? 1 : 0, E.W.lb, E.W.lxo, E.W.lbo, E.W.lx, E.W.lr,
                                                   E.W.lcols);
        note_launch();
        SKS_CUDA_TRY(cudaGetLastError());
        T.b = E.W.lbo;
        T.resid = 0;
        T.restart = 1;
        T.first = 1;
        T.tol2 = 0.0;
        T.rel2 = o->inner_tol * o->inner_tol;
        T.outer_tol2 = tol2;
        T.max_iter = std::max<int64_t>(inner_budget, 1);
        SKS_TRY(loop_run(E, T, &h));
        E.S.outer_iters += 1;
        bool all_done = true;
        int64_t tmax = 0;
        double est = 0.0;
        for (int c = 0; c < kc; ++c) {
          const LoopCol& q = h.cols[c];
          all_done = all_done && q.outer_done;
          tmax = std::max<int64_t>(tmax, q.t);
          E.S.iters += q.t;
          // the decrement at the outer iterate estimates its error
          est = std::max(est, q.btx_outer > 0 ? std::sqrt(std::max(0.0, fac * q.dt0 / q.btx_outer)) : 0.0);
        }
        E.S.est_rel_err = est;
        if (all_done) {
          converged = true;
          break;
        }
        loop_outer_add_kernel<<<dim3((unsigned)std::min(64, (d + 255) / 256), (unsigned)lw), 256, 0, stream>>>(
            d, kc, E.W.lcols, E.W.lx, E.W.lxo);
        note_launch();
        SKS_CUDA_TRY(cudaGetLastError());
        inner_budget -= tmax;
        if (inner_budget <= 0) break;
      }
    }
    SKS_CUDA_TRY(cudaMemcpyAsync(X_io + c0 * d, X0, (size_t)d * kc * sizeof(double), cudaMemcpyDeviceToDevice,
                                 stream));
    SKS_TRY(read_status(E.W.st, stream, "solver loop"));
    if (!converged && result == SKS_OK) result = fail(SKS_ERR_NO_CONVERGENCE, "max_iter reached before tol");
  }
  return result;
}

// Solve H X = B column by column with the engine's current sketch and
// preconditioner (X holds x_0 on entry).
sks_status solve_columns(Engine& E, const double* B, double* X_io) {
  if (E.fused && !E.fixed && (E.method == PCG || E.method == IHS)) return solve_columns_fused(E, B, X_io);
  const sks_problem* prob = E.prob;
  const sks_opts* o = E.o;
  cudaStream_t stream = E.stream;
  const int d = E.d;
  const double tol2 = stop_coefficient(prob, o);
  const double fac = (E.method == PCG || E.method == CG) ? 1.0 : 2.0;
  sks_status result = SKS_OK;
  for (int64_t col = 0; col < prob->k && result == SKS_OK; ++col) {
    E.cur_col = (int)col;
    const double* b = B + col * d;
    double* xcol = X_io + col * d;
    bool converged = false;
    double dt0 = 0;
    Ctl h;
    std::memset(&h, 0, sizeof(h));
    if (!E.mixed) {
      SKS_CUDA_TRY(cudaMemcpyAsync(E.W.x, xcol, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      sks_status r = E.inner(b, tol2, 0.0, o->max_iter, &converged, &dt0, &h);
      SKS_CUDA_TRY(cudaMemcpyAsync(xcol, E.W.x, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      if (r != SKS_OK) return r;
      if (E.method == CG)  // relative residual ||r|| / ||b||
        E.S.est_rel_err = E.cg_bb > 0 ? std::sqrt(std::max(0.0, h.dt / E.cg_bb)) : 0.0;
      else
        E.S.est_rel_err = h.btx > 0 ? std::sqrt(std::max(0.0, fac * h.dt / h.btx)) : 0.0;
    } else {
      // Iterative refinement: r = b - H x in float64 arithmetic, inner adaptive
      // solve of H dx = r in the precision of A, x += dx.
      SKS_CUDA_TRY(cudaMemcpyAsync(E.W.xo, xcol, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      int64_t inner_budget = o->max_iter;
      // x_0 = 0 (the usual start): r = b exactly, without a pass over A
      bool x0_zero = false;
      {
        int* flag = (int*)(E.W.scal + 3);
        any_nonzero_kernel<<<1, 256, 0, stream>>>(d, E.W.xo, flag);
        note_launch();
        int h_flag = 1;
        SKS_CUDA_TRY(cudaMemcpyAsync(&h_flag, flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
        SKS_CUDA_TRY(cudaStreamSynchronize(stream));
        x0_zero = h_flag == 0;
      }
      for (int64_t k = 0; k < o->max_outer; ++k) {
        E.outer = (int)k + 1;
        if (k == 0 && x0_zero) {
          SKS_CUDA_TRY(cudaMemcpyAsync(E.W.bo, b, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
        } else {
          SKS_TRY(E.hess64(E.W.xo, E.W.bo, -1.0, b, 1.0));
        }
        dot_kernel<<<1, kStepThreads, 0, stream>>>(d, b, E.W.xo, E.W.scal);
        note_launch();
        bool inner_conv = false, done = false;
        sks_status r = E.inner(E.W.bo, 0.0, o->inner_tol * o->inner_tol, std::max<int64_t>(inner_budget, 1),
                               &inner_conv, &dt0, &h, E.W.scal, tol2, fac, &done);
        if (r != SKS_OK) return r;
        E.S.outer_iters += 1;
        if (done) {
          converged = true;
          break;
        }
        axpy_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, 1.0, E.W.x, E.W.xo);
        note_launch();
        inner_budget -= h.t;
        if (inner_budget <= 0) break;
      }
      SKS_CUDA_TRY(cudaMemcpyAsync(xcol, E.W.xo, d * sizeof(double), cudaMemcpyDeviceToDevice, stream));
      SKS_TRY(read_status(E.W.st, stream, "refinement"));
    }
    if (!converged) result = fail(SKS_ERR_NO_CONVERGENCE, "max_iter reached before tol");
  }
  return result;
}

sks_status write_state(Engine& E) {
  SolveState h;
  std::memset(&h, 0, sizeof(h));
  h.magic = kStateMagic;
  h.n = E.prob->n;
  h.d = E.prob->d;
  h.m = E.m;
  h.dtype = (int)E.prob->dtype;
  h.precision = (int)E.o->precision;
  h.kind = (int)E.o->kind;
  h.sjlt_s = E.o->sjlt_s;
  h.seed = E.o->seed;
  SKS_CUDA_TRY(cudaMemcpyAsync(E.W.state, &h, sizeof(h), cudaMemcpyHostToDevice, E.stream));
  SKS_CUDA_TRY(cudaStreamSynchronize(E.stream));
  return SKS_OK;
}

sks_status adaptive_solve_impl(Method method, const sks_problem* prob, const sks_opts* o, double* x_io,
                               sks_stats* stats, void* ws, size_t ws_bytes, cudaStream_t stream, bool fixed = false) {
  SKS_TRY(check_opts(prob, o, x_io));
  if (method == CG && o->precision != SKS_PLAIN_F64)
    return fail(SKS_ERR_UNSUPPORTED, "the unpreconditioned CG runs in the plain float64 form only");
  if (method == CG && o->stop_rule == SKS_STOP_CERTIFIED)
    return fail(SKS_ERR_UNSUPPORTED, "the certified stop rule needs a sketched preconditioner");
  const int d = (int)prob->d;
  size_t need = 0;
  SKS_TRY(solve_layout(prob, o, nullptr, 0, nullptr, &need));
  if (!ws || ws_bytes < need) return fail(SKS_ERR_WORKSPACE, "solve workspace too small (need " + std::to_string(need) + " bytes)");
  Engine E;
  Timer t_total(stream), t_sketch(stream), t_factor(stream);
  E.t_sketch = &t_sketch;
  E.t_factor = &t_factor;
  t_total.start();
  SKS_TRY(E.init(method, prob, o, ws, ws_bytes, stream));
  E.fixed = fixed;
  SKS_CUDA_TRY(cudaMemsetAsync(E.W.state, 0, sizeof(SolveState), stream));
  SKS_CUDA_TRY(cudaMemsetAsync(E.W.st, 0, sizeof(DevStatus), stream));
  check_lambda_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, prob->lambda_diag, E.W.st);
  note_launch();
  SKS_TRY(read_status(E.W.st, stream, "input check"));
  SKS_TRY(E.first_sketch());
  const sks_status result = solve_columns(E, prob->b, x_io);
  // CG leaves no preconditioner for the adjoint to reuse
  if ((result == SKS_OK || result == SKS_ERR_NO_CONVERGENCE) && method != CG) SKS_TRY(write_state(E));
  t_total.stop();
  sks_stats& S = E.S;
  S.final_m = E.m;
  S.ms_total = t_total.acc;
  S.ms_sketch = t_sketch.acc;
  S.ms_factor = t_factor.acc;
  S.ms_iter = std::max(0.f, S.ms_total - S.ms_sketch - S.ms_factor);
  S.status = result;
  if (stats) *stats = S;
  if (result != SKS_OK) set_last_error(last_error_cstr());
  return result;
}

// ---------------------------------------------------------------- dual formulation (eq. 2)
// Workspace: D = Lambda^{-1/2} A^T (d x ldd in A's precision), b_dual = A
// Lambda^{-1} b (n x k), ones (n), w (n x k), t (d), then the workspace of the
// adaptive solve of the dual problem (n_dual = d rows, d_dual = n columns).
struct DualWs {
  DevStatus* st;
  void* D;
  long long ldd;
  double *bd, *ones, *w, *t;
  void* inner;
  size_t inner_bytes;
};

sks_problem dual_problem(const sks_problem* p, const DualWs& L) {
  sks_problem q = *p;
  q.n = p->d;
  q.d = p->n;
  q.lda = L.ldd;
  q.A = L.D;
  q.b = L.bd;
  q.lambda_diag = L.ones;
  return q;
}

sks_status dual_layout(const sks_problem* p, const sks_opts* o, void* ws, size_t ws_bytes, DualWs* L, size_t* total) {
  const size_t esz = p->dtype == SKS_F32 ? 4 : 8;
  const long long per16 = (long long)(16 / esz);
  DualWs w;
  w.ldd = (p->n + per16 - 1) / per16 * per16;  // 16-byte rows for the tensor copies
  Carver c(ws, ws_bytes);
  w.st = c.take<DevStatus>(1);
  w.D = c.take<char>((size_t)p->d * (size_t)w.ldd * esz);
  w.bd = c.take<double>((size_t)p->n * (size_t)p->k);
  w.ones = c.take<double>((size_t)p->n);
  w.w = c.take<double>((size_t)p->n * (size_t)p->k);
  w.t = c.take<double>((size_t)p->d);
  sks_problem q = dual_problem(p, w);
  size_t inner = 0;
  SKS_TRY(solve_layout(&q, o, nullptr, 0, nullptr, &inner));
  w.inner_bytes = inner;
  w.inner = c.take<char>(inner);
  if (total) *total = c.used + 256;
  if (L) *L = w;
  if (ws && !c.ok()) return fail(SKS_ERR_WORKSPACE, "dual workspace too small");
  return SKS_OK;
}

sks_status dual_solve_impl(Method method, const sks_problem* prob, const sks_opts* o, double* x_io, sks_stats* stats,
                           void* ws, size_t ws_bytes, cudaStream_t stream) {
  SKS_TRY(check_opts(prob, o, x_io));
  if (prob->n < 1) return fail(SKS_ERR_INVALID_ARG, "the dual formulation needs n >= 1");
  size_t need = 0;
  SKS_TRY(dual_layout(prob, o, nullptr, 0, nullptr, &need));
  if (!ws || ws_bytes < need) return fail(SKS_ERR_WORKSPACE, "dual workspace too small (need " + std::to_string(need) + " bytes)");
  DualWs L;
  SKS_TRY(dual_layout(prob, o, ws, ws_bytes, &L, nullptr));
  const int d = (int)prob->d;
  const int64_t n = prob->n;
  const bool f32 = prob->dtype == SKS_F32;
  // Lambda >= I is checked by the inner solve on the dual's Lambda = I only: check the primal one here
  DevStatus* st = L.st;
  SKS_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), stream));
  check_lambda_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, prob->lambda_diag, st);
  note_launch();
  SKS_TRY(read_status(st, stream, "input check"));
  dim3 tg((unsigned)((n + 31) / 32), (unsigned)((d + 31) / 32));
  if (f32)
    dual_transpose_kernel<float><<<tg, dim3(32, 8), 0, stream>>>(n, d, (const float*)prob->A, prob->lda,
                                                                 prob->lambda_diag, (float*)L.D, L.ldd);
  else
    dual_transpose_kernel<double><<<tg, dim3(32, 8), 0, stream>>>(n, d, (const double*)prob->A, prob->lda,
                                                                  prob->lambda_diag, (double*)L.D, L.ldd);
  note_launch();
  fill_kernel<<<blocks_for(n), 256, 0, stream>>>(n, 1.0, L.ones);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  // b_dual = A Lambda^{-1} b, column by column (row dots of A)
  for (int64_t c = 0; c < prob->k; ++c) {
    if (f32)
      SKS_TRY(gemv_rows<float>(stream, (int)n, d, (const float*)prob->A, prob->lda, 0, prob->b + c * d,
                               prob->lambda_diag, 1.0, L.bd + c * n, 0, nullptr, nullptr, 0.0));
    else
      SKS_TRY(gemv_rows<double>(stream, (int)n, d, (const double*)prob->A, prob->lda, 0, prob->b + c * d,
                                prob->lambda_diag, 1.0, L.bd + c * n, 0, nullptr, nullptr, 0.0));
  }
  SKS_CUDA_TRY(cudaMemsetAsync(L.w, 0, (size_t)n * prob->k * sizeof(double), stream));
  const sks_problem q = dual_problem(prob, L);
  const sks_status r = adaptive_solve_impl(method, &q, o, L.w, stats, L.inner, L.inner_bytes, stream);
  if (r != SKS_OK && r != SKS_ERR_NO_CONVERGENCE) return r;
  // x = Lambda^{-1} (b - A^T w) / nu^2
  for (int64_t c = 0; c < prob->k; ++c) {
    if (f32)
      SKS_TRY(gemv_rows<float>(stream, d, (int)n, (const float*)L.D, L.ldd, 0, L.w + c * n, nullptr, 1.0, L.t, 0,
                               nullptr, nullptr, 0.0));
    else
      SKS_TRY(gemv_rows<double>(stream, d, (int)n, (const double*)L.D, L.ldd, 0, L.w + c * n, nullptr, 1.0, L.t, 0,
                                nullptr, nullptr, 0.0));
    dual_recover_kernel<<<(d + 255) / 256, 256, 0, stream>>>(d, prob->b + c * d, L.t, prob->lambda_diag,
                                                              prob->nu * prob->nu, x_io + c * d);
    note_launch();
  }
  SKS_CUDA_TRY(cudaGetLastError());
  SKS_CUDA_TRY(cudaStreamSynchronize(stream));
  return r;
}

sks_status adjoint_impl(const sks_problem* prob, const sks_opts* o, const double* x, const double* g, double* db,
                        void* dA, long long ldda, double* dnu, double* dlambda, sks_stats* stats, void* ws,
                        size_t ws_bytes, cudaStream_t stream) {
  SKS_TRY(check_opts(prob, o, x));
  if (!g || !db) return fail(SKS_ERR_INVALID_ARG, "g and db are required");
  if (dA && ldda < prob->d) return fail(SKS_ERR_INVALID_ARG, "ldda < d");
  size_t need = 0;
  SKS_TRY(solve_layout(prob, o, nullptr, 0, nullptr, &need));
  if (!ws || ws_bytes < need) return fail(SKS_ERR_WORKSPACE, "adjoint: workspace too small");
  Engine E;
  Timer t_total(stream), t_sketch(stream), t_factor(stream);
  E.t_sketch = &t_sketch;
  E.t_factor = &t_factor;
  t_total.start();
  SKS_TRY(E.init(PCG, prob, o, ws, ws_bytes, stream));
  SolveState h;
  SKS_CUDA_TRY(cudaMemcpyAsync(&h, E.W.state, sizeof(h), cudaMemcpyDeviceToHost, stream));
  SKS_CUDA_TRY(cudaStreamSynchronize(stream));
  if (h.magic != kStateMagic || h.n != prob->n || h.d != prob->d || h.dtype != (int)prob->dtype ||
      h.precision != (int)o->precision || h.kind != (int)o->kind || h.seed != o->seed || h.m < 1)
    return fail(SKS_ERR_INVALID_ARG,
                "adjoint: the workspace does not hold the preconditioner of a solve of this problem");
  E.restore(h.m);
  SKS_CUDA_TRY(cudaMemsetAsync(E.W.st, 0, sizeof(DevStatus), stream));
  // u = H^{-1} g with the same preconditioner (solved into db: dL/db = u)
  SKS_CUDA_TRY(cudaMemsetAsync(db, 0, (size_t)prob->d * prob->k * sizeof(double), stream));
  const sks_status result = solve_columns(E, g, db);
  if (result == SKS_OK || result == SKS_ERR_NO_CONVERGENCE) {
    SKS_TRY(write_state(E));
    SKS_TRY(adjoint_grads(stream, prob, x, db, dA, ldda, dnu ? E.W.scal + 1 : nullptr, dlambda));
    if (dnu) SKS_CUDA_TRY(cudaMemcpyAsync(dnu, E.W.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, stream));
    SKS_TRY(read_status(E.W.st, stream, "adjoint"));
  }
  t_total.stop();
  sks_stats& S = E.S;
  S.final_m = E.m;
  S.ms_total = t_total.acc;
  S.ms_sketch = t_sketch.acc;
  S.ms_factor = t_factor.acc;
  S.ms_iter = std::max(0.f, S.ms_total - S.ms_sketch - S.ms_factor);
  S.status = result;
  if (stats) *stats = S;
  return result;
}

}  // namespace

// ---------------------------------------------------------------- exported helpers (used by abi.cu)
sks_status solve_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes) {
  SKS_TRY(validate_problem(p));
  if (!o || !bytes) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  return solve_layout(p, o, nullptr, 0, nullptr, bytes);
}

sks_status adaptive_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                          size_t ws_bytes, cudaStream_t stream) {
  return adaptive_solve_impl(method == 0 ? PCG : IHS, p, o, x, stats, ws, ws_bytes, stream);
}

sks_status fixed_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                       size_t ws_bytes, cudaStream_t stream) {
  static const Method kMethods[4] = {PCG, IHS, POLYAK, CG};
  if (method < 0 || method > 3) return fail(SKS_ERR_INVALID_ARG, "bad fixed-sketch method");
  return adaptive_solve_impl(kMethods[method], p, o, x, stats, ws, ws_bytes, stream, true);
}

sks_status dual_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes) {
  SKS_TRY(validate_problem(p));
  if (!o || !bytes) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  return dual_layout(p, o, nullptr, 0, nullptr, bytes);
}

sks_status dual_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                      size_t ws_bytes, cudaStream_t stream) {
  return dual_solve_impl(method == 0 ? PCG : IHS, p, o, x, stats, ws, ws_bytes, stream);
}

sks_status adjoint(const sks_problem* p, const sks_opts* o, const double* x, const double* g, double* db, void* dA,
                   long long ldda, double* dnu, double* dlambda, sks_stats* stats, void* ws, size_t ws_bytes,
                   cudaStream_t stream) {
  return adjoint_impl(p, o, x, g, db, dA, ldda, dnu, dlambda, stats, ws, ws_bytes, stream);
}

sks_status hess_apply_ws(const sks_problem* p, size_t* bytes) {
  SKS_TRY(validate_problem(p));
  if (!bytes) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  const bool f32 = p->dtype == SKS_F32;
  Carver c(nullptr, 0);
  c.take<DevStatus>(1);
  c.take<char>(apass_workspace_bytes(std::max<int64_t>(p->n, 1), p->d, p->k == 8 ? 8 : 1, f32, f32));
  c.take<char>(apass_workspace_bytes(std::max<int64_t>(p->n, 1), p->d, p->k == 8 ? 8 : 1, f32, false));
  c.take<float>((size_t)p->d * p->k * 2);
  *bytes = c.used + 256;
  return SKS_OK;
}

sks_status hess_apply(const sks_problem* p, const double* x, double* y, int extended, void* ws, size_t ws_bytes,
                      cudaStream_t stream) {
  SKS_TRY(validate_problem(p));
  if (!x || !y) return fail(SKS_ERR_INVALID_ARG, "x or y is NULL");
  size_t need = 0;
  SKS_TRY(hess_apply_ws(p, &need));
  if (!ws || ws_bytes < need) return fail(SKS_ERR_WORKSPACE, "hess_apply workspace too small");
  const bool f32 = p->dtype == SKS_F32;
  const bool vec32 = f32 && !extended;
  const int64_t kb = p->k == 8 ? 8 : 1;
  Carver c(ws, ws_bytes);
  DevStatus* st = c.take<DevStatus>(1);
  void* part32 = c.take<char>(apass_workspace_bytes(std::max<int64_t>(p->n, 1), p->d, kb, f32, f32));
  void* part64 = c.take<char>(apass_workspace_bytes(std::max<int64_t>(p->n, 1), p->d, kb, f32, false));
  float* xf = c.take<float>((size_t)p->d * p->k);
  float* yf = c.take<float>((size_t)p->d * p->k);
  SKS_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), stream));
  ApassPlan plan;
  SKS_TRY(apass_plan(std::max<int64_t>(p->n, 1), p->d, kb, f32, vec32, &plan));
  CUtensorMap tmap;
  if (p->n > 0) SKS_TRY(map_for(p, &tmap, plan));
  apass_use_bulk(&plan, p->A, p->d, p->lda, f32);
  const double nu2 = p->nu * p->nu;
  for (int64_t c0 = 0; c0 < p->k; c0 += kb) {
    const double* xc = x + c0 * p->d;
    double* yc = y + c0 * p->d;
    if (vec32) {
      const long long cnt = (long long)p->d * kb;
      f64_to_f32_kernel<<<blocks_for(cnt), 256, 0, stream>>>(cnt, xc, xf);
      note_launch();
      SKS_TRY(apass_launch(plan, &tmap, p->n, p->d, kb, true, true, xf, yf, nu2, p->lambda_diag, part32, st, stream));
      f32_to_f64_kernel<<<blocks_for(cnt), 256, 0, stream>>>(cnt, yf, yc);
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
    } else {
      SKS_TRY(apass_launch(plan, &tmap, p->n, p->d, kb, f32, false, xc, yc, nu2, p->lambda_diag, part64, st, stream));
    }
  }
  return read_status(st, stream, "hess_apply");
}

}  // namespace sks

// ============================================================================ C ABI: sketch / precond

using namespace sks;

extern "C" sks_status sks_sketch_workspace_size(const sks_problem* p, sks_kind kind, int64_t m_max, int sjlt_s,
                                                size_t* bytes) {
  SKS_TRY(validate_problem(p));
  if (!bytes) return fail(SKS_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = sketch_ws_bytes(p, kind, resolve_m_max(p, kind, m_max), sjlt_s);
  return SKS_OK;
}

extern "C" sks_status sks_sketch_create(sks_sketch** out, const sks_problem* p, sks_kind kind, int64_t m_init,
                                        int64_t m_max, int sjlt_s, uint64_t seed, void* ws, size_t ws_bytes,
                                        void* stream) {
  if (!out) return fail(SKS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  SKS_TRY(validate_problem(p));
  if (kind != SKS_SRHT && kind != SKS_GAUSSIAN && kind != SKS_SJLT && kind != SKS_RADEMACHER &&
      kind != SKS_GAUSSIAN_E4M3)
    return fail(SKS_ERR_INVALID_ARG, "bad kind");
  if (kind == SKS_GAUSSIAN_E4M3 && p->dtype != SKS_F32)
    return fail(SKS_ERR_UNSUPPORTED, "the 8-bit Gaussian sketch needs a float32 A");
  if (sjlt_s < 1 || sjlt_s > kSjltMaxS) return fail(SKS_ERR_INVALID_ARG, "sjlt_s must be in [1, 16]");
  const int64_t mm = resolve_m_max(p, kind, m_max);
  if (m_init < 1 || m_init > mm) return fail(SKS_ERR_INVALID_ARG, "m_init must be in [1, m_max]");
  if (!ws || ws_bytes < sketch_ws_bytes(p, kind, mm, sjlt_s))
    return fail(SKS_ERR_WORKSPACE, "sketch workspace too small");
  sks_sketch* s = new (std::nothrow) sks_sketch();
  if (!s) return fail(SKS_ERR_INVALID_ARG, "host allocation failed");
  cudaStream_t st = (cudaStream_t)stream;
  sks_status r = sketch_init(s, p, kind, mm, sjlt_s, seed, ws, ws_bytes, nullptr);
  if (r == SKS_OK) {
    cudaMemsetAsync(s->st, 0, sizeof(DevStatus), st);
    r = sketch_to(s, m_init, st);
  }
  if (r == SKS_OK) r = read_status(s->st, st, "sketch_create");
  if (r != SKS_OK) {
    delete s;
    return r;
  }
  *out = s;
  return SKS_OK;
}

extern "C" sks_status sks_sketch_grow(sks_sketch* s, int64_t new_m, void* stream) {
  if (!s) return fail(SKS_ERR_INVALID_ARG, "sketch is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  SKS_TRY(sketch_to(s, new_m, st));
  return read_status(s->st, st, "sketch_grow");
}

extern "C" sks_status sks_sketch_rows(const sks_sketch* s, int64_t* m) {
  if (!s || !m) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  *m = s->m;
  return SKS_OK;
}

extern "C" sks_status sks_sketch_copy_out(const sks_sketch* s, double* SA, void* stream) {
  if (!s || !SA) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  const long long cnt = (long long)s->m * s->d;
  if (cnt == 0) return SKS_OK;
  scale_rows_out_kernel<<<blocks_for(cnt), 256, 0, st>>>((int)s->m, s->d, s->Y, s->f32 ? 1 : 0, s->ldy,
                                                         std::sqrt(s->scale2()), SA);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  SKS_CUDA_TRY(cudaStreamSynchronize(st));
  return SKS_OK;
}

extern "C" void sks_sketch_destroy(sks_sketch* s) { delete s; }

extern "C" sks_status sks_precond_workspace_size(const sks_problem* p, int64_t m_max, size_t* bytes) {
  SKS_TRY(validate_problem(p));
  if (!bytes) return fail(SKS_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = precond_ws_bytes(p, std::max<int64_t>(m_max, 1));
  return SKS_OK;
}

extern "C" sks_status sks_precond_build(sks_precond** out, const sks_sketch* s, const sks_problem* p, void* ws,
                                        size_t ws_bytes, void* stream) {
  return sks_precond_build_ex(out, s, p, SKS_PLAIN_F64, ws, ws_bytes, stream);
}

extern "C" sks_status sks_precond_build_ex(sks_precond** out, const sks_sketch* s, const sks_problem* p,
                                           sks_precision precision, void* ws, size_t ws_bytes, void* stream) {
  if (!out || !s) return fail(SKS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  SKS_TRY(validate_problem(p));
  if (p->d != s->d) return fail(SKS_ERR_INVALID_ARG, "sketch and problem disagree on d");
  if (precision != SKS_PLAIN_F64 && precision != SKS_MIXED_REFINED)
    return fail(SKS_ERR_INVALID_ARG, "unknown precision");
  const bool mixed = precision == SKS_MIXED_REFINED;
  if (mixed && p->dtype != SKS_F32) return fail(SKS_ERR_INVALID_ARG, "the mixed factorisation needs a float32 A");
  if (!ws || ws_bytes < precond_ws_bytes(p, s->m_max)) return fail(SKS_ERR_WORKSPACE, "preconditioner workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  sks_precond* P = new (std::nothrow) sks_precond();
  if (!P) return fail(SKS_ERR_INVALID_ARG, "host allocation failed");
  sks_status r = precond_init(P, p, s->m_max, ws, ws_bytes, nullptr, mixed);
  if (r == SKS_OK) {
    cudaMemsetAsync(P->st, 0, sizeof(DevStatus), st);
    check_lambda_kernel<<<(int)((p->d + 255) / 256), 256, 0, st>>>((int)p->d, p->lambda_diag, P->st);
    note_launch();
    r = precond_factor(P, s, p->nu, p->lambda_diag, st);
  }
  if (r == SKS_OK) r = read_status(P->st, st, "precond_build");
  if (r != SKS_OK) {
    delete P;
    return r;
  }
  *out = P;
  return SKS_OK;
}

extern "C" sks_status sks_precond_apply(const sks_precond* P, const double* z, double* v, int64_t k, void* stream) {
  if (!P || !z || !v || k < 1) return fail(SKS_ERR_INVALID_ARG, "bad argument");
  cudaStream_t st = (cudaStream_t)stream;
  for (int64_t c = 0; c < k; ++c) SKS_TRY(precond_apply1(P, z + c * P->d, v + c * P->d, st));
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

extern "C" void sks_precond_destroy(sks_precond* P) { delete P; }
