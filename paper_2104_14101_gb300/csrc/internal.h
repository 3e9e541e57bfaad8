// internal.h -- host-side declarations shared by the translation units of the
// sks library (not part of the public C ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "common.cuh"
#include "sks.h"

namespace sks {

// ---------------------------------------------------------------- errors
void set_last_error(const std::string& msg);
sks_status fail(sks_status code, const std::string& msg);
const char* last_error_cstr();

// Kernel-launch accounting (thread-local; see sks_kernel_launch_count).
void note_launch(int count = 1);
uint64_t launch_count();

#define SKS_CUDA_TRY(expr)                                                                     \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return ::sks::fail(SKS_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));    \
  } while (0)

#define SKS_TRY(...)                         \
  do {                                       \
    sks_status s_ = (__VA_ARGS__);           \
    if (s_ != SKS_OK) return s_;             \
  } while (0)

// ---------------------------------------------------------------- device info
struct DeviceInfo {
  int device = -1;
  int sms = 0;
  size_t smem_optin = 0;
};
const DeviceInfo& device_info();

// ---------------------------------------------------------------- workspace carving
// Bump allocator over a caller-provided device buffer (256-byte alignment).
struct Carver {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  Carver(void* b, size_t c) : base((char*)b), cap(c) {}
  template <typename T>
  T* take(size_t count) {
    used = (used + 255) & ~(size_t)255;
    T* p = base ? (T*)(base + used) : nullptr;
    used += count * sizeof(T);
    return p;
  }
  bool ok() const { return used <= cap; }
};

// ---------------------------------------------------------------- tensor maps
// 2-D tiled tensor map over a row-major rows x cols matrix with leading
// dimension ld (elements), box (box_cols x box_rows), no swizzle, zero fill.
sks_status make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, size_t elem_bytes,
                        uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_cols, uint32_t box_rows);
// 8-bit rows x cols (row-major, ld = cols), 128-byte swizzle (box_cols == 128).
sks_status make_tmap_2d_u8_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_cols,
                                 uint32_t box_rows);
// bfloat16 rows x cols (row-major, ld = cols), 128-byte swizzle (box_cols * 2 == 128).
sks_status make_tmap_2d_bf16_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                                   uint32_t box_cols, uint32_t box_rows);

// ---------------------------------------------------------------- A-pass (K1)
// Geometry of one A-pass launch (host-computed).
struct ApassPlan {
  int grid = 0, group = 0, q = 0, rows_per_stage = 0, stages = 0, boxw = 0, nbox = 0, dp = 0;
  int bulk = 0;                 // whole-row 1-D bulk copies (set by apass_use_bulk)
  int wide = 0;                 // d > 4096: the wide-row instantiations
  const void* A = nullptr;
  long long lda_bytes = 0;
  size_t smem = 0;
  size_t partial_elems = 0;  // grid * k * d
};

// y = A^T (A x) + nu^2 lambda .* x for k columns.
//   a_f32: A stored float32; vec_f32: x / y float32 (else float64).
//   extended: float64 arithmetic on float32 A (the refinement residual).
// partials: device scratch (plan.partial_elems elements of the vector type).
// With addv: y = sgn * H x + addc * addv (residuals and gradients in one launch).
sks_status apass_plan(int64_t n, int64_t d, int64_t k, bool a_f32, bool vec_f32, ApassPlan* plan);
sks_status apass_launch(const ApassPlan& plan, const CUtensorMap* tmap, int64_t n, int64_t d, int64_t k,
                        bool a_f32, bool vec_f32, const void* x, void* y, double nu2, const double* lambda,
                        void* partials, DevStatus* st, cudaStream_t stream, double sgn = 1.0,
                        const void* addv = nullptr, double addc = 0.0, cudaEvent_t ev_begin = nullptr,
                        cudaEvent_t ev_end = nullptr);
size_t apass_workspace_bytes(int64_t n, int64_t d, int64_t k, bool a_f32, bool vec_f32);
// Switch a plan to whole-row bulk copies when every row of A is a 16-byte
// multiple (stages then hold rows back to back, no column padding).
void apass_use_bulk(ApassPlan* plan, const void* A, int64_t d, int64_t lda, bool a_f32);

// ---------------------------------------------------------------- solver entry points (solver.cu)
// Host-side checks of a problem description (sizes, pointers, alignment).
// validate_operator checks what defines H (A, n, d, lda, k, nu, lambda);
// validate_problem also requires the right-hand side b.
sks_status validate_operator(const sks_problem* p);
sks_status validate_problem(const sks_problem* p);
// Element-wise precision conversions (grid-stride) and the grid size they use.
__global__ void f64_to_f32_kernel(long long count, const double* a, float* b);
__global__ void f32_to_f64_kernel(long long count, const float* a, double* b);
unsigned blocks_for(long long n, int t = 256);
// Reads the device status word (one stream synchronisation) and turns a
// device-side error into an sks_status with a message naming `what`.
sks_status read_status(DevStatus* st, cudaStream_t stream, const char* what);

sks_status solve_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes);
// method 0: adaptive PCG (Algorithm 2); 1: adaptive IHS (Algorithm 1)
sks_status adaptive_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                          size_t ws_bytes, cudaStream_t stream);
// Dual formulation (eq. 2): method 0 adaptive PCG, 1 adaptive IHS on the dual problem.
sks_status dual_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes);
sks_status dual_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                      size_t ws_bytes, cudaStream_t stream);
// method 0: PCG, 1: IHS, 2: Polyak-IHS (all with H_S fixed at m = m_init), 3: CG (H_S = I)
sks_status fixed_solve(int method, const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats, void* ws,
                       size_t ws_bytes, cudaStream_t stream);
sks_status adjoint(const sks_problem* p, const sks_opts* o, const double* x, const double* g, double* db, void* dA,
                   long long ldda, double* dnu, double* dlambda, sks_stats* stats, void* ws, size_t ws_bytes,
                   cudaStream_t stream);
// adjoint.cu: gradients from x and u = H^{-1} g (device pointers, d x k column-major)
sks_status adjoint_grads(cudaStream_t stream, const sks_problem* p, const double* x, const double* u, void* dA,
                         long long ldda, double* dnu_dev, double* dlambda);
sks_status batch_workspace_size(const sks_problem* probs, int count, const sks_opts* o, size_t* bytes);
sks_status solve_batched(const sks_problem* probs, int count, const sks_opts* o, double* const* xs, sks_stats* stats,
                         sks_batch_info* info, int rows_per_unit, void* ws, size_t ws_bytes, cudaStream_t stream);
sks_status batch_create(sks_batch** out, const sks_problem* probs, int count, const sks_opts* o, int rows_per_unit,
                        void* ws, size_t ws_bytes, cudaStream_t stream);
sks_status batch_solve(sks_batch* plan, double* const* xs, sks_stats* stats, sks_batch_info* info,
                       cudaStream_t stream);
void batch_destroy(sks_batch* plan);
sks_status selftest_wait_timeout(long long limit_ns, cudaStream_t stream);
sks_status hess_apply_ws(const sks_problem* p, size_t* bytes);
sks_status hess_apply(const sks_problem* p, const double* x, double* y, int extended, void* ws, size_t ws_bytes,
                      cudaStream_t stream);

}  // namespace sks
