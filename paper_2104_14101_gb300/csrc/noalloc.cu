// noalloc.cu -- a variant of the Hessian pass that needs no caller workspace.
//
// Who this is for: callers that are not allowed to allocate device memory at
// the point where they need H x -- for example code running inside a host
// framework that owns every device allocation through its own fixed-budget
// allocator, or a latency-critical loop that must not pay for cudaMalloc's
// device-wide synchronisation.  Such callers can still pass their own input
// and output vectors; the per-CTA partial sums the pass needs live in a
// library-owned scratch array instead of a caller-provided workspace.
//
// The scratch is a file-scope __device__ array of kNoallocScratchBytes
// (8 MiB).  Every GPU that loads the library holds it until the process
// exits.  All calls share it and it keeps the last call's contents, so calls
// whose GPU work overlaps (different streams, or different host threads on the
// same device) race on it; callers must serialise them.  The status word at
// its start is cleared on every call; the partial sums are fully rewritten.
#include <mutex>

#include "internal.h"

namespace sks {
namespace {

constexpr size_t kNoallocScratchBytes = (size_t)8 << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Device address of g_noalloc_scratch per device ordinal, looked up once per
// device (with that device current) on the first call made there.
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

sks_status scratch_for_current_device(void** out) {
  int dev = -1;
  SKS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(SKS_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
      return fail(SKS_ERR_CUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") + cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return SKS_OK;
}

}  // namespace

sks_status hess_apply_noalloc(const sks_problem* p, const double* x, double* y, int extended, cudaStream_t stream) {
  // the same checks as sks_hess_apply, minus the right-hand side it never reads
  SKS_TRY(validate_operator(p));
  if (!x || !y) return fail(SKS_ERR_INVALID_ARG, "x or y is NULL");
  const bool f32 = p->dtype == SKS_F32;
  const bool vec32 = f32 && !extended;
  const int64_t kb = p->k == 8 ? 8 : 1;
  ApassPlan plan;
  SKS_TRY(apass_plan(std::max<int64_t>(p->n, 1), p->d, kb, f32, vec32, &plan));
  {  // a plan of two CTAs per SM falls back to one per SM (each CTA keeps one set of partial sums)
     // when its partials would not fit; what does not fit then is rejected below
    const size_t esz = vec32 ? 4 : 8;
    const size_t per_cta = plan.partial_elems / (size_t)plan.grid;  // elements
    const int sms = device_info().sms > 0 ? device_info().sms : 152;
    const size_t room = kNoallocScratchBytes - 4096 - (vec32 ? (size_t)2 * p->d * kb * sizeof(float) : 0);
    if (plan.partial_elems * esz > room && plan.grid > sms) {
      plan.grid = sms;
      plan.partial_elems = (size_t)plan.grid * per_cta;
    }
  }
  // Layout inside the static scratch: status | partial sums | float32 copies of x and y.
  Carver c(nullptr, 0);
  c.take<DevStatus>(1);
  c.take<char>(plan.partial_elems * (vec32 ? 4 : 8));
  if (vec32) {
    c.take<float>((size_t)p->d * kb);
    c.take<float>((size_t)p->d * kb);
  }
  if (c.used > kNoallocScratchBytes)
    return fail(SKS_ERR_INVALID_ARG, "problem needs " + std::to_string(c.used) +
                                         " bytes of scratch; the allocation-free Hessian pass holds at most " +
                                         std::to_string(kNoallocScratchBytes));
  void* base = nullptr;
  SKS_TRY(scratch_for_current_device(&base));
  Carver w(base, kNoallocScratchBytes);
  DevStatus* st = w.take<DevStatus>(1);
  void* partials = w.take<char>(plan.partial_elems * (vec32 ? 4 : 8));
  float* xf = vec32 ? w.take<float>((size_t)p->d * kb) : nullptr;
  float* yf = vec32 ? w.take<float>((size_t)p->d * kb) : nullptr;
  SKS_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), stream));
  CUtensorMap tmap;
  if (p->n > 0)
    SKS_TRY(make_tmap_2d(&tmap, p->A, f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64,
                         f32 ? 4 : 8, (uint64_t)p->n, (uint64_t)p->d, (uint64_t)p->lda, (uint32_t)plan.boxw,
                         (uint32_t)plan.rows_per_stage));
  // whole-row bulk copies where rows allow them, as sks_hess_apply (after the
  // tensor map, which keeps the tiled geometry; the partial sums' size is unchanged)
  apass_use_bulk(&plan, p->A, p->d, p->lda, f32);
  const double nu2 = p->nu * p->nu;
  for (int64_t c0 = 0; c0 < p->k; c0 += kb) {
    const double* xc = x + c0 * p->d;
    double* yc = y + c0 * p->d;
    if (vec32) {
      const long long cnt = (long long)p->d * kb;
      f64_to_f32_kernel<<<blocks_for(cnt), 256, 0, stream>>>(cnt, xc, xf);
      note_launch();
      SKS_TRY(apass_launch(plan, &tmap, p->n, p->d, kb, true, true, xf, yf, nu2, p->lambda_diag, partials, st, stream));
      f32_to_f64_kernel<<<blocks_for(cnt), 256, 0, stream>>>(cnt, yf, yc);
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
    } else {
      SKS_TRY(apass_launch(plan, &tmap, p->n, p->d, kb, f32, false, xc, yc, nu2, p->lambda_diag, partials, st, stream));
    }
  }
  return read_status(st, stream, "hess_apply_noalloc");
}

}  // namespace sks

extern "C" sks_status sks_hess_apply_noalloc(const sks_problem* p, const double* x, double* y, int extended,
                                             void* stream) {
  return sks::hess_apply_noalloc(p, x, y, extended, (cudaStream_t)stream);
}
