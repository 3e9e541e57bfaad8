// abi.cu -- the exported C entry points that are not tied to a handle type
// (options, version, errors, the Hessian pass and the adaptive solvers).
#include "internal.h"

using namespace sks;

extern "C" void sks_opts_default(sks_opts* o) {
  if (!o) return;
  o->rho = 0.125;
  o->m_init = 1;
  o->m_max = 0;
  o->kind = SKS_SRHT;
  o->sjlt_s = 1;
  o->tol = 1e-10;
  o->max_iter = 1000;
  o->precision = SKS_PLAIN_F64;
  o->reuse_residual = 1;
  o->seed = 0;
  o->max_outer = 20;
  o->inner_tol = 1e-4;
  o->trace = nullptr;
  o->trace_cap = 0;
  o->stop_rule = SKS_STOP_ESTIMATE;
  o->cert_delta = 0.01;
  o->cert_de = 0.0;
  o->x_star = nullptr;
}

extern "C" const char* sks_version(void) { return "sks 0.1 (sm_103a)"; }

extern "C" const char* sks_last_error(void) { return last_error_cstr(); }

extern "C" uint64_t sks_kernel_launch_count(void) { return launch_count(); }

extern "C" sks_status sks_hess_apply_workspace_size(const sks_problem* p, size_t* bytes) { return hess_apply_ws(p, bytes); }

extern "C" sks_status sks_hess_apply(const sks_problem* p, const double* x, double* y, int extended, void* ws,
                                     size_t ws_bytes, void* stream) {
  return hess_apply(p, x, y, extended, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_solve_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes) {
  return solve_workspace_size(p, o, bytes);
}

extern "C" sks_status sks_adaptive_pcg_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                             void* ws, size_t ws_bytes, void* stream) {
  return adaptive_solve(0, p, o, x, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_adaptive_ihs_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                             void* ws, size_t ws_bytes, void* stream) {
  return adaptive_solve(1, p, o, x, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_dual_workspace_size(const sks_problem* p, const sks_opts* o, size_t* bytes) {
  return dual_workspace_size(p, o, bytes);
}

extern "C" sks_status sks_dual_pcg_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                         void* ws, size_t ws_bytes, void* stream) {
  return dual_solve(0, p, o, x, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_dual_ihs_solve(const sks_problem* p, const sks_opts* o, double* x, sks_stats* stats,
                                         void* ws, size_t ws_bytes, void* stream) {
  return dual_solve(1, p, o, x, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_fixed_solve(sks_fixed_method method, const sks_problem* p, const sks_opts* o, double* x,
                                      sks_stats* stats, void* ws, size_t ws_bytes, void* stream) {
  return fixed_solve((int)method, p, o, x, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_adjoint(const sks_problem* p, const sks_opts* o, const double* x, const double* g,
                                  double* db, void* dA, int64_t ldda, double* dnu, double* dlambda, sks_stats* stats,
                                  void* ws, size_t ws_bytes, void* stream) {
  return adjoint(p, o, x, g, db, dA, ldda, dnu, dlambda, stats, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_batch_workspace_size(const sks_problem* probs, int count, const sks_opts* o, size_t* bytes) {
  return batch_workspace_size(probs, count, o, bytes);
}

extern "C" sks_status sks_solve_batched(const sks_problem* probs, int count, const sks_opts* o, double* const* x,
                                        sks_stats* stats, sks_batch_info* info, int rows_per_unit, void* ws,
                                        size_t ws_bytes, void* stream) {
  return solve_batched(probs, count, o, x, stats, info, rows_per_unit, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_batch_create(sks_batch** out, const sks_problem* probs, int count, const sks_opts* o,
                                       int rows_per_unit, void* ws, size_t ws_bytes, void* stream) {
  return batch_create(out, probs, count, o, rows_per_unit, ws, ws_bytes, (cudaStream_t)stream);
}

extern "C" sks_status sks_batch_solve(sks_batch* plan, double* const* x, sks_stats* stats, sks_batch_info* info,
                                      void* stream) {
  return batch_solve(plan, x, stats, info, (cudaStream_t)stream);
}

extern "C" void sks_batch_destroy(sks_batch* plan) { batch_destroy(plan); }

extern "C" sks_status sks_selftest_wait_timeout(int64_t limit_ns, void* stream) {
  return selftest_wait_timeout((long long)limit_ns, (cudaStream_t)stream);
}
