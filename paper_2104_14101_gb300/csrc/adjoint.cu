// adjoint.cu -- gradients of the solution map of problem (1).
//
// For X = H^{-1} B (k right-hand sides) and an upstream gradient G = dL/dX the
// adjoint solve gives U = H^{-1} G (H is symmetric); then
//     dL/dB = U,   dL/dA = -A (U X^T + X U^T),
//     dL/dnu = -2 nu sum_k u_k^T Lambda x_k,   dL/dLambda_ii = -nu^2 sum_k u_ik x_ik.
// K10: dA is formed in one pass over A: for each row a_i the 2k dots
// p_k = a_i^T u_k and q_k = a_i^T x_k, then row i of dA is
// -sum_k (p_k x_k^T + q_k u_k^T) -- one read of A and one write of dA.
#include <algorithm>

#include "internal.h"

namespace sks {
namespace {

constexpr int kAdjK = 8;  // right-hand sides handled per pass

// One warp per row; U and X (k x d, float64, column-major d x k) staged in
// shared memory in the precision of A.
template <typename TA>
__global__ void __launch_bounds__(256) adjoint_dA_kernel(const TA* __restrict__ A, long long lda, int64_t n, int d,
                                                        int k, const double* __restrict__ U,
                                                        const double* __restrict__ X, TA* __restrict__ dA,
                                                        long long ldda) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TA* us = (TA*)smem_raw;  // [k][d]
  TA* xs = us + (size_t)k * d;
  for (int e = threadIdx.x; e < k * d; e += blockDim.x) {
    us[e] = (TA)U[e];
    xs[e] = (TA)X[e];
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int64_t i = (int64_t)blockIdx.x * nw + warp; i < n; i += (int64_t)gridDim.x * nw) {
    const TA* a = A + i * lda;
    TA p[kAdjK], q[kAdjK];
#pragma unroll
    for (int c = 0; c < kAdjK; ++c) p[c] = q[c] = TA(0);
    for (int j = lane; j < d; j += 32) {
      const TA av = a[j];
#pragma unroll
      for (int c = 0; c < kAdjK; ++c)
        if (c < k) {
          p[c] += av * us[c * d + j];
          q[c] += av * xs[c * d + j];
        }
    }
#pragma unroll
    for (int c = 0; c < kAdjK; ++c)
      if (c < k) {
        p[c] = warp_sum(p[c]);
        q[c] = warp_sum(q[c]);
      }
    TA* out = dA + i * ldda;
    for (int j = lane; j < d; j += 32) {
      TA v = TA(0);
#pragma unroll
      for (int c = 0; c < kAdjK; ++c)
        if (c < k) v += p[c] * xs[c * d + j] + q[c] * us[c * d + j];
      out[j] = -v;
    }
  }
}

// dlambda_i = -nu^2 sum_k u_ik x_ik;  dnu = -2 nu sum_i lambda_i sum_k u_ik x_ik
__global__ void __launch_bounds__(1024) adjoint_small_kernel(int d, int k, const double* __restrict__ U,
                                                             const double* __restrict__ X,
                                                             const double* __restrict__ lam, double nu,
                                                             double* __restrict__ dlam, double* __restrict__ dnu) {
  __shared__ double scratch[32];
  double acc = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < k; ++c) s += U[(size_t)c * d + j] * X[(size_t)c * d + j];
    if (dlam) dlam[j] = -nu * nu * s;
    acc += lam[j] * s;
  }
  acc = block_sum(acc, scratch);
  if (threadIdx.x == 0 && dnu) *dnu = -2.0 * nu * acc;
}

}  // namespace

sks_status adjoint_grads(cudaStream_t stream, const sks_problem* p, const double* x, const double* u, void* dA,
                         long long ldda, double* dnu_dev, double* dlambda) {
  const int d = (int)p->d;
  const int k = (int)p->k;
  if (k > kAdjK && dA) return fail(SKS_ERR_UNSUPPORTED, "adjoint: dA supports at most 8 right-hand sides");
  if (dlambda || dnu_dev) {
    adjoint_small_kernel<<<1, 1024, 0, stream>>>(d, k, u, x, p->lambda_diag, p->nu, dlambda, dnu_dev);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  if (dA && p->n > 0) {
    const int sms = device_info().sms > 0 ? device_info().sms : 152;
    for (int c0 = 0; c0 < k; c0 += kAdjK) {
      const int kc = std::min(kAdjK, k - c0);
      const size_t esz = p->dtype == SKS_F32 ? 4 : 8;
      const size_t smem = (size_t)2 * kc * d * esz;
      if (smem > 200 * 1024) return fail(SKS_ERR_UNSUPPORTED, "adjoint: k * d too large for the dA kernel");
      const unsigned grid = (unsigned)std::min<int64_t>((int64_t)sms * 4, (p->n + 7) / 8);
      const double* uc = u + (size_t)c0 * d;
      const double* xc = x + (size_t)c0 * d;
      if (p->dtype == SKS_F32) {
        SKS_CUDA_TRY(cudaFuncSetAttribute(adjoint_dA_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        adjoint_dA_kernel<float><<<grid, 256, smem, stream>>>((const float*)p->A, p->lda, p->n, d, kc, uc, xc,
                                                              (float*)dA, ldda);
      } else {
        SKS_CUDA_TRY(cudaFuncSetAttribute(adjoint_dA_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
        adjoint_dA_kernel<double><<<grid, 256, smem, stream>>>((const double*)p->A, p->lda, p->n, d, kc, uc, xc,
                                                               (double*)dA, ldda);
      }
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
    }
  }
  return SKS_OK;
}

}  // namespace sks
