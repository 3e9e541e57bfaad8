// dense.h -- dense building blocks of the preconditioner (host launchers).
#pragma once

#include "internal.h"

namespace sks {

// C = alpha * op(A) op(B) + beta * C, row-major, batched (strides in
// elements); lower = only C's lower triangle is written.  split_ws (optional)
// enables split-K with a deterministic float64 reduction.  tri_ops: bit 0 =
// op(A) is lower triangular, bit 1 = op(B) is lower triangular (their zero
// terms are skipped; the sum over the others keeps its order).
template <typename T>
sks_status gemm(cudaStream_t stream, int M, int N, int K, const T* A, long long lda, bool ta, const T* B,
                long long ldb, bool tb, T* C, long long ldc, double alpha, double beta, bool lower, int batch,
                long long sA, long long sB, long long sC, T* split_ws, size_t split_ws_elems, int tri_ops = 0);

template <typename T>
sks_status transpose(cudaStream_t stream, int rows, int cols, const T* S, long long lds, T* D, long long ldd);

// M[i][i] += diag_add + vec_scale * diag_vec[i]
sks_status add_diagonal(cudaStream_t stream, int n, double* M, long long ld, double diag_add, const double* diag_vec,
                        double vec_scale);

size_t cholesky_ws_elems(int n);
size_t cholesky_ws32_elems(int n);
// H (n x n, lower part read) = L L^T and X = L^{-1} (lower, n x n, float64).
//   kCholF64:        float64 throughout; L overwrites H's lower triangle.
//   kCholDf32InvF32: double-float factorisation (chol.cu), inverse factor
//                    merged in float32 (the Cholesky form's apply X^T X is
//                    positive definite for any nonsingular X).
//   kCholDf32:       double-float factorisation and inverse factor (Woodbury
//                    form).  H is left unchanged by the double-float modes.
// ws: cholesky_ws_elems(n) doubles; ws32 (double-float modes):
// cholesky_ws32_elems(n) floats.  Raises SKS_ERR_NOT_PD in `st` on a
// non-positive pivot.
enum { kCholF64 = 0, kCholDf32InvF32 = 1, kCholDf32 = 2 };
sks_status cholesky_and_inverse(cudaStream_t stream, int n, double* H, long long ldh, double* X, long long ldx,
                                double* ws, DevStatus* st, float* ws32 = nullptr, int mode = kCholF64);
sks_status cholesky_inverse_df32(cudaStream_t stream, int n, const double* H, long long ldh, double* X,
                                 long long ldx, double* ws, float* ws32, DevStatus* st, bool f32_inverse);

// y_i = alpha * sum_j M[i][j] x_j / xdiv_j  (tri 0 full, 1 lower, 2 upper);
// mode 1 epilogue: y_i = (z_i - value) / (nu2 * lam_i).
template <typename T>
sks_status gemv_rows(cudaStream_t stream, int rows, int cols, const T* M, long long ldm, int tri, const double* x,
                     const double* xdiv, double alpha, double* y, int mode, const double* z, const double* lam,
                     double nu2);

}  // namespace sks
