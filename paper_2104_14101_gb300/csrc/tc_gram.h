// tc_gram.h -- tensor-core (tcgen05) split-bfloat16 Gram products.
#pragma once

#include <cuda_bf16.h>

#include "internal.h"

namespace sks {

// Elements of one hi (or lo) buffer for an operand of out_rows x K.
size_t tc_gram_split_elems(int out_rows, int K);

// X (rows x cols float32, leading dimension ldx) -> bfloat16 hi/lo slices of
// shape out_rows x Kp (Kp = K rounded up to 64, zero padded), where the
// operand is X (out_rows = rows, K = cols) or X^T (transpose: out_rows =
// cols, K = rows); optional division of column c of X by sqrt(colscale[c])
// (then colfac, 2 cols doubles, receives 1/sqrt(colscale) and sqrt(colscale)
// for tc_unsplit).  Each operand row is split against its own maximum
// exponent so that the tensor-core products are exact (tc_gram.cu).  rmax:
// out_rows scratch words.
sks_status tc_split(cudaStream_t stream, const float* X, long long ldx, int rows, int cols, bool transpose,
                    const double* colscale, __nv_bfloat16* Hh, __nv_bfloat16* Hl, unsigned* rmax, int* Kp_out,
                    double* colfac = nullptr);

// Y (rows x cols float64) = (Hh + Hl) * diag(sq): the matrix the split
// operands represent exactly (sq = the second half of tc_split's colfac, or
// NULL for no scaling).
sks_status tc_unsplit(cudaStream_t stream, const __nv_bfloat16* Hh, const __nv_bfloat16* Hl, int rows, int cols,
                      int Kp, const double* sq, double* Y, long long ldy);

// C = alpha * (Ah + Al)(Bh + Bl)^T + beta * C (float64 C, M x N); operands
// M x Kp and N x Kp bfloat16 row-major; lower: only C's lower triangle (M == N).
sks_status tc_gram(cudaStream_t stream, int M, int N, int Kp, const __nv_bfloat16* Ah, const __nv_bfloat16* Al,
                   const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, double alpha, double beta, double* C,
                   long long ldc, bool lower, DevStatus* st);

// ---- double-float trailing update of the mixed factorisation on the tensor cores
// T -= P P^T (lower part, rest x rest, float32 hi/lo planes with leading
// dimension ldt), P = rest x 64 hi/lo planes (leading dimension ld): P sliced
// per row into six bfloat16 integer slices, the slice products summed exactly
// per level in TMEM (tc_gram.cu).  ws: tc_syrk_ws_bytes(rest) bytes.
size_t tc_syrk_ws_bytes(int n);
sks_status tc_syrk_df32(cudaStream_t stream, int rest, const float* Ph, const float* Pl, long long ld, float* Th,
                        float* Tl, long long ldt, void* ws, size_t ws_bytes, DevStatus* st);

// ---- Gaussian sketch of a float32 A on the tensor cores (K4)
// Padded K (data rows rounded up to 64) of the split A^T.
int tc_gauss_kp(long long n);
// float32 elements of the slice partials for up to max_rows new rows per call.
size_t tc_gauss_part_elems(long long n, int d, int max_rows);
// Hh/Hl (d x Kp bfloat16): the element-wise split of A^T, hi = bf16(a),
// lo = bf16(a - hi), |a - hi - lo| <= 2^-17 |a|.
sks_status tc_split_t(cudaStream_t stream, const float* A, long long lda, long long n, int d, __nv_bfloat16* Hh,
                      __nv_bfloat16* Hl);
// Y[m_off .. m_off + m_add) = bf16(G) (Hh + Hl)^T, G[r][i] the Philox /
// Box-Muller entry of sketch row r and data row i (float32, rounded to
// bfloat16), generated inside the kernel; unscaled (S A = Y / sqrt(m)).
// rademacher: the +-1 entries of the Rademacher embedding instead of G.
// With A8t (d x Kp e4m3 bytes) and scale ([slices][d]): the 8-bit sketch,
// e4m3(G) times A quantised to e4m3 against one power-of-two scale per column
// and K slice of 16384 data rows (tc_split8_t), each slice scaled back.
sks_status tc_gauss_sketch(cudaStream_t stream, const __nv_bfloat16* Hh, const __nv_bfloat16* Hl, long long n, int d,
                           uint64_t seed, int m_off, int m_add, float* part, size_t part_elems, float* Y,
                           long long ldy, DevStatus* st, bool rademacher = false,
                           const unsigned char* A8t = nullptr, const float* scale = nullptr);
// K slices of the tensor-core sketch (slices of 16384 data rows).
int tc_gauss_slices(long long n);
// The 8-bit operand of the sketch: per (slice, column) scales from the
// column maxima (smax: slices x d scratch words), A8t = e4m3(A / scale)^T
// (d x Kp bytes), and frob2 = ||A||_F^2 (float64, device).
sks_status tc_split8_t(cudaStream_t stream, const float* A, long long lda, long long n, int d, unsigned char* A8t,
                       float* scale, unsigned* smax, double* frob2);

}  // namespace sks
