// chol.cu -- the factorisation of the sketched preconditioner (Section 4.1.1)
// in double-float arithmetic: H = L L^T of H_S (m >= d) or of the Woodbury
// system W_S (m < d), and the inverse factor X = L^{-1} that the apply uses.
//
// Every value is the unevaluated sum hi + lo of two float32 numbers (about
// 48 significant bits) and every operation runs on the float32 pipe: on this
// part float64 arithmetic -- format conversions included -- runs at ~1/64 of
// the float32 rate, so the matrix is split into two float planes once (with
// integer operations) and stays there until the inverse factor is written.
//
// Per block column k (64 columns; one launch each):
//   chol_panel_df32_kernel  every CTA factors the 64 x 64 diagonal block and
//                           inverts its factor (replicated, so that no launch
//                           waits on another); CTA 0 stores L_kk^{-1}, the
//                           others form their rows of the panel
//                           L_ik = H_ik L_kk^{-T} = H_ik (L_kk^{-1})^T;
//   trailing update       H_ij -= L_ik L_jk^T on the lower part: on the tensor
//                           cores from order kTcSyrkMin up (tc_syrk_df32: each
//                           row of the panel split into six bfloat16 integer
//                           slices, the slice products summed exactly per level),
//                           else syrk_df32_planes_kernel on the float32 pipe.
// Then X from the diagonal-block inverses by recursive merging,
//   inv([A 0; B C]) = [A^{-1} 0; -C^{-1} B A^{-1}  C^{-1}],
// in float32 (Cholesky form: the apply X^T X is positive definite for any
// nonsingular X) or in double-float (Woodbury form, whose apply subtracts two
// terms of size ~1/nu^2).
//
// Double-float operations: TwoSum (Knuth), FastTwoSum (Dekker) and the
// FMA-based TwoProd (Ogita, Rump and Oishi, SISC 2005); sums of products keep
// the low part unnormalised until the end, which bounds the error of a dot
// product of length K by ~K * 2^-47 times the sum of the magnitudes.
#include <algorithm>

#include "dense.h"
#include "df32.cuh"
#include "tc_gram.h"

namespace sks {

namespace {

constexpr int NB = 64;       // block size of the factorisation
constexpr int kTcSyrkMin = 256;  // trailing matrices from this order up go to the tensor cores
constexpr int kCT = 256;     // threads of the factor and update kernels

SKS_DEV void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
SKS_DEV void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }


// ---------------------------------------------------------------- split and scale
// s = floor(e / 2) for the binary exponent e of the largest diagonal entry:
// the factorisation runs on 2^(-2s) H (largest diagonal in [1, 4)), whose
// factor is 2^(-s) L and inverse factor 2^s X.  Exact (powers of two).
__global__ void __launch_bounds__(256) diag_scale_kernel(int n, const double* __restrict__ H, long long ldh,
                                                         int* __restrict__ s_out) {
  __shared__ double part[256];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) v = fmax(v, H[(long long)i * ldh + i]);
  part[threadIdx.x] = v;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) part[threadIdx.x] = fmax(part[threadIdx.x], part[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = part[0];
    const int E = (int)(((unsigned long long)__double_as_longlong(m) >> 52) & 0x7ff);
    // zero, subnormal or non-finite maximum: no scaling (the pivot check reports it)
    *s_out = (E == 0 || E == 0x7ff) ? 0 : ((E - 1023) >> 1);
  }
}

// 2^(-2s) H (lower triangle, float64) -> hi/lo planes (n x n, ld n).
__global__ void split_lower_kernel(int n, const double* __restrict__ H, long long ldh, const int* __restrict__ s_in,
                                   float* __restrict__ Hh, float* __restrict__ Hl) {
  const int i = blockIdx.y;
  const int s2 = -2 * *s_in;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= i && j < n; j += gridDim.x * blockDim.x) {
    const F2 v = split_f64(scale_pow2(H[(long long)i * ldh + j], s2));
    Hh[(long long)i * n + j] = v.h;
    Hl[(long long)i * n + j] = v.l;
  }
}

// ---------------------------------------------------------------- diagonal block + panel
// The 64 x 64 diagonal block is factored by 16-column sub-blocks, all in
// shared memory (hi/lo planes A and X):
//   (1) the 16 x 16 diagonal sub-block: 16 right-looking steps, one barrier
//       each; the columns are scaled by rd_k = 1/sqrt(pivot_k) afterwards, and
//       its inverse W is built alongside (W = I; at step k,
//       W_ij -= L_ik (W_kj rd_k) for i > k >= j; row k is scaled by rd_k);
//   (2) the rows of the block below the sub-block: L = A X_cc^T;
//   (3) the block's own trailing update A_ij -= sum_q L_iq L_jq.
// Then the off-diagonal 16 x 16 blocks of X = L^{-1} in three rounds,
// X_rc = -X_rr sum_{c <= q < r} L_rq X_qc.
constexpr int kSub = 16;
constexpr int kSubTri = kSub * (kSub + 1) / 2;  // 136 entries of a lower 16 x 16 block

SKS_DEV void tri_index(int t, int& i, int& j) {  // t -> (i, j), j <= i, row-major lower triangle
  i = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  j = t - i * (i + 1) / 2;
}

template <int PR>
__global__ void __launch_bounds__(kCT) chol_panel_df32_kernel(float* __restrict__ Hh, float* __restrict__ Hl,
                                                               long long ld, int n, int k0, int nb,
                                                               float* __restrict__ Dh, float* __restrict__ Dl,
                                                               DevStatus* st) {
  extern __shared__ float cp_smem[];
  float (*Ah)[NB + 1] = (float (*)[NB + 1])cp_smem;  // the block, becoming L
  float (*Al)[NB + 1] = Ah + NB;
  float (*Xh)[NB + 1] = Al + NB;                      // its inverse factor
  float (*Xl)[NB + 1] = Xh + NB;
  float (*Ph)[NB + 1] = Xl + NB;                      // PR panel rows
  float (*Pl)[NB + 1] = Ph + PR;
  __shared__ float rdh[NB], rdl[NB];
  const int tid = threadIdx.x;
  const bool panel = blockIdx.x > 0;
  const int r0 = k0 + nb + ((int)blockIdx.x - 1) * PR;
  const int prow = panel ? min(PR, n - r0) : 0;
  if (panel) {  // the panel rows do not depend on the factorisation: copy them first
    for (int e = tid; e < PR * NB; e += kCT) {
      const int r = e / NB, q = e % NB;
      if (r < prow && q < nb) {
        const long long g = (long long)(r0 + r) * ld + k0 + q;
        cp_async4(&Ph[r][q], Hh + g);
        cp_async4(&Pl[r][q], Hl + g);
      } else {
        Ph[r][q] = 0.f;
        Pl[r][q] = 0.f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  for (int e = tid; e < NB * NB; e += kCT) {  // identity padding past nb
    const int i = e / NB, j = e % NB;
    const bool in = j <= i && i < nb;
    const long long g = (long long)(k0 + i) * ld + k0 + j;
    Ah[i][j] = in ? Hh[g] : (i == j ? 1.f : 0.f);
    Al[i][j] = in ? Hl[g] : 0.f;
    Xh[i][j] = 0.f;
    Xl[i][j] = 0.f;
  }
  // this thread's entries of a 16 x 16 lower triangle (two sets: Cholesky and inverse)
  int ti0, tj0;
  tri_index(tid < kSubTri ? tid : tid - kSubTri, ti0, tj0);
  const bool tinv = tid >= kSubTri;  // threads 136..255 take inverse entries 0..119
  int ti1 = 0, tj1 = 0;
  if (tid < 2 * kSubTri - kCT) tri_index(kCT - kSubTri + tid, ti1, tj1);  // inverse entries 120..135
  const bool has1 = tid < 2 * kSubTri - kCT;
  for (int c = 0; c < NB / kSub; ++c) {
    const int c0 = kSub * c;
    if (tid < kSub) Xh[c0 + tid][c0 + tid] = 1.f;  // W = I
    __syncthreads();
    for (int k = 0; k < kSub; ++k) {
      const int kk = c0 + k;
      F2 piv = {Ah[kk][kk], Al[kk][kk]};
      if (!(piv.h > 0.f) || !(piv.h < INFINITY)) {
        if (tid == 0 && blockIdx.x == 0) raise_status(st, SKS_ERR_NOT_PD, 21, k0 + kk);
        piv = {1.f, 0.f};
      }
      const F2 r = f2_rsqrt(piv);
      if (tid == 0) {
        rdh[kk] = r.h;
        rdl[kk] = r.l;
      }
      if (!tinv) {  // Cholesky entry (i, j): A_ij -= (A_ik r)(A_jk r) for j > k
        if (tj0 > k) {
          const F2 li = f2_mul({Ah[c0 + ti0][kk], Al[c0 + ti0][kk]}, r);
          const F2 lj = f2_mul({Ah[c0 + tj0][kk], Al[c0 + tj0][kk]}, r);
          f2_acc<true>(Ah[c0 + ti0][c0 + tj0], Al[c0 + ti0][c0 + tj0], li, lj);
        }
      } else if (ti0 > k && tj0 <= k) {  // inverse entry: W_ij -= (A_ik r)(W_kj r)
        const F2 li = f2_mul({Ah[c0 + ti0][kk], Al[c0 + ti0][kk]}, r);
        const F2 xk = f2_mul({Xh[kk][c0 + tj0], Xl[kk][c0 + tj0]}, r);
        f2_acc<true>(Xh[c0 + ti0][c0 + tj0], Xl[c0 + ti0][c0 + tj0], li, xk);
      }
      if (has1 && ti1 > k && tj1 <= k) {
        const F2 li = f2_mul({Ah[c0 + ti1][kk], Al[c0 + ti1][kk]}, r);
        const F2 xk = f2_mul({Xh[kk][c0 + tj1], Xl[kk][c0 + tj1]}, r);
        f2_acc<true>(Xh[c0 + ti1][c0 + tj1], Xl[c0 + ti1][c0 + tj1], li, xk);
      }
      __syncthreads();
    }
    // scale: L_ij = A_ij rd_j (j <= i), X_ij = W_ij rd_i
    if (!tinv) {
      const F2 v = f2_mul({Ah[c0 + ti0][c0 + tj0], Al[c0 + ti0][c0 + tj0]}, {rdh[c0 + tj0], rdl[c0 + tj0]});
      Ah[c0 + ti0][c0 + tj0] = v.h;
      Al[c0 + ti0][c0 + tj0] = v.l;
    } else {
      const F2 v = f2_mul({Xh[c0 + ti0][c0 + tj0], Xl[c0 + ti0][c0 + tj0]}, {rdh[c0 + ti0], rdl[c0 + ti0]});
      Xh[c0 + ti0][c0 + tj0] = v.h;
      Xl[c0 + ti0][c0 + tj0] = v.l;
    }
    if (has1) {
      const F2 v = f2_mul({Xh[c0 + ti1][c0 + tj1], Xl[c0 + ti1][c0 + tj1]}, {rdh[c0 + ti1], rdl[c0 + ti1]});
      Xh[c0 + ti1][c0 + tj1] = v.h;
      Xl[c0 + ti1][c0 + tj1] = v.l;
    }
    __syncthreads();
    const int below = NB - c0 - kSub;  // rows of the block under the sub-block
    if (below == 0) break;
    // (2) L_ij = sum_{q <= j} A_iq X_jq for the rows below (values kept until all are read)
    F2 res[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int e = tid + u * kCT;
      res[u] = {0.f, 0.f};
      if (e < below * kSub) {
        const int i = c0 + kSub + e / kSub, j = e % kSub;
        float sh = 0.f, sl = 0.f;
        for (int q = 0; q <= j; ++q)
          f2_acc<false>(sh, sl, {Ah[i][c0 + q], Al[i][c0 + q]}, {Xh[c0 + j][c0 + q], Xl[c0 + j][c0 + q]});
        res[u] = f2_two_sum(sh, sl);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int e = tid + u * kCT;
      if (e < below * kSub) {
        const int i = c0 + kSub + e / kSub, j = e % kSub;
        Ah[i][c0 + j] = res[u].h;
        Al[i][c0 + j] = res[u].l;
      }
    }
    __syncthreads();
    // (3) A_ij -= sum_{q in the sub-block} L_iq L_jq, c0 + 16 <= j <= i < 64
    const int tcount = below * (below + 1) / 2;
    for (int e = tid; e < tcount; e += kCT) {
      int i, j;
      tri_index(e, i, j);
      i += c0 + kSub;
      j += c0 + kSub;
      float sh = Ah[i][j], sl = Al[i][j];
#pragma unroll 4
      for (int q = 0; q < kSub; ++q)
        f2_acc<true>(sh, sl, {Ah[i][c0 + q], Al[i][c0 + q]}, {Ah[j][c0 + q], Al[j][c0 + q]});
      const F2 v = f2_two_sum(sh, sl);
      Ah[i][j] = v.h;
      Al[i][j] = v.l;
    }
    __syncthreads();
  }
  // off-diagonal 16 x 16 blocks of X, round s: (r, c) = (c + s, c)
  for (int s = 1; s < NB / kSub; ++s) {
    const int nblk16 = NB / kSub - s;
    F2 res[3];
    // T_rc = sum_{c16 <= q < r16} L_iq X_qj   (X_qj = 0 for q < j inside X_cc)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int e = tid + u * kCT;
      res[u] = {0.f, 0.f};
      if (e < nblk16 * kSub * kSub) {
        const int c = e / (kSub * kSub), rr = c + s;
        const int i = rr * kSub + (e / kSub) % kSub, j = c * kSub + e % kSub;
        float sh = 0.f, sl = 0.f;
        for (int q = j; q < rr * kSub; ++q) f2_acc<false>(sh, sl, {Ah[i][q], Al[i][q]}, {Xh[q][j], Xl[q][j]});
        res[u] = f2_two_sum(sh, sl);
      }
    }
#pragma unroll
    for (int u = 0; u < 3; ++u) {  // T into the (still zero) X_rc block
      const int e = tid + u * kCT;
      if (e < nblk16 * kSub * kSub) {
        const int c = e / (kSub * kSub), rr = c + s;
        const int i = rr * kSub + (e / kSub) % kSub, j = c * kSub + e % kSub;
        Xh[i][j] = res[u].h;
        Xl[i][j] = res[u].l;
      }
    }
    __syncthreads();
    // X_rc = -X_rr T_rc   (X_rr lower)
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int e = tid + u * kCT;
      res[u] = {0.f, 0.f};
      if (e < nblk16 * kSub * kSub) {
        const int c = e / (kSub * kSub), rr = c + s;
        const int il = (e / kSub) % kSub;
        const int i = rr * kSub + il, j = c * kSub + e % kSub;
        float sh = 0.f, sl = 0.f;
        for (int q = 0; q <= il; ++q)
          f2_acc<true>(sh, sl, {Xh[i][rr * kSub + q], Xl[i][rr * kSub + q]}, {Xh[rr * kSub + q][j], Xl[rr * kSub + q][j]});
        res[u] = f2_two_sum(sh, sl);
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < 3; ++u) {
      const int e = tid + u * kCT;
      if (e < nblk16 * kSub * kSub) {
        const int c = e / (kSub * kSub), rr = c + s;
        const int i = rr * kSub + (e / kSub) % kSub, j = c * kSub + e % kSub;
        Xh[i][j] = res[u].h;
        Xl[i][j] = res[u].l;
      }
    }
    __syncthreads();
  }
  // L_kk itself is not stored: only its inverse is used later (the panel
  // below and the merges read blocks strictly below the diagonal blocks), so
  // the other CTAs may still be reading the diagonal block.
  if (!panel) {
    for (int e = tid; e < NB * NB; e += kCT) {
      Dh[e] = Xh[e / NB][e % NB];
      Dl[e] = Xl[e / NB][e % NB];
    }
    return;
  }
  cp_async_wait_all();
  __syncthreads();
  // panel rows: L_rj = sum_{q <= j} P_rq X_jq; rows ty + 16a, columns tx + 16b
  const int ty = tid >> 4, tx = tid & 15;
  constexpr int RA = PR / 16;
  float sh[RA][4], sl[RA][4];
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.f;
#pragma unroll
  for (int c = 0; c < 4; ++c) {  // X_jq = 0 for q > j: the q segment c only meets columns b >= c
    if (16 * c >= nb) break;
#pragma unroll 4
    for (int qq = 0; qq < 16; ++qq) {
      const int q = 16 * c + qq;
      F2 p[RA];
#pragma unroll
      for (int a = 0; a < RA; ++a) p[a] = {Ph[ty + 16 * a][q], Pl[ty + 16 * a][q]};
#pragma unroll
      for (int b = c; b < 4; ++b) {
        const F2 x = {Xh[tx + 16 * b][q], Xl[tx + 16 * b][q]};
#pragma unroll
        for (int a = 0; a < RA; ++a) f2_acc<false>(sh[a][b], sl[a][b], p[a], x);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < RA; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int r = ty + 16 * a, j = tx + 16 * b;
      if (r < prow && j < nb) {
        const F2 v = f2_two_sum(sh[a][b], sl[a][b]);
        const long long g = (long long)(r0 + r) * ld + k0 + j;
        Hh[g] = v.h;
        Hl[g] = v.l;
      }
    }
}

// ---------------------------------------------------------------- trailing update
// T_ij -= sum_{q < kk} P_iq P_jq for the lower 64 x 64 tiles of the trailing
// matrix T (rest x rest); P = the panel just formed (rest x kk, kk <= 64).
// Planes in, planes out; each thread keeps 4 x 4 double-float sums.
__global__ void __launch_bounds__(kCT) syrk_df32_planes_kernel(int rest, int kk, const float* __restrict__ Ph,
                                                               const float* __restrict__ Pl, float* __restrict__ Th,
                                                               float* __restrict__ Tl, long long ld) {
  extern __shared__ float sy_smem[];
  float (*Ah)[NB + 1] = (float (*)[NB + 1])sy_smem;
  float (*Al)[NB + 1] = Ah + NB;
  float (*Bh)[NB + 1] = Al + NB;
  float (*Bl)[NB + 1] = Bh + NB;
  // lower tile (ti, tj), ti >= tj, from the linear block index
  int ti = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);
  while ((ti + 1) * (ti + 2) / 2 <= (int)blockIdx.x) ++ti;
  while (ti * (ti + 1) / 2 > (int)blockIdx.x) --ti;
  const int tj = (int)blockIdx.x - ti * (ti + 1) / 2;
  const int i0 = ti * NB, j0 = tj * NB;
  for (int e = threadIdx.x; e < NB * NB; e += kCT) {
    const int r = e / NB, q = e % NB;
    const bool qok = q < kk;
    const long long ga = (long long)(i0 + r) * ld + q, gb = (long long)(j0 + r) * ld + q;
    const bool aok = qok && i0 + r < rest, bok = qok && j0 + r < rest;
    Ah[r][q] = aok ? Ph[ga] : 0.f;
    Al[r][q] = aok ? Pl[ga] : 0.f;
    Bh[r][q] = bok ? Ph[gb] : 0.f;
    Bl[r][q] = bok ? Pl[gb] : 0.f;
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.f;
#pragma unroll 2
  for (int q = 0; q < kk; ++q) {
    F2 x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      x[a] = {Ah[ty * 4 + a][q], Al[ty * 4 + a][q]};
      y[a] = {Bh[tx * 4 + a][q], Bl[tx * 4 + a][q]};
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) f2_acc<false>(sh[a][b], sl[a][b], x[a], y[b]);
  }
  float* th = Th;
  float* tl = Tl;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gi = i0 + ty * 4 + a, gj = j0 + tx * 4 + b;
      if (gi < rest && gj < rest && gj <= gi) {
        const long long g = (long long)gi * ld + gj;
        const F2 t = f2_two_sum(th[g], -sh[a][b]);
        const F2 v = f2_fast_two_sum(t.h, __fadd_rn(t.l, __fsub_rn(tl[g], sl[a][b])));
        th[g] = v.h;
        tl[g] = v.l;
      }
    }
}

// ---------------------------------------------------------------- double-float GEMM (merges)
// C = alpha * A B (row-major planes; alpha = +1 or -1), batched over
// blockIdx.z with element strides sA, sB, sC.  a_lower: A is lower triangular
// (terms k > i are zero and skipped); b_lower: B is lower triangular (terms
// k < j skipped).  64 x 64 tiles, K in steps of 32.
constexpr int kGK = 32;
__global__ void __launch_bounds__(kCT) gemm_df32_kernel(int M, int N, int K, const float* __restrict__ Ah_,
                                                        const float* __restrict__ Al_, long long lda, long long sA,
                                                        const float* __restrict__ Bh_, const float* __restrict__ Bl_,
                                                        long long ldb, long long sB, float* __restrict__ Ch,
                                                        float* __restrict__ Cl, long long ldc, long long sC,
                                                        float alpha, int a_lower, int b_lower) {
  __shared__ float Ash[NB][kGK + 1], Asl[NB][kGK + 1];  // A tile [row][k]
  __shared__ float Bsh[NB][kGK + 1], Bsl[NB][kGK + 1];  // B tile transposed [col][k]
  const int row0 = blockIdx.y * NB, col0 = blockIdx.x * NB;
  Ah_ += blockIdx.z * sA;  // batch entry z
  Al_ += blockIdx.z * sA;
  Bh_ += blockIdx.z * sB;
  Bl_ += blockIdx.z * sB;
  Ch += blockIdx.z * sC;
  Cl += blockIdx.z * sC;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int kb = 0, ke = K;
  if (a_lower) ke = min(K, row0 + NB);
  if (b_lower) kb = (col0 / kGK) * kGK;
  float sh[4][4], sl[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) sh[a][b] = sl[a][b] = 0.f;
  for (int k0 = kb; k0 < ke; k0 += kGK) {
    for (int e = threadIdx.x; e < NB * kGK; e += kCT) {
      const int r = e / kGK, q = e % kGK;  // A: row r, k q
      const int gi = row0 + r, gk = k0 + q;
      const bool ok = gi < M && gk < K;
      Ash[r][q] = ok ? Ah_[(long long)gi * lda + gk] : 0.f;
      Asl[r][q] = ok ? Al_[(long long)gi * lda + gk] : 0.f;
      const int c = e % NB, qb = e / NB;  // B: k qb, column c
      const int gj = col0 + c, gkb = k0 + qb;
      const bool okb = gj < N && gkb < K;
      Bsh[c][qb] = okb ? Bh_[(long long)gkb * ldb + gj] : 0.f;
      Bsl[c][qb] = okb ? Bl_[(long long)gkb * ldb + gj] : 0.f;
    }
    __syncthreads();
#pragma unroll 4
    for (int q = 0; q < kGK; ++q) {
      F2 x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        x[a] = {Ash[ty * 4 + a][q], Asl[ty * 4 + a][q]};
        y[a] = {Bsh[tx * 4 + a][q], Bsl[tx * 4 + a][q]};
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) f2_acc<false>(sh[a][b], sl[a][b], x[a], y[b]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int gi = row0 + ty * 4 + a, gj = col0 + tx * 4 + b;
      if (gi < M && gj < N) {
        const F2 v = f2_two_sum(sh[a][b], sl[a][b]);
        Ch[(long long)gi * ldc + gj] = alpha * v.h;
        Cl[(long long)gi * ldc + gj] = alpha * v.l;
      }
    }
}

// ---------------------------------------------------------------- placement and output
// the diagonal-block inverses (NB x NB each, planes) into zeroed X planes
__global__ void place_dinv_kernel(int n, int nblk, const float* __restrict__ Dh, const float* __restrict__ Dl,
                                  float* __restrict__ Xh, float* __restrict__ Xl, long long ldx) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nblk * NB * NB) return;
  const int kb = (int)(e / (NB * NB)), i = (int)(e / NB % NB), j = (int)(e % NB);
  const int gi = kb * NB + i, gj = kb * NB + j;
  if (gi >= n || gj >= n) return;
  Xh[(long long)gi * ldx + gj] = Dh[e];
  if (Xl) Xl[(long long)gi * ldx + gj] = Dl[e];
}

// X = 2^(-s) (hi + lo) in float64 (lo may be NULL: float32 inverse); the
// widening and the power-of-two scaling are exact integer operations, one
// float64 addition remains.
__global__ void planes_to_f64_kernel(int n, const float* __restrict__ Xh, const float* __restrict__ Xl, long long ldp,
                                     const int* __restrict__ s_in, double* __restrict__ X, long long ldx) {
  const int i = blockIdx.y;
  const int s = *s_in;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const long long g = (long long)i * ldp + j;
    double v = f32_to_f64_bits(Xh[g]);
    if (Xl) v += f32_to_f64_bits(Xl[g]);
    X[(long long)i * ldx + j] = scale_pow2(v, -s);
  }
}
}  // namespace

template <int PR>
static sks_status launch_panel(cudaStream_t stream, int grid, float* Hh, float* Hl, long long ld, int n, int k0, int nb,
                               float* Dh, float* Dl, DevStatus* st) {
  constexpr size_t smem = (size_t)(4 * NB + 2 * PR) * (NB + 1) * sizeof(float);
  SKS_CUDA_TRY(cudaFuncSetAttribute(chol_panel_df32_kernel<PR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
  chol_panel_df32_kernel<PR><<<grid, kCT, smem, stream>>>(Hh, Hl, ld, n, k0, nb, Dh, Dl, st);
  note_launch();
  return cudaGetLastError() == cudaSuccess ? SKS_OK : fail(SKS_ERR_CUDA, "chol_panel_df32_kernel launch");
}

static sks_status gemm_df32(cudaStream_t stream, int M, int N, int K, const float* Ah, const float* Al, long long lda,
                            long long sA, const float* Bh, const float* Bl, long long ldb, long long sB, float* Ch,
                            float* Cl, long long ldc, long long sC, float alpha, bool a_lower, bool b_lower,
                            int batch) {
  if (M <= 0 || N <= 0 || batch <= 0) return SKS_OK;
  const dim3 grid((unsigned)((N + NB - 1) / NB), (unsigned)((M + NB - 1) / NB), (unsigned)batch);
  gemm_df32_kernel<<<grid, kCT, 0, stream>>>(M, N, K, Ah, Al, lda, sA, Bh, Bl, ldb, sB, Ch, Cl, ldc, sC, alpha,
                                             a_lower ? 1 : 0, b_lower ? 1 : 0);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

// Double-float factorisation of H (n x n, lower part read, float64) and its
// inverse factor X (float64, lower, n x n): float32 merges (f32_inverse) or
// double-float merges.  ws: cholesky_ws_elems(n) doubles; ws32:
// cholesky_ws32_elems(n) floats.  A non-positive pivot raises SKS_ERR_NOT_PD.
sks_status cholesky_inverse_df32(cudaStream_t stream, int n, const double* H, long long ldh, double* X,
                                 long long ldx, double* ws, float* ws32, DevStatus* st, bool f32_inverse) {
  if (n <= 0) return SKS_OK;
  if (ws == nullptr || ws32 == nullptr) return fail(SKS_ERR_WORKSPACE, "double-float Cholesky needs both workspaces");
  const int nblk = (n + NB - 1) / NB;
  const long long ld = n;
  float* wsf = reinterpret_cast<float*>(ws);
  int* sexp = reinterpret_cast<int*>(wsf);           // the scaling exponent s
  float* Dh = wsf + 64;                               // diagonal-block inverses, NB x NB each
  float* Dl = Dh + (size_t)nblk * NB * NB;
  float* R = Dl + (size_t)nblk * NB * NB;             // X32, or the X planes
  float* Hh = ws32;
  float* Hl = ws32 + (size_t)n * n;
  float* T = ws32 + (size_t)2 * n * n;                // merge (and trailing-update) scratch: 2 n^2 + 64 floats
  const size_t T_bytes = ((size_t)2 * n * n + 64) * sizeof(float);
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  diag_scale_kernel<<<1, 256, 0, stream>>>(n, H, ldh, sexp);
  note_launch();
  const unsigned gx = (unsigned)std::min(8, (n + 255) / 256);
  split_lower_kernel<<<dim3(gx, (unsigned)n), 256, 0, stream>>>(n, H, ldh, sexp, Hh, Hl);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  constexpr size_t kSySmem = 4 * NB * (NB + 1) * sizeof(float);
  SKS_CUDA_TRY(cudaFuncSetAttribute(syrk_df32_planes_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kSySmem));
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, nb = std::min(NB, n - k0);
    const int rest = n - k0 - nb;
    float* dh = Dh + (size_t)kb * NB * NB;
    float* dl = Dl + (size_t)kb * NB * NB;
    // 32 panel rows per CTA while the grid fits on the SMs, else 64
    if (1 + (rest + 31) / 32 <= sms) SKS_TRY(launch_panel<32>(stream, 1 + (rest + 31) / 32, Hh, Hl, ld, n, k0, nb, dh, dl, st));
    else SKS_TRY(launch_panel<64>(stream, 1 + (rest + 63) / 64, Hh, Hl, ld, n, k0, nb, dh, dl, st));
    if (rest > 0) {
      const long long pan = (long long)(k0 + nb) * ld + k0;
      const long long tr = (long long)(k0 + nb) * ld + k0 + nb;
      if (nb == NB && rest >= kTcSyrkMin && T_bytes >= tc_syrk_ws_bytes(rest)) {
        // full 64-column panels of a large trailing matrix: the tensor cores (exact slice products)
        SKS_TRY(tc_syrk_df32(stream, rest, Hh + pan, Hl + pan, ld, Hh + tr, Hl + tr, ld, T, T_bytes, st));
      } else {
        const int tb = (rest + NB - 1) / NB;
        syrk_df32_planes_kernel<<<(unsigned)(tb * (tb + 1) / 2), kCT, kSySmem, stream>>>(rest, nb, Hh + pan,
                                                                                        Hl + pan, Hh + tr, Hl + tr, ld);
        note_launch();
        SKS_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  // X' = L'^{-1} of the scaled factor from the diagonal-block inverses by merging
  const long long nn = (long long)n * n;
  const unsigned pg = (unsigned)(((long long)nblk * NB * NB + 255) / 256);
  if (f32_inverse) {
    float* X32 = R;
    SKS_CUDA_TRY(cudaMemsetAsync(X32, 0, (size_t)nn * sizeof(float), stream));
    place_dinv_kernel<<<pg, 256, 0, stream>>>(n, nblk, Dh, nullptr, X32, nullptr, ld);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    // one batched pair of products per level for the full pairs (n2 = b), one for a ragged last pair
    for (int b = NB; b < n; b *= 2) {
      const int full = n / (2 * b);
      const int r0l = full * 2 * b;
      const int n2l = std::max(0, std::min(b, n - r0l - b));
      for (int part = 0; part < 2; ++part) {
        const int cnt = part == 0 ? full : (n2l > 0 ? 1 : 0);
        if (cnt == 0) continue;
        const int r0 = part == 0 ? 0 : r0l, n1 = b, n2 = part == 0 ? b : n2l;
        const long long sd = (long long)2 * b * (ld + 1);  // from one pair's diagonal corner to the next
        float* tmp32 = T;
        float* part32 = T + (size_t)cnt * n2 * n1;
        const size_t rest32 = (size_t)2 * n * n + 64 - (size_t)cnt * n2 * n1;
        const float* Ainv = X32 + (long long)r0 * ld + r0;
        const float* Lb = Hh + (long long)(r0 + b) * ld + r0;
        const float* Cinv = X32 + (long long)(r0 + b) * ld + (r0 + b);
        float* out = X32 + (long long)(r0 + b) * ld + r0;
        SKS_TRY(gemm<float>(stream, n2, n1, n1, Lb, ld, false, Ainv, ld, false, tmp32, n1, 1.0, 0.0, false, cnt, sd,
                            sd, (long long)n2 * n1, part32, rest32, 2));
        SKS_TRY(gemm<float>(stream, n2, n1, n2, Cinv, ld, false, tmp32, n1, false, out, ld, -1.0, 0.0, false, cnt, sd,
                            (long long)n2 * n1, sd, part32, rest32, 1));
      }
    }
    planes_to_f64_kernel<<<dim3(gx, (unsigned)n), 256, 0, stream>>>(n, X32, nullptr, ld, sexp, X, ldx);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    return SKS_OK;
  }
  float* Xh = R;
  float* Xl = R + (size_t)nn;
  SKS_CUDA_TRY(cudaMemsetAsync(Xh, 0, (size_t)2 * nn * sizeof(float), stream));
  place_dinv_kernel<<<pg, 256, 0, stream>>>(n, nblk, Dh, Dl, Xh, Xl, ld);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  for (int b = NB; b < n; b *= 2) {
    const int full = n / (2 * b);
    const int r0l = full * 2 * b;
    const int n2l = std::max(0, std::min(b, n - r0l - b));
    for (int part = 0; part < 2; ++part) {
      const int cnt = part == 0 ? full : (n2l > 0 ? 1 : 0);
      if (cnt == 0) continue;
      const int r0 = part == 0 ? 0 : r0l, n1 = b, n2 = part == 0 ? b : n2l;
      const long long sd = (long long)2 * b * (ld + 1);
      const long long oa = (long long)r0 * ld + r0, ob = (long long)(r0 + b) * ld + r0;
      const long long oc = (long long)(r0 + b) * ld + (r0 + b);
      const long long st = (long long)n2 * n1;
      float* th = T;
      float* tl = T + (size_t)cnt * st;
      // tmp = B A^{-1} (A^{-1} lower), then X_21 = -C^{-1} tmp (C^{-1} lower)
      SKS_TRY(gemm_df32(stream, n2, n1, n1, Hh + ob, Hl + ob, ld, sd, Xh + oa, Xl + oa, ld, sd, th, tl, n1, st, 1.f,
                        false, true, cnt));
      SKS_TRY(gemm_df32(stream, n2, n1, n2, Xh + oc, Xl + oc, ld, sd, th, tl, n1, st, Xh + ob, Xl + ob, ld, sd, -1.f,
                        true, false, cnt));
    }
  }
  planes_to_f64_kernel<<<dim3(gx, (unsigned)n), 256, 0, stream>>>(n, Xh, Xl, ld, sexp, X, ldx);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

}  // namespace sks
