// dense.cu -- dense kernels of the sketched preconditioner (Section 4.1.1):
// Gram matrices (K6), blocked Cholesky with pivot check (K7), the explicit
// inverse of the triangular factor, transposes and the row-parallel
// matrix-vector products of the preconditioner apply (a6).
//
// GB300 note: float64 runs at ~1/64 of the float32 rate on this part, so
// these kernels are bound by the float64 FMA pipe; a 64x64 register-tiled
// CUDA-core GEMM already saturates it.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "dense.h"

namespace sks {

namespace {

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

template <typename T>
struct GemmArgs {
  int M, N, K;
  const T* A;
  long long lda, sA;
  int ta;
  const T* B;
  long long ldb, sB;
  int tb;
  T* C;
  long long ldc, sC;
  double alpha, beta;
  int lower;      // 1: only tiles with row block >= col block (C lower part)
  int a_lower;    // op(A) lower triangular: terms k > i are zero and skipped
  int b_lower;    // op(B) lower triangular: terms k < j are zero and skipped
  int splits;     // split-K factor
  int kchunk;     // K range per split (multiple of BK)
  T* part;        // split partials [batch*splits][M][N] when splits > 1
  int batch;
};

template <typename T>
__global__ void __launch_bounds__(GT) gemm_kernel(GemmArgs<T> g) {
  __shared__ T As[BK][BM + 1];
  __shared__ T Bs[BK][BN + 1];
  const int bz = blockIdx.z / g.splits, sp = blockIdx.z % g.splits;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  if (g.lower && col0 > row0 + BM - 1) return;
  const T* A = g.A + bz * g.sA;
  const T* B = g.B + bz * g.sB;
  const int tid = threadIdx.x;
  const int tr = tid / 16, tc = tid % 16;  // 16 x 16 threads, 4 x 4 outputs each
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  // the K range of this split, without the terms a triangular operand makes zero
  const int k_begin = max(sp * g.kchunk, g.b_lower ? col0 : 0);
  const int k_end = min(min(g.K, sp * g.kchunk + g.kchunk), g.a_lower ? row0 + BM : g.K);
  for (int k0 = k_begin; k0 < k_end; k0 += BK) {
    // op(A) tile: BM x BK
#pragma unroll
    for (int t = 0; t < (BM * BK) / GT; ++t) {
      const int e = tid + t * GT;
      int i, k;
      if (!g.ta) { k = e % BK; i = e / BK; } else { i = e % BM; k = e / BM; }
      const int gi = row0 + i, gk = k0 + k;
      T v = T(0);
      if (gi < g.M && gk < k_end) v = g.ta ? A[(long long)gk * g.lda + gi] : A[(long long)gi * g.lda + gk];
      As[k][i] = v;
    }
    // op(B) tile: BK x BN
#pragma unroll
    for (int t = 0; t < (BN * BK) / GT; ++t) {
      const int e = tid + t * GT;
      int j, k;
      if (!g.tb) { j = e % BN; k = e / BN; } else { k = e % BK; j = e / BK; }
      const int gj = col0 + j, gk = k0 + k;
      T v = T(0);
      if (gj < g.N && gk < k_end) v = g.tb ? B[(long long)gj * g.ldb + gk] : B[(long long)gk * g.ldb + gj];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] += a[i] * b[j];
    }
    __syncthreads();
  }
  if (g.splits > 1) {
    T* P = g.part + (long long)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int gi = row0 + tr + 16 * i, gj = col0 + tc + 16 * j;
        if (gi < g.M && gj < g.N) P[(long long)gi * g.N + gj] = acc[i][j];
      }
    return;
  }
  T* C = g.C + bz * g.sC;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gi = row0 + tr + 16 * i, gj = col0 + tc + 16 * j;
      if (gi < g.M && gj < g.N && (!g.lower || gj <= gi)) {
        T* c = C + (long long)gi * g.ldc + gj;
        const double v = g.alpha * (double)acc[i][j];
        *c = (T)(g.beta == 0.0 ? v : v + g.beta * (double)(*c));
      }
    }
}

template <typename T>
__global__ void split_reduce_kernel(GemmArgs<T> g) {
  const long long mn = (long long)g.M * g.N;
  const int bz = blockIdx.y;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mn; e += (long long)gridDim.x * blockDim.x) {
    const int gi = (int)(e / g.N), gj = (int)(e % g.N);
    if (g.lower && gj > gi) continue;
    double s = 0.0;
    for (int p = 0; p < g.splits; ++p) s += (double)g.part[((long long)bz * g.splits + p) * mn + e];
    T* c = g.C + bz * g.sC + (long long)gi * g.ldc + gj;
    const double v = g.alpha * s;
    *c = (T)(g.beta == 0.0 ? v : v + g.beta * (double)(*c));
  }
}

// ------------------------------------------------------------------ Cholesky
constexpr int NB = 64;

// Factor the nb x nb diagonal block D (leading dim ld) in place (lower) and
// write the inverse of its factor to Dinv (nb x nb, ld nb).  Raises NOT_PD on
// a pivot <= 0 or non-finite.  One CTA of 256 threads.
// 1/sqrt(p) for p > 0 in float64: float32 seed, two Newton steps
// (r <- r (3 - p r^2) / 2; relative error ~1e-7 -> ~1e-14 -> below 1 ulp)
SKS_DEV double rsqrt_newton(double p) {
  if (!(p > 1e-30 && p < 1e30)) return 1.0 / sqrt(p);  // outside the float32 seed's range
  double r = (double)rsqrtf((float)p);
  r = r * (1.5 - 0.5 * p * r * r);
  r = r * (1.5 - 0.5 * p * r * r);
  return r;
}

// In-place Cholesky of the nb x nb block L (float64, shared memory, 256
// threads); rd[k] = 1 / L[k][k].  Per column: one thread takes the pivot
// while the column is copied, then the scaled column and the trailing
// update are written in one pass (two barriers per column).  A
// non-positive pivot raises SKS_ERR_NOT_PD (when `report`) and continues with 1.
SKS_DEV void chol_block(double (*L)[NB + 1], double* colk, double* rd, int nb, DevStatus* st, int col_base,
                        bool report) {
  const int tid = threadIdx.x;
  __shared__ double s_r;
  for (int k = 0; k < nb; ++k) {
    if (tid == 0) {
      double p = L[k][k];
      if (!(p > 0.0) || !isfinite(p)) {
        if (report) raise_status(st, SKS_ERR_NOT_PD, 21, col_base + k);
        p = 1.0;
      }
      const double r = rsqrt_newton(p);
      s_r = r;
      rd[k] = r;
      L[k][k] = p * r;
    }
    for (int i = k + 1 + tid; i < nb; i += blockDim.x) colk[i] = L[i][k];
    __syncthreads();
    const double r = s_r, r2 = r * r;
    for (int i = k + 1 + tid; i < nb; i += blockDim.x) L[i][k] = colk[i] * r;
    {
      const int ty = tid >> 4, tx = tid & 15;
      for (int i = k + 1 + ty; i < nb; i += 16) {
        const double ci = colk[i] * r2;
        for (int j = k + 1 + tx; j <= i; j += 16) L[i][j] -= ci * colk[j];
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) potrf_diag_kernel(double* D, long long ld, int nb, double* Dinv, int col_base,
                                                        DevStatus* st) {
  __shared__ double L[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < NB * NB; e += blockDim.x) {
    const int i = e / NB, j = e % NB;
    L[i][j] = (i < nb && j < nb && j <= i) ? D[(long long)i * ld + j] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  __shared__ double colk[NB];
  __shared__ double rd[NB];
  chol_block(L, colk, rd, nb, st, col_base, true);
  // inverse of the lower-triangular L, row by row:
  //   X[i][j] = -(sum_{j <= q < i} L[i][q] X[q][j]) / L[i][i]  (j < i),  X[i][i] = 1 / L[i][i];
  // the 256 threads split each row's dots four ways (64 columns x 4 parts).
  __shared__ double part[4][NB];
  for (int e = tid; e < NB * NB; e += blockDim.x) X[e / NB][e % NB] = 0.0;
  __syncthreads();
  const int jj = tid & (NB - 1), pp = tid >> 6;
  __shared__ double rdiag[NB];
  if (tid < NB) rdiag[tid] = tid < nb ? rd[tid] : 1.0;
  __syncthreads();
  for (int i = 0; i < NB; ++i) {
    double acc = 0.0;
    if (jj < i)
      for (int q = jj + pp; q < i; q += 4) acc += L[i][q] * X[q][jj];
    part[pp][jj] = acc;
    __syncthreads();
    if (tid < NB) {
      const double inv = rdiag[i];
      if (tid < i) X[i][tid] = -((part[0][tid] + part[1][tid]) + (part[2][tid] + part[3][tid])) * inv;
      else if (tid == i) X[i][i] = inv;
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e / nb, j = e % nb;
    if (j <= i) D[(long long)i * ld + j] = L[i][j];
    else D[(long long)i * ld + j] = 0.0;
    Dinv[(long long)i * NB + j] = X[i][j];
  }
}

// One step of the blocked factorisation with the panel fused in: every CTA
// factors the nb x nb diagonal block (float64, in shared memory) and forms its
// inverse; CTA 0 writes L_kk (to Lout, NB x NB: the block in H is still being
// read by the other CTAs; the caller copies it back after the kernel) and
// L_kk^{-1}; CTA b >= 1 replaces its 64 rows of the panel below the block by
// P L_kk^{-T} in double-float arithmetic.  The diagonal work is repeated per
// CTA so that no launch waits for another.
template <typename T>
__global__ void transpose_kernel(int rows, int cols, const T* __restrict__ S, long long lds, T* __restrict__ D,
                                 long long ldd) {
  __shared__ T tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = by + k, c = bx + threadIdx.x;
    if (r < rows && c < cols) tile[k][threadIdx.x] = S[(long long)r * lds + c];
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int c = bx + k, r = by + threadIdx.x;
    if (r < rows && c < cols) D[(long long)c * ldd + r] = tile[threadIdx.x][k];
  }
}

__global__ void set_identity_scaled_kernel(int n, double* M, long long ld, double diag_add, const double* diag_vec,
                                           double vec_scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) M[(long long)i * ld + i] += diag_add + (diag_vec ? vec_scale * diag_vec[i] : 0.0);
}

// y_i = epilogue( alpha * sum_{j in range(i)} M[i][j] * (x_j / xdiv_j) )
// One warp per row; tri: 0 full, 1 lower (j <= i), 2 upper (j >= i).
// mode 0: y_i = v; mode 1: y_i = (z_i - v) / (nu2 * lam_i).
template <typename T>
__global__ void gemv_rows_kernel(int rows, int cols, const T* __restrict__ M, long long ldm, int tri,
                                 const double* __restrict__ x, const double* __restrict__ xdiv, double alpha,
                                 double* __restrict__ y, int mode, const double* __restrict__ z,
                                 const double* __restrict__ lam, double nu2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const int i = warp;
  int jlo = 0, jhi = cols;
  if (tri == 1) jhi = min(cols, i + 1);
  if (tri == 2) jlo = i;
  const T* row = M + (long long)i * ldm;
  double s = 0.0;
  for (int j = jlo + lane; j < jhi; j += 32) {
    const double xv = xdiv ? x[j] / xdiv[j] : x[j];
    s += (double)row[j] * xv;
  }
  s = warp_sum(s);
  if (lane == 0) {
    const double v = alpha * s;
    y[i] = (mode == 0) ? v : (z[i] - v) / (nu2 * lam[i]);
  }
}

}  // namespace

// ============================================================================ host

// float32 C = alpha * A B (both row-major, not transposed), batched over
// blockIdx.z: 128 x 128 tiles, K in steps of 8 through a double-buffered
// shared-memory pair, each of 256 threads keeping 8 x 8 outputs in registers
// (rows ty*4 + {0..3} and 64 + ty*4 + {0..3}, likewise the columns), so that a
// K step is four 16-byte shared loads per 64 FMAs.  a_lower / b_lower skip the
// K range a triangular operand makes zero.  Needs lda, ldb, ldc and every
// batch stride to be multiples of 4 floats and 16-byte aligned bases.
constexpr int SG_M = 128, SG_N = 128, SG_K = 8, SG_T = 256;
__global__ void __launch_bounds__(SG_T) sgemm128_kernel(int M, int N, int K, const float* __restrict__ A0,
                                                        long long lda, long long sA, const float* __restrict__ B0,
                                                        long long ldb, long long sB, float* __restrict__ C0,
                                                        long long ldc, long long sC, float alpha, int a_lower,
                                                        int b_lower) {
  __shared__ __align__(16) float As[2][SG_K][SG_M];
  __shared__ __align__(16) float Bs[2][SG_K][SG_N];
  const float* A = A0 + blockIdx.z * sA;
  const float* B = B0 + blockIdx.z * sB;
  float* C = C0 + blockIdx.z * sC;
  const int row0 = blockIdx.y * SG_M, col0 = blockIdx.x * SG_N;
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  int kb = 0, ke = K;
  if (a_lower) ke = min(K, row0 + SG_M);
  if (b_lower) kb = (min(col0, K) / SG_K) * SG_K;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  // loader roles: A: row tid/2, k (tid%2)*4 .. +4; B: k tid/32, columns (tid%32)*4 .. +4
  const int ar = tid >> 1, ak = (tid & 1) * 4;
  const int bk = tid >> 5, bn = (tid & 31) * 4;
  float4 ra, rb;
  auto load = [&](int k0) {
    const int gi = row0 + ar, gk = k0 + ak;
    ra = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gi < M) {
      if (gk + 3 < ke) ra = *reinterpret_cast<const float4*>(A + (long long)gi * lda + gk);
      else {
        float t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = gk + q < ke ? A[(long long)gi * lda + gk + q] : 0.f;
        ra = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
    const int gkb = k0 + bk, gj = col0 + bn;
    rb = make_float4(0.f, 0.f, 0.f, 0.f);
    if (gkb < ke) {
      if (gj + 3 < N) rb = *reinterpret_cast<const float4*>(B + (long long)gkb * ldb + gj);
      else {
        float t[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) t[q] = gj + q < N ? B[(long long)gkb * ldb + gj + q] : 0.f;
        rb = make_float4(t[0], t[1], t[2], t[3]);
      }
    }
  };
  auto store = [&](int buf) {
    As[buf][ak + 0][ar] = ra.x;
    As[buf][ak + 1][ar] = ra.y;
    As[buf][ak + 2][ar] = ra.z;
    As[buf][ak + 3][ar] = ra.w;
    *reinterpret_cast<float4*>(&Bs[buf][bk][bn]) = rb;
  };
  if (kb < ke) {
    load(kb);
    store(0);
  }
  __syncthreads();
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += SG_K) {
    const bool more = k0 + SG_K < ke;
    if (more) load(k0 + SG_K);  // in flight while this step computes
#pragma unroll
    for (int k = 0; k < SG_K; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gi = row0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
    if (gi >= M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gj = col0 + h * 64 + tx * 4;
      float* c = C + (long long)gi * ldc + gj;
      const float4 v = make_float4(alpha * acc[i][h * 4], alpha * acc[i][h * 4 + 1], alpha * acc[i][h * 4 + 2],
                                   alpha * acc[i][h * 4 + 3]);
      if (gj + 3 < N) *reinterpret_cast<float4*>(c) = v;
      else {
        const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (gj + q < N) c[q] = vv[q];
      }
    }
  }
}

template <typename T>
sks_status gemm(cudaStream_t stream, int M, int N, int K, const T* A, long long lda, bool ta, const T* B,
                long long ldb, bool tb, T* C, long long ldc, double alpha, double beta, bool lower, int batch,
                long long sA, long long sB, long long sC, T* split_ws, size_t split_ws_elems, int tri_ops) {
  if (M <= 0 || N <= 0 || batch <= 0) return SKS_OK;
  if constexpr (std::is_same<T, float>::value) {
    // the 128 x 128 register-blocked kernel: plain (not transposed) operands, C overwritten
    const bool al = ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0 && ((uintptr_t)C & 15) == 0 &&
                    lda % 4 == 0 && ldb % 4 == 0 && ldc % 4 == 0 && sA % 4 == 0 && sB % 4 == 0 && sC % 4 == 0;
    if (!ta && !tb && !lower && beta == 0.0 && al && K > 0 && M >= 64 && N >= 64) {
      const dim3 grid((unsigned)((N + SG_N - 1) / SG_N), (unsigned)((M + SG_M - 1) / SG_M), (unsigned)batch);
      sgemm128_kernel<<<grid, SG_T, 0, stream>>>(M, N, K, A, lda, sA, B, ldb, sB, C, ldc, sC, (float)alpha,
                                                 (tri_ops & 1) ? 1 : 0, (tri_ops & 2) ? 1 : 0);
      note_launch();
      SKS_CUDA_TRY(cudaGetLastError());
      return SKS_OK;
    }
  }
  GemmArgs<T> g;
  g.a_lower = (tri_ops & 1) ? 1 : 0;
  g.b_lower = (tri_ops & 2) ? 1 : 0;
  g.M = M; g.N = N; g.K = K;
  g.A = A; g.lda = lda; g.sA = sA; g.ta = ta;
  g.B = B; g.ldb = ldb; g.sB = sB; g.tb = tb;
  g.C = C; g.ldc = ldc; g.sC = sC;
  g.alpha = alpha; g.beta = beta; g.lower = lower; g.batch = batch;
  const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN) * batch;
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  int splits = 1;
  if (K > 0 && split_ws != nullptr) {
    // enough CTAs to cover the GPU twice, while each split keeps >= 256 of K
    while (tiles * splits < 2 * sms && K / (splits * 2) >= 256) splits *= 2;
    while (splits > 1 && (size_t)splits * batch * M * N > split_ws_elems) splits /= 2;
  }
  int kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  if (K <= 0) kchunk = 0;
  g.splits = splits;
  g.kchunk = kchunk;
  g.part = split_ws;
  dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch * splits);
  if (K <= 0) {
    // C = beta * C (alpha * 0)
    g.splits = 1;
    g.kchunk = 0;
    grid.z = batch;
  }
  gemm_kernel<T><<<grid, GT, 0, stream>>>(g);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  if (g.splits > 1) {
    dim3 rg((unsigned)std::min<long long>(4096, ((long long)M * N + 255) / 256), batch);
    split_reduce_kernel<T><<<rg, 256, 0, stream>>>(g);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  return SKS_OK;
}

template sks_status gemm<double>(cudaStream_t, int, int, int, const double*, long long, bool, const double*, long long,
                                 bool, double*, long long, double, double, bool, int, long long, long long, long long,
                                 double*, size_t, int);
template sks_status gemm<float>(cudaStream_t, int, int, int, const float*, long long, bool, const float*, long long,
                                bool, float*, long long, double, double, bool, int, long long, long long, long long,
                                float*, size_t, int);

template <typename T>
sks_status transpose(cudaStream_t stream, int rows, int cols, const T* S, long long lds, T* D, long long ldd) {
  if (rows <= 0 || cols <= 0) return SKS_OK;
  dim3 grid((cols + 31) / 32, (rows + 31) / 32);
  transpose_kernel<T><<<grid, dim3(32, 8), 0, stream>>>(rows, cols, S, lds, D, ldd);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}
template sks_status transpose<double>(cudaStream_t, int, int, const double*, long long, double*, long long);
template sks_status transpose<float>(cudaStream_t, int, int, const float*, long long, float*, long long);

sks_status add_diagonal(cudaStream_t stream, int n, double* M, long long ld, double diag_add, const double* diag_vec,
                        double vec_scale) {
  if (n <= 0) return SKS_OK;
  set_identity_scaled_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, M, ld, diag_add, diag_vec, vec_scale);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

size_t cholesky_ws_elems(int n) {
  // diagonal-block inverses + split-K partials of the trailing updates
  const int nblk = (n + NB - 1) / NB;
  return (size_t)nblk * NB * NB + (size_t)8 * n * NB + (size_t)n * n;
}

// In-place blocked right-looking Cholesky H = L L^T (lower; upper set to 0),
// then X = L^{-1} by recursive block inversion.  ws: cholesky_ws_elems(n).
sks_status cholesky_and_inverse(cudaStream_t stream, int n, double* H, long long ldh, double* X, long long ldx,
                                double* ws, DevStatus* st, float* ws32, int mode) {
  if (n <= 0) return SKS_OK;
  if (mode == kCholDf32InvF32 || mode == kCholDf32)
    return cholesky_inverse_df32(stream, n, H, ldh, X, ldx, ws, ws32, st, mode == kCholDf32InvF32);
  const int nblk = (n + NB - 1) / NB;
  double* dinv = ws;                              // nblk * NB * NB
  double* split = ws + (size_t)nblk * NB * NB;    // scratch for split-K
  const size_t split_elems = (size_t)8 * n * NB + (size_t)n * n;
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, nb = std::min(NB, n - k0);
    double* Dk = H + (long long)k0 * ldh + k0;
    double* Dinv = dinv + (size_t)kb * NB * NB;
    potrf_diag_kernel<<<1, 256, 0, stream>>>(Dk, ldh, nb, Dinv, k0, st);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    const int rest = n - k0 - nb;
    if (rest > 0) {
      double* P = H + (long long)(k0 + nb) * ldh + k0;  // panel below the block
      // panel <- panel * Dinv^T   (in place: one CTA column covers the nb columns)
      SKS_TRY(gemm<double>(stream, rest, nb, nb, P, ldh, false, Dinv, NB, true, split, nb, 1.0, 0.0, false, 1, 0, 0,
                           0, nullptr, 0));
      SKS_CUDA_TRY(cudaMemcpy2DAsync(P, ldh * sizeof(double), split, nb * sizeof(double), nb * sizeof(double), rest,
                                     cudaMemcpyDeviceToDevice, stream));
      // trailing lower update  T <- T - P P^T
      double* T = H + (long long)(k0 + nb) * ldh + (k0 + nb);
      SKS_TRY(gemm<double>(stream, rest, rest, nb, P, ldh, false, P, ldh, true, T, ldh, -1.0, 1.0, true, 1, 0, 0, 0,
                           nullptr, 0));
    }
  }
  // H now holds L in its lower triangle (the strict upper triangle outside the
  // diagonal blocks keeps old values and is never read).
  // X = L^{-1}: start with the diagonal-block inverses, then merge pairs.
  SKS_CUDA_TRY(cudaMemset2DAsync(X, ldx * sizeof(double), 0, n * sizeof(double), n, stream));
  for (int kb = 0; kb < nblk; ++kb) {
    const int k0 = kb * NB, nb = std::min(NB, n - k0);
    SKS_CUDA_TRY(cudaMemcpy2DAsync(X + (long long)k0 * ldx + k0, ldx * sizeof(double), dinv + (size_t)kb * NB * NB,
                                   NB * sizeof(double), nb * sizeof(double), nb, cudaMemcpyDeviceToDevice, stream));
  }
  // inv([A 0; B C]) = [A^-1 0; -C^-1 B A^-1  C^-1]
  for (int b = NB; b < n; b *= 2) {
    for (int r0 = 0; r0 + b < n; r0 += 2 * b) {
      const int n1 = b, n2 = std::min(b, n - r0 - b);
      const double* Binv_A = X + (long long)r0 * ldx + r0;          // A^{-1}: n1 x n1
      const double* Lb = H + (long long)(r0 + b) * ldh + r0;        // B: n2 x n1
      const double* Cinv = X + (long long)(r0 + b) * ldx + (r0 + b);  // C^{-1}: n2 x n2
      double* out = X + (long long)(r0 + b) * ldx + r0;             // n2 x n1
      double* tmp = split;                                          // n2 x n1
      const size_t rest_elems = split_elems - (size_t)n2 * n1;
      // A^{-1} and C^{-1} are lower triangular: half of each product's terms are skipped
      SKS_TRY(gemm<double>(stream, n2, n1, n1, Lb, ldh, false, Binv_A, ldx, false, tmp, n1, 1.0, 0.0, false, 1, 0, 0,
                           0, split + (size_t)n2 * n1, rest_elems, 2));
      SKS_TRY(gemm<double>(stream, n2, n1, n2, Cinv, ldx, false, tmp, n1, false, out, ldx, -1.0, 0.0, false, 1, 0, 0,
                           0, split + (size_t)n2 * n1, rest_elems, 1));
    }
  }
  return SKS_OK;
}

size_t cholesky_ws32_elems(int n) { return (size_t)4 * n * n + 64; }

template <typename T>
sks_status gemv_rows(cudaStream_t stream, int rows, int cols, const T* M, long long ldm, int tri, const double* x,
                     const double* xdiv, double alpha, double* y, int mode, const double* z, const double* lam,
                     double nu2) {
  if (rows <= 0) return SKS_OK;
  const int threads = 256;
  const int blocks = (rows * 32 + threads - 1) / threads;
  gemv_rows_kernel<T><<<blocks, threads, 0, stream>>>(rows, cols, M, ldm, tri, x, xdiv, alpha, y, mode, z, lam, nu2);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}
template sks_status gemv_rows<double>(cudaStream_t, int, int, const double*, long long, int, const double*,
                                      const double*, double, double*, int, const double*, const double*, double);
template sks_status gemv_rows<float>(cudaStream_t, int, int, const float*, long long, int, const double*,
                                     const double*, double, double*, int, const double*, const double*, double);

}  // namespace sks
