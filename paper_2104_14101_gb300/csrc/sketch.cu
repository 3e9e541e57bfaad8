// sketch.cu -- the random embeddings of Section 2.1 on the GPU.
//
//  K2 SRHT: B = H_{+-1} E A_pad (n_pad x d), the fast Walsh-Hadamard transform
//     along the rows of the sign-flipped, zero-padded A.  Butterflies pair
//     whole rows (r, r + h), so every pass holds 2^L rows x 32 contiguous
//     columns (lane = column) in registers and applies L <= 9 levels there,
//     with one shared-memory exchange; ceil(log2(n_pad) / 9) passes (8 for
//     float64) cover all levels.  Formed once per solve; a larger sketch only
//     gathers more rows of B.
//  K3 SRHT gather: Y[r] = B[pi(r)] for the new rows r, pi the keyed Feistel
//     permutation (nested subsampling R).
//  K4 Gaussian: Y[r] = sum_i G[r][i] a_i, G from Philox + Box-Muller, produced
//     chunk by chunk and multiplied with the CUDA-core GEMM (float64 form).
//  K5 SJLT: Y[h_k(i)] += sigma_k(i)/sqrt(s_eff) a_i, one warp per data row,
//     float64 atomics.
// All sketches are stored unscaled (S A = scale * Y).
#include <algorithm>

#include "sketch.h"
#include "dense.h"

namespace sks {

namespace {

constexpr int kFwhtCols = 32;  // one warp lane per column: 128-byte (float) row segments

// One FWHT pass over the row bits [a, a + L), L = LOGR + logw: the CTA
// (2^logw warps) owns the 2^L rows r(j) = hi * 2^(a+L) + j * 2^a + lo and the
// columns [c0, c0 + 32); lane c holds column c0 + c.
//   phase 1: warp w holds local rows j = w * 2^LOGR + i (i < 2^LOGR) in
//            registers and applies the levels on local bits [0, LOGR);
//   phase 2: after one exchange through shared memory, warp w holds rows
//            j = i * 2^logw + w and applies the levels on bits [LOGR, L)
//            (bits [LOGR - logw, LOGR) of i; logw <= LOGR).
// Levels of the transform commute, so their order is free.  The first pass
// reads A (rows >= n are zero) times the signs E.
template <typename T, int LOGR>
__global__ void __launch_bounds__(256, 2) fwht_pass_kernel(const T* __restrict__ A, long long lda, int64_t n,
                                                       T* __restrict__ B, long long ldb, int d, int a, int logw,
                                                       int first, Key key, int ncb) {
  constexpr int R = 1 << LOGR;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = LOGR + logw;
  T* tile = (T*)smem_raw;                                   // [2^L][32] (logw > 0)
  T* sign = tile + (logw > 0 ? ((size_t)kFwhtCols << L) : 0);  // [2^L], first pass only
  const int cb = blockIdx.x % ncb;
  const long long grp = blockIdx.x / ncb;
  const long long lo = grp & ((1ll << a) - 1);
  const long long hi = grp >> a;
  const long long base = (hi << (a + L)) + lo;
  const int w = threadIdx.x >> 5, c = threadIdx.x & 31;
  const int col = cb * kFwhtCols + c;
  const bool cok = col < d;
  if (first) {
    // one Philox evaluation per row of the tile, not per element
    for (int j = threadIdx.x; j < (1 << L); j += blockDim.x) {
      const long long r = base + ((long long)j << a);
      sign[j] = (r < n) ? (T)srht_sign(key, (uint32_t)r) : T(0);
    }
    __syncthreads();
  }
  T v[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = w * R + i;
    const long long r = base + ((long long)j << a);
    T x = T(0);
    if (first) {
      if (cok && r < n) x = A[r * lda + col] * sign[j];
    } else if (cok) {
      x = B[r * ldb + col];
    }
    v[i] = x;
  }
#pragma unroll
  for (int h = 1; h < R; h <<= 1)
#pragma unroll
    for (int i = 0; i < R; ++i)
      if (!(i & h)) {
        const T u = v[i], z = v[i + h];
        v[i] = u + z;
        v[i + h] = u - z;
      }
  if (logw > 0) {
#pragma unroll
    for (int i = 0; i < R; ++i) tile[(size_t)(w * R + i) * kFwhtCols + c] = v[i];
    __syncthreads();
    const int W = 1 << logw;
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = tile[(size_t)(i * W + w) * kFwhtCols + c];
#pragma unroll
    for (int b = 0; b < LOGR; ++b) {
      if (b < LOGR - logw) continue;
      const int h = 1 << b;
#pragma unroll
      for (int i = 0; i < R; ++i)
        if (!(i & h)) {
          const T u = v[i], z = v[i + h];
          v[i] = u + z;
          v[i + h] = u - z;
        }
    }
    if (cok)
#pragma unroll
      for (int i = 0; i < R; ++i) B[(base + ((long long)(i * W + w) << a)) * ldb + col] = v[i];
  } else if (cok) {
#pragma unroll
    for (int i = 0; i < R; ++i) B[(base + ((long long)i << a)) * ldb + col] = v[i];
  }
}

template <typename T, int LOGR>
sks_status fwht_launch(cudaStream_t stream, const T* A, long long lda, int64_t n, T* B, long long ldb, int d, int a,
                       int logw, int bits, int first, Key key) {
  const int L = LOGR + logw;
  const int ncb = (d + kFwhtCols - 1) / kFwhtCols;
  const long long blocks = (1ll << (bits - L)) * ncb;
  if (blocks > 0x7fffffffll) return fail(SKS_ERR_UNSUPPORTED, "FWHT grid too large");
  const size_t smem = (logw > 0 ? ((size_t)kFwhtCols << L) * sizeof(T) : 0) + (first ? ((size_t)1 << L) * sizeof(T) : 0);
  SKS_CUDA_TRY(cudaFuncSetAttribute(fwht_pass_kernel<T, LOGR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  fwht_pass_kernel<T, LOGR><<<(unsigned)blocks, 32 << logw, smem, stream>>>(A, lda, n, B, ldb, d, a, logw, first,
                                                                           key, ncb);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

// Y[r] = B[pi(r)] for r in [r0, r1); one CTA per row.
template <typename TB, typename TY>
__global__ void srht_gather_kernel(const TB* __restrict__ B, long long ldb, int d, int bits, Key key, int r0,
                                   TY* __restrict__ Y, long long ldy, DevStatus* st) {
  const int r = r0 + blockIdx.x;
  __shared__ uint32_t src;
  if (threadIdx.x == 0) {
    src = feistel_perm(key, (uint32_t)r, bits);
    if (src == 0xffffffffu) raise_status(st, SKS_ERR_NUMERIC, 31, r);
  }
  __syncthreads();
  if (src == 0xffffffffu) return;
  const TB* row = B + (long long)src * ldb;
  TY* out = Y + (long long)r * ldy;
  for (int c = threadIdx.x; c < d; c += blockDim.x) out[c] = (TY)row[c];
}

// G[r][i] (r < m_add, i < icnt) = N(0,1) entry of global sketch row m_off + r
// and data row i0 + i; one thread per (quad, data row).
template <typename T>
__global__ void gauss_gen_kernel(Key key, int m_off, int m_add, int64_t i0, int icnt, T* __restrict__ G,
                                 long long ldg) {
  const int q0 = m_off / 4;
  const int q1 = (m_off + m_add - 1) / 4;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nq = (long long)(q1 - q0 + 1);
  if (e >= nq * icnt) return;
  const int i = (int)(e % icnt);
  const int q = q0 + (int)(e / icnt);
  T g[4];
  if (sizeof(T) == 8) {
    double gd[4];
    gauss4_d(key, (uint32_t)(i0 + i), (uint32_t)q, gd);
    for (int t = 0; t < 4; ++t) g[t] = (T)gd[t];
  } else {
    float gf[4];
    gauss4_f(key, (uint32_t)(i0 + i), (uint32_t)q, gf);
    for (int t = 0; t < 4; ++t) g[t] = (T)gf[t];
  }
  for (int t = 0; t < 4; ++t) {
    const int rg = 4 * q + t;
    if (rg >= m_off && rg < m_off + m_add) G[(long long)(rg - m_off) * ldg + i] = g[t];
  }
}

// SJLT scatter: one warp per data row; float32 sketches add 16-byte vectors
// with one atomic each (4x fewer L2 atomic operations than scalar adds).
template <typename TA, typename TY>
__global__ void sjlt_scatter_kernel(const TA* __restrict__ A, long long lda, int64_t n, int d, uint32_t m, int s_eff,
                                    Key key, TY* __restrict__ Y, long long ldy) {
  const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n) return;
  uint32_t rows[kSjltMaxS];
  float signs[kSjltMaxS];
  sjlt_hash(key, (uint32_t)warp, m, s_eff, rows, signs);
  const TY inv = (TY)(1.0 / sqrt((double)s_eff));
  const TA* a = A + warp * lda;
  if (sizeof(TY) == 4 && sizeof(TA) == 4 && (d & 3) == 0 && (lda & 3) == 0 && (ldy & 3) == 0) {
    for (int c = lane * 4; c < d; c += 128) {
      const float4 v = __ldcs((const float4*)(a + c));  // streamed once: evict first, keep Y in L2
      for (int k = 0; k < s_eff; ++k) {
        const float w = signs[k] * (float)inv;
        atomicAdd((float4*)(Y + (long long)rows[k] * ldy + c), make_float4(w * v.x, w * v.y, w * v.z, w * v.w));
      }
    }
    return;
  }
  for (int c = lane; c < d; c += 32) {
    const TY v = (TY)__ldcs(a + c) * inv;
    for (int k = 0; k < s_eff; ++k) atomicAdd(&Y[(long long)rows[k] * ldy + c], (TY)signs[k] * v);
  }
}

// Small sketches (m * d fits in shared memory): every CTA accumulates its
// rows into a private copy of Y and flushes it with one atomic per entry.
template <typename TA, typename TY>
__global__ void __launch_bounds__(256) sjlt_private_kernel(const TA* __restrict__ A, long long lda, int64_t n, int d,
                                                          uint32_t m, int s_eff, Key key, TY* __restrict__ Y,
                                                          long long ldy, int64_t rows_per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TY* Ys = (TY*)smem_raw;  // m x d
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < (int)m * d; e += blockDim.x) Ys[e] = TY(0);
  __syncthreads();
  const TY inv = (TY)(1.0 / sqrt((double)s_eff));
  const int64_t r0 = blockIdx.x * rows_per_cta;
  const int64_t r1 = min(n, r0 + rows_per_cta);
  for (int64_t i = r0 + warp; i < r1; i += blockDim.x / 32) {
    uint32_t rows[kSjltMaxS];
    float signs[kSjltMaxS];
    sjlt_hash(key, (uint32_t)i, m, s_eff, rows, signs);
    const TA* a = A + i * lda;
    for (int c = lane; c < d; c += 32) {
      const TY v = (TY)a[c] * inv;
      for (int k = 0; k < s_eff; ++k) atomicAdd(&Ys[rows[k] * d + c], (TY)signs[k] * v);
    }
  }
  __syncthreads();
  for (int e = tid; e < (int)m * d; e += blockDim.x) {
    const int r = e / d, c = e % d;
    atomicAdd(&Y[(long long)r * ldy + c], Ys[e]);
  }
}

}  // namespace

int ilog2_ceil(int64_t n) {
  int b = 0;
  while ((1ll << b) < n) ++b;
  return b;
}

template <typename T>
sks_status srht_form(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, T* B, long long ldb,
                     uint64_t seed) {
  const int bits = ilog2_ceil(n);
  // levels per pass: up to 2^6 (float) / 2^5 (float64) rows per thread in
  // registers times up to 8 warps; passes balanced in size
  constexpr int kLogRMax = sizeof(T) == 4 ? 6 : 5;
  constexpr int kLMax = kLogRMax + 3;
  const int passes = bits == 0 ? 1 : (bits + kLMax - 1) / kLMax;
  const Key key = make_key(seed);
  int a = 0;
  for (int p = 0; p < passes; ++p) {
    const int L = bits / passes + (p < bits % passes ? 1 : 0);
    const int logw = std::min(3, L / 2);
    const int logr = L - logw;
    const int first = p == 0 ? 1 : 0;
    sks_status st;
    switch (logr) {
      case 0: st = fwht_launch<T, 0>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      case 1: st = fwht_launch<T, 1>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      case 2: st = fwht_launch<T, 2>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      case 3: st = fwht_launch<T, 3>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      case 4: st = fwht_launch<T, 4>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      case 5: st = fwht_launch<T, 5>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key); break;
      default: st = fwht_launch<T, (sizeof(T) == 4 ? 6 : 5)>(stream, A, lda, n, B, ldb, d, a, logw, bits, first, key);
    }
    if (st != SKS_OK) return st;
    a += L;
  }
  return SKS_OK;
}
template sks_status srht_form<double>(cudaStream_t, const double*, long long, int64_t, int, double*, long long,
                                      uint64_t);
template sks_status srht_form<float>(cudaStream_t, const float*, long long, int64_t, int, float*, long long, uint64_t);

template <typename TB, typename TY>
sks_status srht_gather(cudaStream_t stream, const TB* B, long long ldb, int d, int64_t n_pad, uint64_t seed, int r0,
                       int r1, TY* Y, long long ldy, DevStatus* st) {
  if (r1 <= r0) return SKS_OK;
  const int bits = ilog2_ceil(n_pad);
  srht_gather_kernel<TB, TY><<<r1 - r0, 128, 0, stream>>>(B, ldb, d, bits, make_key(seed), r0, Y, ldy, st);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}
template sks_status srht_gather<double, double>(cudaStream_t, const double*, long long, int, int64_t, uint64_t, int,
                                                int, double*, long long, DevStatus*);
template sks_status srht_gather<float, float>(cudaStream_t, const float*, long long, int, int64_t, uint64_t, int, int,
                                              float*, long long, DevStatus*);

template <typename T>
sks_status gaussian_extend(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, uint64_t seed, int m_off,
                           int m_add, T* Y, long long ldy, T* gbuf, size_t gbuf_elems, T* split_ws,
                           size_t split_elems) {
  if (m_add <= 0) return SKS_OK;
  if (n == 0) {
    SKS_CUDA_TRY(cudaMemset2DAsync(Y + (long long)m_off * ldy, ldy * sizeof(T), 0, d * sizeof(T), m_add, stream));
    return SKS_OK;
  }
  int64_t chunk = (int64_t)(gbuf_elems / (size_t)m_add);
  chunk = std::min<int64_t>(chunk, n);
  if (chunk < 1) return fail(SKS_ERR_WORKSPACE, "Gaussian sketch buffer too small");
  const Key key = make_key(seed);
  for (int64_t i0 = 0; i0 < n; i0 += chunk) {
    const int icnt = (int)std::min<int64_t>(chunk, n - i0);
    const long long nq = (m_off + m_add - 1) / 4 - m_off / 4 + 1;
    const long long threads = nq * icnt;
    gauss_gen_kernel<T><<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(key, m_off, m_add, i0, icnt, gbuf,
                                                                                icnt);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    SKS_TRY(gemm<T>(stream, m_add, d, icnt, gbuf, icnt, false, A + i0 * lda, lda, false, Y + (long long)m_off * ldy,
                    ldy, 1.0, i0 == 0 ? 0.0 : 1.0, false, 1, 0, 0, 0, split_ws, split_elems));
  }
  return SKS_OK;
}
template sks_status gaussian_extend<double>(cudaStream_t, const double*, long long, int64_t, int, uint64_t, int, int,
                                            double*, long long, double*, size_t, double*, size_t);
template sks_status gaussian_extend<float>(cudaStream_t, const float*, long long, int64_t, int, uint64_t, int, int,
                                           float*, long long, float*, size_t, float*, size_t);

template <typename TA, typename TY>
sks_status sjlt_form(cudaStream_t stream, const TA* A, long long lda, int64_t n, int d, int m, int s, uint64_t seed,
                     TY* Y, long long ldy) {
  SKS_CUDA_TRY(cudaMemset2DAsync(Y, ldy * sizeof(TY), 0, d * sizeof(TY), m, stream));
  if (n == 0) return SKS_OK;
  const int s_eff = std::min(s, m);
  if (s_eff > kSjltMaxS) return fail(SKS_ERR_UNSUPPORTED, "SJLT s > 16");
  const size_t priv_bytes = (size_t)m * d * sizeof(TY);
  if (priv_bytes <= 96 * 1024) {
    const int sms = device_info().sms > 0 ? device_info().sms : 152;
    const int64_t ctas = std::min<int64_t>((int64_t)sms * 2, (n + 255) / 256);
    const int64_t per = (n + ctas - 1) / ctas;
    SKS_CUDA_TRY(cudaFuncSetAttribute(sjlt_private_kernel<TA, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)priv_bytes));
    sjlt_private_kernel<TA, TY><<<(unsigned)ctas, 256, priv_bytes, stream>>>(A, lda, n, d, (uint32_t)m, s_eff,
                                                                          make_key(seed), Y, ldy, per);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    return SKS_OK;
  }
  const long long threads = n * 32;
  sjlt_scatter_kernel<TA, TY><<<(unsigned)((threads + 255) / 256), 256, 0, stream>>>(A, lda, n, d, (uint32_t)m, s_eff,
                                                                                    make_key(seed), Y, ldy);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}
template sks_status sjlt_form<double, double>(cudaStream_t, const double*, long long, int64_t, int, int, int, uint64_t,
                                              double*, long long);
template sks_status sjlt_form<float, float>(cudaStream_t, const float*, long long, int64_t, int, int, int, uint64_t,
                                            float*, long long);

}  // namespace sks
