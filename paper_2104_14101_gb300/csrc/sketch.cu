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
//  K5 SJLT: Y[h_k(i)] += sigma_k(i)/sqrt(s_eff) a_i, one warp per (data row,
//     512-column block), column blocks in sequence so the live part of Y
//     stays in L2; small sketches accumulate in shared memory first.
// All sketches are stored unscaled (S A = scale * Y).
#include <algorithm>
#include <type_traits>

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
                                 long long ldg, int rade) {
  const int q0 = m_off / 4;
  const int q1 = (m_off + m_add - 1) / 4;
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nq = (long long)(q1 - q0 + 1);
  if (e >= nq * icnt) return;
  const int i = (int)(e % icnt);
  const int q = q0 + (int)(e / icnt);
  T g[4];
  if (rade) {
    float gf[4];
    rade4_f(key, (uint32_t)(i0 + i), (uint32_t)q, gf);
    for (int t = 0; t < 4; ++t) g[t] = (T)gf[t];
  } else if (sizeof(T) == 8) {
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

// SJLT scatter, tiled by column blocks: warp = one data row x one block of
// kSjltCols columns, and the grid walks all rows of one column block before
// the next, so the live part of Y (m x kSjltCols) stays in L2 while the
// atomics land.  float32 sketches add 16-byte vectors with one atomic each.
constexpr int kSjltCols = 512;
template <typename TA, typename TY>
__global__ void __launch_bounds__(256) sjlt_scatter_kernel(const TA* __restrict__ A, long long lda, int64_t n, int d,
                                                          uint32_t m, int s_eff, Key key, TY* __restrict__ Y,
                                                          long long ldy, long long row_blocks) {
  const long long cb = blockIdx.x / row_blocks;
  const long long i = (blockIdx.x - cb * row_blocks) * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (i >= n) return;
  uint32_t rows[kSjltMaxS];
  float signs[kSjltMaxS];
  sjlt_hash(key, (uint32_t)i, m, s_eff, rows, signs);
  const TY inv = (TY)(1.0 / sqrt((double)s_eff));
  const TA* a = A + i * lda;
  const int c0 = (int)cb * kSjltCols;
  const int c1 = min(d, c0 + kSjltCols);
  if (sizeof(TY) == 4 && sizeof(TA) == 4 && (d & 3) == 0 && (lda & 3) == 0 && (ldy & 3) == 0) {
#pragma unroll 4
    for (int c = c0 + lane * 4; c < c1; c += 128) {
      const float4 v = __ldcs((const float4*)(a + c));  // streamed once: evict first, keep Y in L2
#pragma unroll
      for (int k = 0; k < kSjltMaxS; ++k) {
        if (k >= s_eff) break;
        const float w = signs[k] * (float)inv;
        atomicAdd((float4*)(Y + (long long)rows[k] * ldy + c), make_float4(w * v.x, w * v.y, w * v.z, w * v.w));
      }
    }
    return;
  }
  for (int c = c0 + lane; c < c1; c += 32) {
    const TY v = (TY)__ldcs(a + c) * inv;
#pragma unroll
    for (int k = 0; k < kSjltMaxS; ++k) {
      if (k >= s_eff) break;
      atomicAdd(&Y[(long long)rows[k] * ldy + c], (TY)signs[k] * v);
    }
  }
}

// ---------------------------------------------------------------- SJLT by gathering (larger m, float64)
// The scatter moves s n d additions through L2 read-modify-writes (for float64
// one 8-byte atomic each, there being no vector float64 atomics).  Instead:
// (1) count the data rows hashed to every sketch row, (2) scan the counts into
// bucket offsets, (3) fill each bucket with its data rows (index | sign bit)
// by atomic cursors -- a grid-stride walk keeps the buckets nearly sorted by
// row, (4) one warp per chunk of the bucket-ordered entries sums its rows of
// A for one column block in registers and adds the sum into its sketch row
// when the bucket changes (a few vector atomics per chunk).  All chunks of a
// column block run in one wave and walk the data rows at the same pace, so
// the s readers of a row segment of A meet in L2 and A leaves HBM about once.
constexpr int kSjGatherWarps = 8;

__global__ void sjlt_count_kernel(int64_t n, uint32_t m, int s_eff, Key key, uint32_t* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rows[kSjltMaxS];
    float sg[kSjltMaxS];
    sjlt_hash(key, (uint32_t)i, m, s_eff, rows, sg);
    for (int k = 0; k < s_eff; ++k) atomicAdd(&counts[rows[k]], 1u);
  }
}

// offsets[r] = sum_{q < r} counts[q] (offsets[m] = total); cursor = offsets
// (cursor may alias counts: each count is read before its slot is overwritten)
__global__ void __launch_bounds__(1024) sjlt_scan_kernel(uint32_t m, const uint32_t* counts, uint32_t* offsets,
                                                         uint32_t* cursor) {
  __shared__ uint32_t part[1024];
  const uint32_t t = threadIdx.x;
  const uint32_t per = (m + 1023) / 1024;
  const uint32_t q0 = min(m, t * per), q1 = min(m, q0 + per);
  uint32_t sum = 0;
  for (uint32_t q = q0; q < q1; ++q) sum += counts[q];
  part[t] = sum;
  __syncthreads();
  for (uint32_t off = 1; off < 1024; off <<= 1) {  // inclusive scan of the 1024 partial sums
    const uint32_t v = t >= off ? part[t - off] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t run = t == 0 ? 0u : part[t - 1];
  for (uint32_t q = q0; q < q1; ++q) {
    const uint32_t cq = counts[q];
    offsets[q] = run;
    cursor[q] = run;
    run += cq;
  }
  if (t == 1023) offsets[m] = part[1023];
}

__global__ void sjlt_fill_kernel(int64_t n, uint32_t m, int s_eff, Key key, uint32_t* __restrict__ cursor,
                                 uint32_t* __restrict__ entries) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t rows[kSjltMaxS];
    float sg[kSjltMaxS];
    sjlt_hash(key, (uint32_t)i, m, s_eff, rows, sg);
    for (int k = 0; k < s_eff; ++k) {
      const uint32_t pos = atomicAdd(&cursor[rows[k]], 1u);
      entries[pos] = (uint32_t)i | (sg[k] < 0.f ? 0x80000000u : 0u);
    }
  }
}

template <typename T>
SKS_DEV void sj_flush(T* Y, long long ldy, uint32_t r, int c, const T* acc, T scale);
template <>
SKS_DEV void sj_flush<float>(float* Y, long long ldy, uint32_t r, int c, const float* acc, float scale) {
  atomicAdd((float4*)(Y + (long long)r * ldy + c),
            make_float4(acc[0] * scale, acc[1] * scale, acc[2] * scale, acc[3] * scale));
}
template <>
SKS_DEV void sj_flush<double>(double* Y, long long ldy, uint32_t r, int c, const double* acc, double scale) {
  atomicAdd(Y + (long long)r * ldy + c, acc[0] * scale);
  atomicAdd(Y + (long long)r * ldy + c + 1, acc[1] * scale);
}

// task = (column block of 32 * 16 bytes, chunk of `chunk` entries), column block major
template <typename T>
__global__ void __launch_bounds__(kSjGatherWarps * 32) sjlt_gather_kernel(
    const T* __restrict__ A, long long lda, int d, const uint32_t* __restrict__ entries,
    const uint32_t* __restrict__ offsets, uint32_t m, long long total, long long chunk, long long chunks, T scale,
    T* __restrict__ Y, long long ldy) {
  constexpr int kVec = 16 / (int)sizeof(T);
  constexpr int kW = 32 * kVec;  // columns per block
  constexpr int kU = 8;          // entries in flight per warp
  using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long task = (long long)blockIdx.x * kSjGatherWarps + warp;
  const long long cb = task / chunks;
  const long long e0 = (task - cb * chunks) * chunk;
  const long long e1 = min(total, e0 + chunk);
  if ((long long)cb * kW >= d || e0 >= e1) return;
  const int c = (int)cb * kW + lane * kVec;
  const bool cok = c < d;  // d is a multiple of kVec: a lane's vector is whole or absent
  // the bucket holding entry e0: the last r with offsets[r] <= e0
  uint32_t lo = 0, hi = m;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if ((long long)offsets[mid] <= e0) lo = mid;
    else hi = mid;
  }
  uint32_t r = lo;
  long long rend = offsets[r + 1];
  T acc[kVec];
#pragma unroll
  for (int t = 0; t < kVec; ++t) acc[t] = T(0);
  for (long long e = e0; e < e1; e += 32) {
    const int cnt = (int)min(32ll, e1 - e);
    const uint32_t mine = lane < cnt ? entries[e + lane] : 0u;
    for (int j0 = 0; j0 < cnt; j0 += kU) {
      V v[kU];
      uint32_t ent[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        ent[u] = __shfl_sync(0xffffffffu, mine, (j0 + u) & 31);
        if (cok && j0 + u < cnt) v[u] = __ldcs((const V*)(A + (long long)(ent[u] & 0x7fffffffu) * lda + c));
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        if (j0 + u >= cnt) break;
        const long long ee = e + j0 + u;
        while (ee >= rend) {  // warp-uniform: the entry belongs to a later bucket
          if (cok) sj_flush<T>(Y, ldy, r, c, acc, scale);
#pragma unroll
          for (int t = 0; t < kVec; ++t) acc[t] = T(0);
          ++r;
          rend = offsets[r + 1];
        }
        if (cok) {
          const T sg = (ent[u] >> 31) ? T(-1) : T(1);
          const T* vv = (const T*)&v[u];
#pragma unroll
          for (int t = 0; t < kVec; ++t) acc[t] = fma(sg, vv[t], acc[t]);
        }
      }
    }
  }
  if (cok) sj_flush<T>(Y, ldy, r, c, acc, scale);
}

template <typename T>
sks_status sjlt_gather_launch(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, int m, int s_eff,
                              uint64_t seed, T* Y, long long ldy, uint32_t* ws) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  uint32_t* counts = ws;
  uint32_t* offsets = ws + (m + 1);
  uint32_t* entries = ws + 2 * (size_t)(m + 1);
  const Key key = make_key(seed);
  SKS_CUDA_TRY(cudaMemsetAsync(counts, 0, (size_t)(m + 1) * sizeof(uint32_t), stream));
  sjlt_count_kernel<<<sms * 4, 256, 0, stream>>>(n, (uint32_t)m, s_eff, key, counts);
  note_launch();
  sjlt_scan_kernel<<<1, 1024, 0, stream>>>((uint32_t)m, counts, offsets, counts);
  note_launch();
  // one CTA per SM walks the rows in grid-stride order: the buckets fill in nearly ascending row order
  sjlt_fill_kernel<<<sms, 256, 0, stream>>>(n, (uint32_t)m, s_eff, key, counts, entries);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  constexpr int kW = 32 * (16 / (int)sizeof(T));
  const long long total = (long long)n * s_eff;
  const long long ncb = (d + kW - 1) / kW;
  // a column block's chunks fit in one wave of resident warps
  int per_sm = 0;
  SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sjlt_gather_kernel<T>, kSjGatherWarps * 32, 0));
  const long long wave = (long long)sms * std::max(1, per_sm) * kSjGatherWarps;
  const long long chunk = std::max<long long>(256, (total + wave - 1) / wave);
  const long long chunks = (total + chunk - 1) / chunk;
  const long long blocks = (ncb * chunks + kSjGatherWarps - 1) / kSjGatherWarps;
  if (blocks > 0x7fffffffll) return fail(SKS_ERR_UNSUPPORTED, "SJLT grid too large");
  sjlt_gather_kernel<T><<<(unsigned)blocks, kSjGatherWarps * 32, 0, stream>>>(
      A, lda, d, entries, offsets, (uint32_t)m, total, chunk, chunks, (T)(1.0 / std::sqrt((double)s_eff)), Y, ldy);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

// Small sketches (m rows of a column block fit in shared memory): the CTA
// owns a block of 256 * VEC columns and a contiguous chunk of data rows;
// thread t owns columns [t * VEC, t * VEC + VEC) of every one of the m partial
// rows, so it accumulates without atomics.  The hashes of 256 rows at a time
// are formed once into shared memory; the partial rows are flushed with one
// (vector) atomic per entry at the end.
template <typename T, int VEC>
struct SjVec;
template <>
struct SjVec<float, 4> {
  using V = float4;
  static SKS_DEV V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static SKS_DEV void axpy(V& y, float w, const V& x) {
    y.x += w * x.x;
    y.y += w * x.y;
    y.z += w * x.z;
    y.w += w * x.w;
  }
  static SKS_DEV void flush(float* dst, const V& v) { atomicAdd((float4*)dst, v); }
};
template <>
struct SjVec<float, 2> {
  using V = float2;
  static SKS_DEV V zero() { return make_float2(0.f, 0.f); }
  static SKS_DEV void axpy(V& y, float w, const V& x) {
    y.x += w * x.x;
    y.y += w * x.y;
  }
  static SKS_DEV void flush(float* dst, const V& v) { atomicAdd((float2*)dst, v); }
};
template <>
struct SjVec<float, 1> {
  using V = float;
  static SKS_DEV V zero() { return 0.f; }
  static SKS_DEV void axpy(V& y, float w, const V& x) { y += w * x; }
  static SKS_DEV void flush(float* dst, const V& v) { atomicAdd(dst, v); }
};
template <>
struct SjVec<double, 2> {
  using V = double2;
  static SKS_DEV V zero() { return make_double2(0.0, 0.0); }
  static SKS_DEV void axpy(V& y, double w, const V& x) {
    y.x += w * x.x;
    y.y += w * x.y;
  }
  static SKS_DEV void flush(double* dst, const V& v) {
    atomicAdd(dst, v.x);
    atomicAdd(dst + 1, v.y);
  }
};
template <>
struct SjVec<double, 1> {
  using V = double;
  static SKS_DEV V zero() { return 0.0; }
  static SKS_DEV void axpy(V& y, double w, const V& x) { y += w * x; }
  static SKS_DEV void flush(double* dst, const V& v) { atomicAdd(dst, v); }
};

constexpr int kSjBlockThreads = 256;

// Small and medium sketches: the CTA owns a block of 256 * VEC columns and a
// contiguous chunk of data rows; thread t owns columns [t * VEC, t * VEC + VEC)
// of every one of the m partial rows (shared memory), so it accumulates
// without atomics.  The hashes of 256 rows at a time are formed once into
// shared memory; the partial rows are flushed with one (vector) atomic per
// entry at the end.  VEC shrinks as m grows so that m partial rows fit.
template <typename T, int VEC>
__global__ void __launch_bounds__(kSjBlockThreads) sjlt_block_kernel(const T* __restrict__ A, long long lda, int64_t n,
                                                                    int d, uint32_t m, int s_eff, Key key,
                                                                    T* __restrict__ Y, long long ldy, int ncb,
                                                                    int64_t rows_per_cta) {
  using SV = SjVec<T, VEC>;
  using V = typename SV::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  V* Ys = (V*)smem_raw;                                                   // [m][256]
  uint32_t* hrow = (uint32_t*)(Ys + (size_t)m * kSjBlockThreads);          // [256][s_eff]
  float* hsgn = (float*)(hrow + (size_t)kSjBlockThreads * s_eff);          // [256][s_eff]
  const int tid = threadIdx.x;
  const int cb = blockIdx.x % ncb;
  const int64_t r0 = (int64_t)(blockIdx.x / ncb) * rows_per_cta;
  const int64_t r1 = min(n, r0 + rows_per_cta);
  const int c = cb * kSjBlockThreads * VEC + tid * VEC;
  const bool cok = c < d;
  for (uint32_t h = 0; h < m; ++h) Ys[(size_t)h * kSjBlockThreads + tid] = SV::zero();
  const T inv = (T)(1.0 / sqrt((double)s_eff));
  for (int64_t base = r0; base < r1; base += kSjBlockThreads) {
    __syncthreads();  // previous batch's hashes fully consumed
    if (base + tid < r1) {
      uint32_t rows[kSjltMaxS];
      float signs[kSjltMaxS];
      sjlt_hash(key, (uint32_t)(base + tid), m, s_eff, rows, signs);
      for (int k = 0; k < s_eff; ++k) {
        hrow[tid * s_eff + k] = rows[k];
        hsgn[tid * s_eff + k] = signs[k];
      }
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kSjBlockThreads, r1 - base);
    if (!cok) continue;
    const T* a = A + base * lda + c;
#pragma unroll 8
    for (int j = 0; j < cnt; ++j) {
      const V v = *(const V*)(a + (int64_t)j * lda);
      for (int k = 0; k < s_eff; ++k) {
        V& y = Ys[(size_t)hrow[j * s_eff + k] * kSjBlockThreads + tid];
        SV::axpy(y, (T)hsgn[j * s_eff + k] * inv, v);
      }
    }
  }
  if (!cok) return;
  for (uint32_t h = 0; h < m; ++h) SV::flush(Y + (long long)h * ldy + c, Ys[(size_t)h * kSjBlockThreads + tid]);
}

// Small m, float32 (m <= MR <= 32): the m partial rows of the thread's VEC
// columns live in registers.  For a batch of 256 data rows every thread
// expands one row's hash into a dense coefficient row w[MR] (the scaled
// sign at the s_eff hashed rows, 0 elsewhere) in shared memory; then each data
// row costs one load and MR * VEC FMAs against the broadcast w row, instead
// of s_eff read-modify-writes of shared memory.  Flushed with one vector
// atomic per partial row at the end.
constexpr int kSjRegThreads = 256;
template <int MR, int VEC>
__global__ void __launch_bounds__(kSjRegThreads, MR <= 8 ? 3 : (MR <= 16 ? 2 : 1))
    sjlt_reg_kernel(const float* __restrict__ A, long long lda, int64_t n, int d, uint32_t m, int s_eff, Key key,
                    float* __restrict__ Y, long long ldy, int ncb, int64_t rows_per_cta) {
  using V = typename std::conditional<VEC == 4, float4, float2>::type;
  constexpr int kBatch = MR <= 32 ? 256 : 128;  // data rows hashed per batch (w: <= 32 KB)
  __shared__ __align__(16) float w[kBatch][MR];
  const int tid = threadIdx.x;
  const int cb = blockIdx.x % ncb;
  const int64_t r0 = (int64_t)(blockIdx.x / ncb) * rows_per_cta;
  const int64_t r1 = min(n, r0 + rows_per_cta);
  const int c = cb * kSjRegThreads * VEC + tid * VEC;
  const bool cok = c < d;
  float acc[MR][VEC];
#pragma unroll
  for (int r = 0; r < MR; ++r)
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[r][e] = 0.f;
  const float inv = (float)(1.0 / sqrt((double)s_eff));
  for (int64_t base = r0; base < r1; base += kBatch) {
    __syncthreads();  // the previous batch's coefficient rows are consumed
    if (tid < kBatch) {
      float wr[MR];
#pragma unroll
      for (int r = 0; r < MR; ++r) wr[r] = 0.f;
      if (base + tid < r1) {
        uint32_t rows[kSjltMaxS];
        float signs[kSjltMaxS];
        sjlt_hash(key, (uint32_t)(base + tid), m, s_eff, rows, signs);
        for (int k = 0; k < s_eff; ++k)
#pragma unroll
          for (int r = 0; r < MR; ++r)
            if (rows[k] == (uint32_t)r) wr[r] = signs[k] * inv;
      }
#pragma unroll
      for (int r = 0; r < MR; r += 4) *(float4*)&w[tid][r] = make_float4(wr[r], wr[r + 1], wr[r + 2], wr[r + 3]);
    }
    __syncthreads();
    const int cnt = (int)min((int64_t)kBatch, r1 - base);
    if (!cok) continue;
    const float* a = A + base * lda + c;
#pragma unroll 8
    for (int j = 0; j < cnt; ++j) {
      const V v = __ldcs((const V*)(a + (int64_t)j * lda));
      const float* vv = (const float*)&v;
#pragma unroll
      for (int r = 0; r < MR; r += 4) {
        const float4 wq = *(const float4*)&w[j][r];
        const float wv[4] = {wq.x, wq.y, wq.z, wq.w};
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
          for (int e = 0; e < VEC; ++e) acc[r + t][e] = fmaf(wv[t], vv[e], acc[r + t][e]);
      }
    }
  }
  if (!cok) return;
#pragma unroll
  for (int r = 0; r < MR; ++r) {
    if (r >= (int)m) break;
    if constexpr (VEC == 4)
      atomicAdd((float4*)(Y + (long long)r * ldy + c), make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]));
    else
      atomicAdd((float2*)(Y + (long long)r * ldy + c), make_float2(acc[r][0], acc[r][1]));
  }
}

template <int MR, int VEC>
sks_status sjlt_reg_launch(cudaStream_t stream, const float* A, long long lda, int64_t n, int d, int m, int s_eff,
                           uint64_t seed, float* Y, long long ldy) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int ncb = (d + kSjRegThreads * VEC - 1) / (kSjRegThreads * VEC);
  const int64_t chunks =
      std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ((int64_t)sms * 6 + ncb - 1) / ncb));
  const int64_t per = (n + chunks - 1) / chunks;
  sjlt_reg_kernel<MR, VEC><<<(unsigned)(chunks * ncb), kSjRegThreads, 0, stream>>>(A, lda, n, d, (uint32_t)m, s_eff,
                                                                                  make_key(seed), Y, ldy, ncb, per);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

template <typename T, int VEC>
sks_status sjlt_block_launch(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, int m, int s_eff,
                             uint64_t seed, T* Y, long long ldy, size_t smem) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int ncb = (d + kSjBlockThreads * VEC - 1) / (kSjBlockThreads * VEC);
  const int per_sm = smem <= 100 * 1024 ? 2 : 1;
  const int64_t chunks =
      std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, ((int64_t)sms * 4 * per_sm + ncb - 1) / ncb));
  const int64_t per = (n + chunks - 1) / chunks;
  auto kern = sjlt_block_kernel<T, VEC>;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<(unsigned)(chunks * ncb), kSjBlockThreads, smem, stream>>>(A, lda, n, d, (uint32_t)m, s_eff, make_key(seed),
                                                                    Y, ldy, ncb, per);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

// ---------------------------------------------------------------- SJLT by warp groups (float32, 16 < m <= 128)
// The s target rows of every data row are hashed once per pass into a table
// (one record per 32 data rows: the (row, local sketch row, sign) entries
// sorted by warp group, and the group offsets).  A CTA owns a block of 128
// columns and a run of 32-row stages; G consumer warps each keep the sketch
// rows [g RPG, (g + 1) RPG) of those columns in registers (lane = 4 columns),
// a producer warp streams the A tiles (TMA) and the table records into a
// 4-stage ring.  Per stage a warp takes its own entries, and for every local
// row r (unrolled, so that acc[r] is a register) the entries hitting r (a warp
// ballot) add their A row, read from shared memory, into acc[r].  A leaves HBM
// once and the s-fold replication happens on chip; the register rows are
// flushed to Y with one vector atomic per row and lane when the CTA finishes.
constexpr int kSgRows = 32;                     // data rows per stage (one table record)
constexpr int kSgStages = 4;
constexpr int kSgVec = 4;                       // columns per lane
constexpr int kSgW = 32 * kSgVec;               // columns per CTA
constexpr int kSgRecU16 = 152;                  // 128 entries + up to 17 offsets (+ pad): 304 bytes
constexpr int kSgMaxS = 4;

__global__ void sjlt_table_kernel(int64_t n, uint32_t m, int s_eff, Key key, int rpg, int groups,
                                  uint16_t* __restrict__ tab, int64_t nstages) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t sg = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); sg < nstages; sg += nwarps) {
    const int64_t i = sg * kSgRows + lane;
    uint32_t rows[kSjltMaxS];
    float sgn[kSjltMaxS];
    int cnt = 0;
    if (i < n) cnt = sjlt_hash(key, (uint32_t)i, m, s_eff, rows, sgn);
    uint16_t* rec = tab + sg * kSgRecU16;
    int base = 0;
    for (int g = 0; g < groups; ++g) {
      int c = 0;
      for (int k = 0; k < cnt; ++k) c += (int)(rows[k] / (uint32_t)rpg) == g;
      int incl = c;  // inclusive scan over the lanes
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int tot = __shfl_sync(0xffffffffu, incl, 31);
      int pos = base + incl - c;
      for (int k = 0; k < cnt; ++k)
        if ((int)(rows[k] / (uint32_t)rpg) == g)
          rec[pos++] = (uint16_t)((uint32_t)lane | ((rows[k] % (uint32_t)rpg) << 5) | (sgn[k] < 0.f ? 0x8000u : 0u));
      if (lane == 0) rec[128 + g] = (uint16_t)base;
      base += tot;
    }
    if (lane == 0) rec[128 + groups] = (uint16_t)base;
  }
}

template <int RPG, int G>
__global__ void __launch_bounds__((G + 1) * 32, 1) sjlt_grp_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                    const uint16_t* __restrict__ tab, int64_t nstages,
                                                                    int d, uint32_t m, int64_t ncb, float scale,
                                                                    float* __restrict__ Y, long long ldy,
                                                                    DevStatus* st) {
  constexpr int kTile = kSgRows * kSgW;        // floats per stage
  extern __shared__ __align__(128) unsigned char sg_smem[];
  float* tiles = reinterpret_cast<float*>(sg_smem);
  uint16_t* recs = reinterpret_cast<uint16_t*>(sg_smem + (size_t)kSgStages * kTile * sizeof(float));
  uint64_t* full = reinterpret_cast<uint64_t*>(sg_smem + (size_t)kSgStages * (kTile * sizeof(float) + 2 * kSgRecU16));
  uint64_t* empty = full + kSgStages;
  __shared__ int abort_flag;
  __shared__ long long issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // CTA b takes column block b % ncb and an equal share of its stages
  const int64_t cb = (int64_t)blockIdx.x % ncb, idx = (int64_t)blockIdx.x / ncb;
  const int64_t k = (int64_t)gridDim.x / ncb + (cb < (int64_t)gridDim.x % ncb ? 1 : 0);
  const int64_t s0 = nstages * idx / k, s1 = nstages * (idx + 1) / k;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSgStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], G);
    }
    abort_flag = 0;
    issued = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == G) {  // producer
    if (lane == 0) {
      long long it = 0;
      for (int64_t sg = s0; sg < s1; ++sg, ++it) {
        const int slot = (int)(it % kSgStages);
        if (it >= kSgStages && !mbar_wait(&empty[slot], (uint32_t)((it / kSgStages - 1) & 1), st, 41)) break;
        if (*(volatile int*)&abort_flag) break;
        mbar_arrive_expect_tx(&full[slot], (uint32_t)(kTile * sizeof(float) + 2 * kSgRecU16));
        tma_load_2d(tiles + (size_t)slot * kTile, &tmap, &full[slot], (int)(cb * kSgW), (int)(sg * kSgRows));
        bulk_load(recs + slot * kSgRecU16, tab + sg * kSgRecU16, 2 * kSgRecU16, &full[slot]);
      }
      issued = it;
    }
  } else {  // consumer warp: sketch rows [warp RPG, (warp + 1) RPG)
    float acc[RPG][kSgVec];
#pragma unroll
    for (int r = 0; r < RPG; ++r)
#pragma unroll
      for (int e = 0; e < kSgVec; ++e) acc[r][e] = 0.f;
    long long it = 0;
    bool ok = true;
    for (int64_t sg = s0; sg < s1; ++sg, ++it) {
      const int slot = (int)(it % kSgStages);
      if (!mbar_wait_warp(&full[slot], (uint32_t)((it / kSgStages) & 1), st, 42)) {
        if (lane == 0) atomicExch(&abort_flag, 1);
        ok = false;
        break;
      }
      const uint16_t* rec = recs + slot * kSgRecU16;
      const int e0 = rec[128 + warp], e1 = rec[129 + warp];
      const float* tile = tiles + (size_t)slot * kTile + lane * kSgVec;
      for (int base = e0; base < e1; base += 32) {
        const int cnt = min(32, e1 - base);
        const uint32_t mine = lane < cnt ? (uint32_t)rec[base + lane] : 0u;
        const uint32_t myloc = lane < cnt ? (mine >> 5) & 127u : 0xFFu;
#pragma unroll
        for (int r = 0; r < RPG; ++r) {
          uint32_t mask = __ballot_sync(0xffffffffu, myloc == (uint32_t)r);
          while (mask) {
            const int t = __ffs(mask) - 1;
            mask &= mask - 1;
            const uint32_t ent = __shfl_sync(0xffffffffu, mine, t);
            const float4 v = *reinterpret_cast<const float4*>(tile + (ent & 31u) * kSgW);
            const float sgn = (ent & 0x8000u) ? -1.f : 1.f;
            acc[r][0] = fmaf(sgn, v.x, acc[r][0]);
            acc[r][1] = fmaf(sgn, v.y, acc[r][1]);
            acc[r][2] = fmaf(sgn, v.z, acc[r][2]);
            acc[r][3] = fmaf(sgn, v.w, acc[r][3]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
    const int c = (int)cb * kSgW + lane * kSgVec;
    if (ok && s0 < s1 && c < d) {
#pragma unroll
      for (int r = 0; r < RPG; ++r) {
        const uint32_t row = (uint32_t)(warp * RPG + r);
        if (row < m)
          atomicAdd(reinterpret_cast<float4*>(Y + (long long)row * ldy + c),
                    make_float4(acc[r][0] * scale, acc[r][1] * scale, acc[r][2] * scale, acc[r][3] * scale));
      }
    }
  }
  // no bulk copy may still be writing into this CTA's shared memory when it exits
  __syncthreads();
  if (threadIdx.x == G * 32) {
    for (long long t = issued > kSgStages ? issued - kSgStages : 0; t < issued; ++t)
      mbar_wait(&full[t % kSgStages], (uint32_t)((t / kSgStages) & 1), st, 43);
  }
}

size_t sjlt_grp_smem() {
  return (size_t)kSgStages * ((size_t)kSgRows * kSgW * sizeof(float) + 2 * kSgRecU16) + 2 * kSgStages * 8;
}

template <int RPG, int G>
sks_status sjlt_grp_launch(cudaStream_t stream, const float* A, long long lda, int64_t n, int d, int m, int s_eff,
                           uint64_t seed, float* Y, long long ldy, uint16_t* tab, DevStatus* st) {
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int64_t nstages = (n + kSgRows - 1) / kSgRows;
  sjlt_table_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nstages + 7) / 8, (int64_t)sms * 16)), 256, 0,
                      stream>>>(n, (uint32_t)m, s_eff, make_key(seed), RPG, G, tab, nstages);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  CUtensorMap tmap;
  SKS_TRY(make_tmap_2d(&tmap, A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), (uint64_t)n, (uint64_t)d,
                       (uint64_t)lda, (uint32_t)kSgW, (uint32_t)kSgRows));
  const size_t smem = sjlt_grp_smem();
  auto kern = sjlt_grp_kernel<RPG, G>;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (G + 1) * 32, smem));
  const int64_t ncb = (d + kSgW - 1) / kSgW;
  // every column block gets at least one CTA; more CTAs split its stages
  int64_t grid = std::max<int64_t>(ncb, (int64_t)sms * std::max(1, per_sm));
  grid = std::min<int64_t>(grid, ncb * nstages);
  kern<<<(unsigned)grid, (G + 1) * 32, smem, stream>>>(tmap, tab, nstages, d, (uint32_t)m, ncb,
                                                       (float)(1.0 / std::sqrt((double)s_eff)), Y, ldy, st);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

// ---------------------------------------------------------------- SJLT by warp groups, rows in shared memory (128 < m <= 512)
// Same table, ring and column-block schedule as sjlt_grp_kernel, but each of
// the 16 consumer warps keeps its RPG = m / 16 sketch rows (of 32 VEC columns)
// in a private shared-memory slab and applies an entry as a read-modify-write
// of one slab row.  Two entries are taken per step (their rows may coincide:
// then both go into one update), so two row updates are in flight per warp.
constexpr int kSlG = 16;  // consumer warps

template <int VEC>
__global__ void __launch_bounds__((kSlG + 1) * 32, 1) sjlt_slab_kernel(const __grid_constant__ CUtensorMap tmap,
                                                                       const uint16_t* __restrict__ tab,
                                                                       int64_t nstages, int d, uint32_t m, int rpg,
                                                                       int64_t ncb, float scale, float* __restrict__ Y,
                                                                       long long ldy, DevStatus* st) {
  using V = typename std::conditional<VEC == 4, float4, typename std::conditional<VEC == 2, float2, float>::type>::type;
  constexpr int W = 32 * VEC;
  constexpr int kTile = kSgRows * W;
  extern __shared__ __align__(128) unsigned char sl_smem[];
  float* tiles = reinterpret_cast<float*>(sl_smem);
  uint16_t* recs = reinterpret_cast<uint16_t*>(sl_smem + (size_t)kSgStages * kTile * sizeof(float));
  uint64_t* full = reinterpret_cast<uint64_t*>(sl_smem + (size_t)kSgStages * (kTile * sizeof(float) + 2 * kSgRecU16));
  uint64_t* empty = full + kSgStages;
  float* slab = reinterpret_cast<float*>(empty + kSgStages);  // kSlG * rpg rows of W floats
  __shared__ int abort_flag;
  __shared__ long long issued;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t cb = (int64_t)blockIdx.x % ncb, idx = (int64_t)blockIdx.x / ncb;
  const int64_t k = (int64_t)gridDim.x / ncb + (cb < (int64_t)gridDim.x % ncb ? 1 : 0);
  const int64_t s0 = nstages * idx / k, s1 = nstages * (idx + 1) / k;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kSgStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kSlG);
    }
    abort_flag = 0;
    issued = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == kSlG) {  // producer
    if (lane == 0) {
      long long it = 0;
      for (int64_t sg = s0; sg < s1; ++sg, ++it) {
        const int slot = (int)(it % kSgStages);
        if (it >= kSgStages && !mbar_wait(&empty[slot], (uint32_t)((it / kSgStages - 1) & 1), st, 44)) break;
        if (*(volatile int*)&abort_flag) break;
        mbar_arrive_expect_tx(&full[slot], (uint32_t)(kTile * sizeof(float) + 2 * kSgRecU16));
        tma_load_2d(tiles + (size_t)slot * kTile, &tmap, &full[slot], (int)(cb * W), (int)(sg * kSgRows));
        bulk_load(recs + slot * kSgRecU16, tab + sg * kSgRecU16, 2 * kSgRecU16, &full[slot]);
      }
      issued = it;
    }
  } else {
    float* my = slab + (size_t)warp * rpg * W + lane * VEC;  // this warp's rows, this lane's columns
    for (int r = 0; r < rpg; ++r)
#pragma unroll
      for (int e = 0; e < VEC; ++e) my[r * W + e] = 0.f;
    long long it = 0;
    bool ok = true;
    for (int64_t sg = s0; sg < s1; ++sg, ++it) {
      const int slot = (int)(it % kSgStages);
      if (!mbar_wait_warp(&full[slot], (uint32_t)((it / kSgStages) & 1), st, 45)) {
        if (lane == 0) atomicExch(&abort_flag, 1);
        ok = false;
        break;
      }
      const uint16_t* rec = recs + slot * kSgRecU16;
      const int e0 = rec[128 + warp], e1 = rec[129 + warp];
      const float* tile = tiles + (size_t)slot * kTile + lane * VEC;
      int e = e0;
      for (; e + 1 < e1; e += 2) {
        const uint32_t a = rec[e], b = rec[e + 1];
        const uint32_t ra = (a >> 5) & 1023u, rb = (b >> 5) & 1023u;
        const V va = *reinterpret_cast<const V*>(tile + (a & 31u) * W);
        const V vb = *reinterpret_cast<const V*>(tile + (b & 31u) * W);
        V sa = *reinterpret_cast<const V*>(my + ra * W);
        V sb = *reinterpret_cast<const V*>(my + rb * W);
        const float ga = (a & 0x8000u) ? -1.f : 1.f, gb = (b & 0x8000u) ? -1.f : 1.f;
        const bool same = ra == rb;
        float* pa = reinterpret_cast<float*>(&sa);
        float* pb = reinterpret_cast<float*>(&sb);
        const float* qa = reinterpret_cast<const float*>(&va);
        const float* qb = reinterpret_cast<const float*>(&vb);
#pragma unroll
        for (int q = 0; q < VEC; ++q) {
          pa[q] = fmaf(ga, qa[q], pa[q]);
          pb[q] = fmaf(gb, qb[q], pb[q]);
          if (same) pa[q] = fmaf(gb, qb[q], pa[q]);
        }
        *reinterpret_cast<V*>(my + ra * W) = sa;
        if (!same) *reinterpret_cast<V*>(my + rb * W) = sb;
      }
      if (e < e1) {
        const uint32_t a = rec[e];
        const uint32_t ra = (a >> 5) & 1023u;
        const V va = *reinterpret_cast<const V*>(tile + (a & 31u) * W);
        V sa = *reinterpret_cast<const V*>(my + ra * W);
        const float ga = (a & 0x8000u) ? -1.f : 1.f;
        float* pa = reinterpret_cast<float*>(&sa);
        const float* qa = reinterpret_cast<const float*>(&va);
#pragma unroll
        for (int q = 0; q < VEC; ++q) pa[q] = fmaf(ga, qa[q], pa[q]);
        *reinterpret_cast<V*>(my + ra * W) = sa;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[slot]);
    }
    const int c = (int)cb * W + lane * VEC;
    if (ok && s0 < s1 && c < d) {
      for (int r = 0; r < rpg; ++r) {
        const uint32_t row = (uint32_t)(warp * rpg + r);
        if (row >= m) break;
        float* y = Y + (long long)row * ldy + c;
        if constexpr (VEC == 4)
          atomicAdd(reinterpret_cast<float4*>(y), make_float4(my[r * W] * scale, my[r * W + 1] * scale,
                                                              my[r * W + 2] * scale, my[r * W + 3] * scale));
        else if constexpr (VEC == 2)
          atomicAdd(reinterpret_cast<float2*>(y), make_float2(my[r * W] * scale, my[r * W + 1] * scale));
        else
          atomicAdd(y, my[r * W] * scale);
      }
    }
  }
  __syncthreads();
  if (threadIdx.x == kSlG * 32) {
    for (long long t = issued > kSgStages ? issued - kSgStages : 0; t < issued; ++t)
      mbar_wait(&full[t % kSgStages], (uint32_t)((t / kSgStages) & 1), st, 46);
  }
}

template <int VEC>
size_t sjlt_slab_smem(int rpg) {
  return (size_t)kSgStages * ((size_t)kSgRows * 32 * VEC * sizeof(float) + 2 * kSgRecU16) + 2 * kSgStages * 8 +
         (size_t)kSlG * rpg * 32 * VEC * sizeof(float);
}

template <int VEC>
sks_status sjlt_slab_launch(cudaStream_t stream, const float* A, long long lda, int64_t n, int d, int m, int s_eff,
                            uint64_t seed, float* Y, long long ldy, uint16_t* tab, DevStatus* st) {
  constexpr int W = 32 * VEC;
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  const int64_t nstages = (n + kSgRows - 1) / kSgRows;
  const int rpg = (m + kSlG - 1) / kSlG;
  sjlt_table_kernel<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((nstages + 7) / 8, (int64_t)sms * 16)), 256, 0,
                      stream>>>(n, (uint32_t)m, s_eff, make_key(seed), rpg, kSlG, tab, nstages);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  CUtensorMap tmap;
  SKS_TRY(make_tmap_2d(&tmap, A, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, sizeof(float), (uint64_t)n, (uint64_t)d,
                       (uint64_t)lda, (uint32_t)W, (uint32_t)kSgRows));
  const size_t smem = sjlt_slab_smem<VEC>(rpg);
  auto kern = sjlt_slab_kernel<VEC>;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  SKS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, (kSlG + 1) * 32, smem));
  const int64_t ncb = (d + W - 1) / W;
  int64_t grid = std::max<int64_t>(ncb, (int64_t)sms * std::max(1, per_sm));
  grid = std::min<int64_t>(grid, ncb * nstages);
  kern<<<(unsigned)grid, (kSlG + 1) * 32, smem, stream>>>(tmap, tab, nstages, d, (uint32_t)m, rpg, ncb,
                                                          (float)(1.0 / std::sqrt((double)s_eff)), Y, ldy, st);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

}  // namespace

size_t sjlt_table_bytes(int64_t n) { return (size_t)((n + kSgRows - 1) / kSgRows) * 2 * kSgRecU16; }

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
                           size_t split_elems, bool rademacher) {
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
                                                                                icnt, rademacher ? 1 : 0);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    SKS_TRY(gemm<T>(stream, m_add, d, icnt, gbuf, icnt, false, A + i0 * lda, lda, false, Y + (long long)m_off * ldy,
                    ldy, 1.0, i0 == 0 ? 0.0 : 1.0, false, 1, 0, 0, 0, split_ws, split_elems));
  }
  return SKS_OK;
}
template sks_status gaussian_extend<double>(cudaStream_t, const double*, long long, int64_t, int, uint64_t, int, int,
                                            double*, long long, double*, size_t, double*, size_t, bool);
template sks_status gaussian_extend<float>(cudaStream_t, const float*, long long, int64_t, int, uint64_t, int, int,
                                           float*, long long, float*, size_t, float*, size_t, bool);

size_t sjlt_gather_ws_elems(int64_t n, int64_t m_max, int s) {
  return 2 * (size_t)(m_max + 1) + (size_t)std::max<int64_t>(n, 1) * (size_t)std::min<int64_t>(s, m_max) + 64;
}

template <typename TA, typename TY>
sks_status sjlt_form(cudaStream_t stream, const TA* A, long long lda, int64_t n, int d, int m, int s, uint64_t seed,
                     TY* Y, long long ldy, uint32_t* sj_ws, size_t sj_ws_elems, DevStatus* st) {
  SKS_CUDA_TRY(cudaMemset2DAsync(Y, ldy * sizeof(TY), 0, d * sizeof(TY), m, stream));
  if (n == 0) return SKS_OK;
  const int s_eff = std::min(s, m);
  if (s_eff > kSjltMaxS) return fail(SKS_ERR_UNSUPPORTED, "SJLT s > 16");
  if constexpr (std::is_same<TA, TY>::value && sizeof(TY) == 8) {
    // float64, larger m with 16-byte rows: gather the buckets (no L2 read-modify-write of Y per
    // entry; 611 vs 936 ms for the 14 re-sketches of a 2^20 x 4096 A).  For float32 the scatter's
    // 16-byte vector atomics are slightly faster (12.9 vs 14.2 ms per pass there).
    const bool al16 = ((uintptr_t)A & 15) == 0 && ((uintptr_t)Y & 15) == 0 && (d * sizeof(TY)) % 16 == 0 &&
                      (lda * sizeof(TY)) % 16 == 0 && (ldy * sizeof(TY)) % 16 == 0;
    if (sj_ws && al16 && m > 64 && (long long)n * s_eff < (1ll << 31) &&
        sj_ws_elems >= 2 * (size_t)(m + 1) + (size_t)n * (size_t)s_eff)
      return sjlt_gather_launch<TY>(stream, (const TY*)A, lda, n, d, m, s_eff, seed, Y, ldy, sj_ws);
  }
  // small and medium m: column-block kernel (partial rows in shared memory);
  // the widest column vector whose m partial rows fit in 200 KB
  if constexpr (std::is_same<TA, TY>::value) {
    const size_t hash_bytes = (size_t)kSjBlockThreads * s_eff * 8;
    const bool al16 = ((uintptr_t)A & 15) == 0 && ((uintptr_t)Y & 15) == 0;
    const TY* At = (const TY*)A;
    constexpr size_t kMax = 200 * 1024;
    auto fits = [&](int vec) {
      return (size_t)m * kSjBlockThreads * vec * sizeof(TY) + hash_bytes <= kMax && d % vec == 0 &&
             lda % vec == 0 && ldy % vec == 0 && (vec == 1 || al16);
    };
    auto bytes = [&](int vec) { return (size_t)m * kSjBlockThreads * vec * sizeof(TY) + hash_bytes; };
    // 16-byte columns only: narrower ones keep too few bytes in flight at one
    // CTA per SM, and the L2 scatter is faster there
    if constexpr (sizeof(TY) == 4) {
      // partial rows in registers: 16-byte columns up to m = 32 (measured at n = 2^20, d = 4096:
      // 2.6 / 3.6 / 7.9 ms for 8 / 16 / 32 rows; 64 rows of 2 columns took 20.6 ms, slower than the
      // scatter's 12 ms, so m > 32 goes to the shared-memory kernel or the scatter)
      if (al16 && d % 4 == 0 && lda % 4 == 0 && ldy % 4 == 0) {
        if (m <= 8) return sjlt_reg_launch<8, 4>(stream, (const float*)A, lda, n, d, m, s_eff, seed, Y, ldy);
        if (m <= 16) return sjlt_reg_launch<16, 4>(stream, (const float*)A, lda, n, d, m, s_eff, seed, Y, ldy);
        // 16 < m <= 256: sketch rows in the registers or shared memory of warp groups (one pass over A
        // from HBM)
        if (m <= 256 && s_eff <= kSgMaxS && sj_ws && sj_ws_elems * sizeof(uint32_t) >= sjlt_table_bytes(n) &&
            n < (1ll << 31)) {
          const float* Af = (const float*)A;
          float* Yf = (float*)Y;
          uint16_t* tab = reinterpret_cast<uint16_t*>(sj_ws);
          // measured at n = 2^20, d = 4096, s = 4: 4.4 / 4.7 / 7.0 / 10.2 ms for m = 32 / 64 / 128 / 256
          // (the scatter: 7.9 (registers) / 18.6 / 16.8 / 12.7 ms)
          if (m <= 32) return sjlt_grp_launch<4, 8>(stream, Af, lda, n, d, m, s_eff, seed, Yf, ldy, tab, st);
          if (m <= 64) return sjlt_grp_launch<8, 8>(stream, Af, lda, n, d, m, s_eff, seed, Yf, ldy, tab, st);
          if (m <= 128) return sjlt_grp_launch<16, 8>(stream, Af, lda, n, d, m, s_eff, seed, Yf, ldy, tab, st);
          // 128 < m <= 512: rows in per-warp shared-memory slabs (7.4 / 9.8 ms at m = 256 / 512; registers
          // of 16 warps: 10.2 ms at m = 256; the scatter: 12.7 / 11.5 ms; slabs of 32 columns at m = 1024:
          // 17.0 ms against the scatter's 10.9)
          return sjlt_slab_launch<4>(stream, Af, lda, n, d, m, s_eff, seed, Yf, ldy, tab, st);
        }
        if (m <= 512 && s_eff <= kSgMaxS && sj_ws && sj_ws_elems * sizeof(uint32_t) >= sjlt_table_bytes(n) &&
            n < (1ll << 31))
          return sjlt_slab_launch<2>(stream, (const float*)A, lda, n, d, m, s_eff, seed, (float*)Y, ldy,
                                     reinterpret_cast<uint16_t*>(sj_ws), st);
        if (m <= 32) return sjlt_reg_launch<32, 4>(stream, (const float*)A, lda, n, d, m, s_eff, seed, Y, ldy);
      }
      if (fits(4)) return sjlt_block_launch<TY, 4>(stream, At, lda, n, d, m, s_eff, seed, Y, ldy, bytes(4));
    } else {
      if (fits(2)) return sjlt_block_launch<TY, 2>(stream, At, lda, n, d, m, s_eff, seed, Y, ldy, bytes(2));
    }
    if (m <= 2 && fits(1)) return sjlt_block_launch<TY, 1>(stream, At, lda, n, d, m, s_eff, seed, Y, ldy, bytes(1));
  }
  const long long row_blocks = (n + 7) / 8;
  const long long blocks = row_blocks * ((d + kSjltCols - 1) / kSjltCols);
  if (blocks > 0x7fffffffll) return fail(SKS_ERR_UNSUPPORTED, "SJLT grid too large");
  sjlt_scatter_kernel<TA, TY><<<(unsigned)blocks, 256, 0, stream>>>(A, lda, n, d, (uint32_t)m, s_eff, make_key(seed),
                                                                   Y, ldy, row_blocks);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}
template sks_status sjlt_form<double, double>(cudaStream_t, const double*, long long, int64_t, int, int, int, uint64_t,
                                              double*, long long, uint32_t*, size_t, DevStatus*);
template sks_status sjlt_form<float, float>(cudaStream_t, const float*, long long, int64_t, int, int, int, uint64_t,
                                            float*, long long, uint32_t*, size_t, DevStatus*);

}  // namespace sks
