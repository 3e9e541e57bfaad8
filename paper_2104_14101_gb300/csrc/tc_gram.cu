// tc_gram.cu -- K6 on the 5th-generation tensor cores: the sketched Gram
// matrices of the preconditioner (Section 4.1.1),
//     C = alpha * A B^T   (A: M x K, B: N x K, float32 in, float64 out),
// i.e. H_S = c^2 Y^T Y (m >= d) or W_S = c^2 Z Z^T, Z = Y Lambda^{-1/2} (m < d).
//
// The preconditioner must resolve eigenvalues down to nu^2 ~ 1e-8 next to
// entries of order 1, and when m ~ d the sketched Gram is nearly singular, so
// float32 rounding of the accumulation (~1e-7) is not acceptable.  The product
// is therefore made EXACT for a 16-bit representation of the operands
// (Ozaki-style splitting): every operand row x is split against its own
// maximum exponent e (|x| < 2^e) into two bfloat16 slices holding integers
//     hi = rint(x 2^(8-e)) 2^(e-8)         (|hi| <= 256 units of 2^(e-8))
//     lo = rint((x - hi) 2^(16-e)) 2^(e-16) (|lo| <= 128 units of 2^(e-16)),
// so x = hi + lo + O(2^(e-17)).  For an output entry (i, j) every hi.hi product
// is an integer multiple of 2^(e_i+f_j-16) below 2^16 of those units, hi.lo and
// lo.hi products multiples of 2^(e_i+f_j-24) below 2^15, lo.lo multiples of
// 2^(e_i+f_j-32) below 2^14: sums of up to 256 K-elements of each class are
// exact in float32.  The three classes accumulate in three TMEM accumulators
// that are drained every 256 K-elements into a double-float (float32 pair)
// sum (~48 bits; float64 adds would be far slower on this part).  The result
// is the exact Gram of the rounded operands, so H_S' = c^2 Y'^T Y' + nu^2
// Lambda is positive definite by construction.
//
// Structure (one CTA per 128 x 128 output tile, 18 warps):
//   warp 0      TMA producer: Ah, Al, Bh, Bl tiles (128 rows x 64 bf16, 128B
//               swizzle) into a 3-stage shared-memory ring;
//   warp 1      MMA issuer: 16 tcgen05.mma (M=128, N=128, K=16) per stage into
//               the three accumulators; tcgen05.commit frees the stage, and
//               after each group of 4 stages publishes the accumulators;
//   warps 2-17  epilogue: tcgen05.ld the accumulators (each warp: its 32 TMEM
//               lanes x 32 columns), double-float accumulate, release them;
//               at the end write alpha * (hi + lo) in float64.
// Every mbarrier wait is bounded; a timed-out role flags the CTA, all roles
// leave their loops, wait (bounded) for their own asynchronous work, and the
// TMEM is freed before exit.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>

#include "internal.h"
#include "tc_gram.h"

namespace sks {
namespace {

constexpr int TBM = 128, TBN = 128, TBK = 64;
constexpr int kStagesTC = 3;
constexpr int kTileBytes = TBM * TBK * 2;     // 16 KB per operand tile
constexpr int kStageBytes = 4 * kTileBytes;   // Ah, Al, Bh, Bl
constexpr int kEpiWarps = 16;                 // 4 per TMEM lane quadrant, 32 columns each
constexpr int kTcThreads = (2 + kEpiWarps) * 32;
constexpr uint32_t kTmemCols = 512;           // three 128-column float32 accumulators (hh, hl+lh, ll)
constexpr int kGroup = 4;                     // stages per exact accumulation group (4 x 64 = 256 K)

// ------------------------------------------------------------------ PTX wrappers
SKS_DEV uint64_t smem_desc_sw128(const void* tile) {
  // K-major, 128-byte swizzle: 8-row core-matrix groups 1024 bytes apart.
  const uint64_t addr = (uint64_t)(smem_addr(tile) >> 4) & 0x3FFF;
  uint64_t d = addr;
  d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major), encoded 1
  d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset between 8-row groups
  d |= (uint64_t)1 << 46;            // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;            // layout: 128-byte swizzle
  return d;
}

// kind::f16 instruction descriptor: bf16 x bf16 -> f32, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

SKS_DEV void umma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// kind::f8f6f4 instruction descriptor: e4m3 x e4m3 -> f32 (format code 0 for
// both operands), both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

SKS_DEV void umma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

SKS_DEV void umma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar))
               : "memory");
}

SKS_DEV void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
SKS_DEV void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 lanes x 16 consecutive float32 columns
SKS_DEV void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 16 consecutive float32 columns, without the wait (tmem_ld_wait()
// before the registers are read): several loads in flight at once
SKS_DEV void tmem_ld16_nowait(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
SKS_DEV void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Double-float accumulation (Knuth's TwoSum): (s, e) += x.
SKS_DEV void df_add(float& s, float& e, float x) {
  const float t = s + x;
  const float bp = t - s;
  const float err = (s - (t - bp)) + (x - bp);
  s = t;
  e += err;
}

struct GramArgs {
  int M, N, Kp;          // Kp: padded K (multiple of 64)
  int tiles_n;           // number of column tiles
  int lower;             // only tiles with col tile <= row tile, and only j <= i written
  double alpha, beta;
  double* C;
  long long ldc;
  DevStatus* st;
};

__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gram_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                   const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl, GramArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t full[kStagesTC], empty[kStagesTC], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  // tile coordinates (lower: linear index over the lower triangle of tiles)
  int tm, tn;
  if (g.lower) {
    const int t = blockIdx.x;
    tm = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((tm + 1) * (tm + 2) / 2 <= t) ++tm;
    while (tm * (tm + 1) / 2 > t) --tm;
    tn = t - tm * (tm + 1) / 2;
  } else {
    tm = blockIdx.x / g.tiles_n;
    tn = blockIdx.x % g.tiles_n;
  }
  const int row0 = tm * TBM, col0 = tn * TBN;
  const int nk = g.Kp / TBK;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kStagesTC; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    fence_mbar_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kk = 0; kk < nk; ++kk) {
        const int s = kk % kStagesTC;
        const uint32_t ph = (uint32_t)(kk / kStagesTC) & 1u;
        if (abort_flag || !mbar_wait(&empty[s], ph ^ 1u, g.st, 41)) {
          abort_flag = 1;
          break;
        }
        unsigned char* st = smem + (size_t)s * kStageBytes;
        mbar_arrive_expect_tx(&full[s], kStageBytes);
        tma_load_2d(st + 0 * kTileBytes, &mAh, &full[s], kk * TBK, row0);
        tma_load_2d(st + 1 * kTileBytes, &mAl, &full[s], kk * TBK, row0);
        tma_load_2d(st + 2 * kTileBytes, &mBh, &full[s], kk * TBK, col0);
        tma_load_2d(st + 3 * kTileBytes, &mBl, &full[s], kk * TBK, col0);
        issued = kk + 1;
      }
      // every issued copy has landed before exit
      const int first = issued > kStagesTC ? issued - kStagesTC : 0;
      for (int k = first; k < issued; ++k) mbar_wait(&full[k % kStagesTC], (uint32_t)(k / kStagesTC) & 1u, g.st, 42);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(TBM, TBN);
      const int ngroups = (nk + kGroup - 1) / kGroup;
      int committed = -1;
      for (int grp = 0; grp < ngroups && !abort_flag; ++grp) {
        // the epilogue has drained the previous group
        if (!mbar_wait(&acc_empty[0], ((uint32_t)grp & 1u) ^ 1u, g.st, 44)) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const int k_end = min(nk, (grp + 1) * kGroup);
        for (int kk = grp * kGroup; kk < k_end; ++kk) {
          const int s = kk % kStagesTC;
          if (abort_flag || !mbar_wait(&full[s], (uint32_t)(kk / kStagesTC) & 1u, g.st, 43)) {
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          unsigned char* st = smem + (size_t)s * kStageBytes;
          const bool first = (kk == grp * kGroup);
          // products: (Ah,Bh) -> acc 0; (Ah,Bl), (Al,Bh) -> acc 1; (Al,Bl) -> acc 2
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const int accn = (p == 0) ? 0 : (p == 3 ? 2 : 1);
            const uint64_t ad = smem_desc_sw128(st + (p >> 1) * kTileBytes);
            const uint64_t bd = smem_desc_sw128(st + (2 + (p & 1)) * kTileBytes);
            const uint32_t d_tmem = tmem + (uint32_t)(accn * TBN);
#pragma unroll
            for (int k = 0; k < TBK / 16; ++k) {
              // advance 16 bf16 = 32 bytes along K inside the swizzle atom;
              // the first MMA of a group into an accumulator overwrites it
              const uint32_t acc = (first && k == 0 && p != 2) ? 0u : 1u;
              umma_bf16(d_tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, acc);
            }
          }
          umma_commit(&empty[s]);  // stage reusable once these MMAs finish
        }
        if (abort_flag) break;
        umma_commit(&acc_full[0]);  // group complete: accumulators ready
        committed = grp;
      }
      // wait (bounded) for the last committed MMA group before leaving
      if (committed >= 0) mbar_wait(&acc_full[0], (uint32_t)committed & 1u, g.st, 45);
    }
  } else {
    // ------------------------------------------------------------ epilogue (warps 2..17)
    const int ew = warp - 2;            // 0..15
    const int quad = warp & 3;          // TMEM lane quadrant this warp may access
    const int cblk = ew >> 2;           // columns [32*cblk, 32*cblk + 32)
    const int row = quad * 32 + lane;   // tile row held by this thread
    const int ngroups = (nk + kGroup - 1) / kGroup;
    float hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) hi[i] = lo[i] = 0.f;
    for (int grp = 0; grp < ngroups; ++grp) {
      const bool ok = mbar_wait_warp(&acc_full[0], (uint32_t)grp & 1u, g.st, 46);
      if (!ok || abort_flag) {
        if (lane == 0) abort_flag = 1;
        break;
      }
      tc_fence_after();
#pragma unroll
      for (int accn = 0; accn < 3; ++accn) {
        const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(accn * TBN + cblk * 32);
        float v[16];
        tmem_ld16(base, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) df_add(hi[i], lo[i], v[i]);
        tmem_ld16(base + 16, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) df_add(hi[16 + i], lo[16 + i], v[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[0]);
    }
    const int gi = row0 + row;
    if (!abort_flag && gi < g.M) {
      double* crow = g.C + (long long)gi * g.ldc;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int gj = col0 + cblk * 32 + i;
        if (gj < g.N && (!g.lower || gj <= gi)) {
          const double v = g.alpha * ((double)hi[i] + (double)lo[i]);
          crow[gj] = g.beta == 0.0 ? v : v + g.beta * crow[gj];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// Operand element (orow, k) of X (transpose: X[k][orow], else X[orow][k]),
// divided by sqrt(colscale[c]) in float64 and rounded once to float32.
// isq: 1/sqrt(colscale) per column (float64, precomputed once), or NULL.
__device__ __forceinline__ float operand_elem(const float* __restrict__ X, long long ldx, int rows, int cols,
                                             int transpose, const double* __restrict__ isq, int orow, int k) {
  const int r = transpose ? k : orow;
  const int c = transpose ? orow : k;
  if (r >= rows || c >= cols) return 0.f;
  float v = X[(long long)r * ldx + c];
  if (isq) v = (float)((double)v * isq[c]);
  return v;
}

// isq[c] = 1 / sqrt(colscale[c]), sq[c] = sqrt(colscale[c])
__global__ void colfac_kernel(int cols, const double* __restrict__ colscale, double* __restrict__ isq,
                              double* __restrict__ sq) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  const double s = sqrt(colscale[c]);
  sq[c] = s;
  isq[c] = 1.0 / s;
}

// Maximum |element| of every operand row (as float bits; non-negative floats
// order like their bit patterns).  Operand rows along the input's rows
// (transpose = 0): one warp per row, no atomics; along its columns: a
// grid-stride walk in the input's layout (coalesced) with one atomic each.
__global__ void rowmax_kernel(const float* __restrict__ X, long long ldx, int rows, int cols, int transpose,
                              const double* __restrict__ isq, unsigned* __restrict__ rmax) {
  if (!transpose) {
    const int lane = threadIdx.x & 31;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long r = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += nw) {
      float mx = 0.f;
      for (int c = lane; c < cols; c += 32) mx = fmaxf(mx, fabsf(operand_elem(X, ldx, rows, cols, 0, isq, (int)r, c)));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0) rmax[r] = __float_as_uint(mx);
    }
    return;
  }
  const long long total = (long long)rows * cols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    const float v = fabsf(operand_elem(X, ldx, rows, cols, 1, isq, c, r));
    atomicMax(&rmax[c], __float_as_uint(v));
  }
}

// hi/lo slices against the row's maximum exponent (see the file comment).
__global__ void split_scaled_kernel(const float* __restrict__ X, long long ldx, int rows, int cols, int transpose,
                                    const double* __restrict__ isq, const unsigned* __restrict__ rmax,
                                    int out_rows, int Kp, __nv_bfloat16* __restrict__ Hh,
                                    __nv_bfloat16* __restrict__ Hl) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)out_rows * Kp) return;
  const int orow = (int)(e / Kp), k = (int)(e % Kp);
  const float v = operand_elem(X, ldx, rows, cols, transpose, isq, orow, k);
  const float mx = __uint_as_float(rmax[orow]);
  float h = 0.f, l = 0.f;
  if (mx > 0.f) {
    int ex;
    frexpf(mx, &ex);  // mx < 2^ex
    h = ldexpf(rintf(ldexpf(v, 8 - ex)), ex - 8);
    l = ldexpf(rintf(ldexpf(v - h, 16 - ex)), ex - 16);
  }
  Hh[e] = __float2bfloat16_rn(h);  // exact: integers below 2^9 times a power of two
  Hl[e] = __float2bfloat16_rn(l);
}

// Y_eff[r][c] = (hi + lo)[r][c] * sqrt(scale[c])  (float64), the sketch that
// the split operands represent exactly.
__global__ void unsplit_kernel(const __nv_bfloat16* __restrict__ Hh, const __nv_bfloat16* __restrict__ Hl, int rows,
                               int cols, int Kp, const double* __restrict__ sq, double* __restrict__ Y,
                               long long ldy) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)rows * cols) return;
  const int r = (int)(e / cols), c = (int)(e % cols);
  const long long k = (long long)r * Kp + c;
  double v = (double)__bfloat162float(Hh[k]) + (double)__bfloat162float(Hl[k]);
  if (sq) v *= sq[c];
  Y[(long long)r * ldy + c] = v;
}

// ------------------------------------------------------------------ cluster (distributed shared memory) helpers
SKS_DEV uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// address of the same shared-memory location in CTA `rank` of the cluster
SKS_DEV uint32_t mapa_shared(uint32_t local, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}
SKS_DEV void st_cluster_b32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.b32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
SKS_DEV void fence_proxy_async_cluster() { asm volatile("fence.proxy.async.shared::cluster;" ::: "memory"); }
SKS_DEV void mbar_arrive_remote(uint32_t addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(addr) : "memory");
}
SKS_DEV bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait with cluster-scope acquire (barriers that other CTAs arrive on)
SKS_DEV bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, DevStatus* st, int where) {
  if (mbar_try_wait_cluster(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (global_ns() - t0 > kWaitLimitNs) {
      raise_status(st, SKS_ERR_TIMEOUT, where, 0);
      return false;
    }
  }
}
SKS_DEV bool mbar_wait_cluster_warp(uint64_t* bar, uint32_t parity, DevStatus* st, int where) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  while (true) {
    const bool ok = mbar_try_wait_cluster(bar, parity);
    if (__all_sync(0xffffffffu, ok)) return true;
    int to = 0;
    if (lane == 0) {
      const uint64_t now = global_ns();
      if (t0 == 0) t0 = now;
      else if (now - t0 > kWaitLimitNs) to = 1;
    }
    to = __shfl_sync(0xffffffffu, to, 0);
    if (to) {
      if (lane == 0) raise_status(st, SKS_ERR_TIMEOUT, where, 0);
      return false;
    }
  }
}
// tcgen05.commit arriving on the same barrier in every CTA of `mask`
SKS_DEV void umma_commit_multicast(uint64_t* bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_addr(bar)),
      "h"(mask)
      : "memory");
}
// 1-D bulk copy of `bytes` from this CTA's shared memory to a peer's, completing
// as transaction bytes on the peer's mbarrier (addresses from mapa_shared)
SKS_DEV void bulk_copy_to_peer(uint32_t dst, const void* src, uint32_t bytes, uint32_t peer_bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "r"(smem_addr(src)), "r"(bytes), "r"(peer_bar)
      : "memory");
}
SKS_DEV void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ Gaussian sketch on tensor cores
//
// K4 for float32 A: Y[r] = sum_i bf16(G[r][i]) (hi + lo)[.][i] (or the
// Rademacher +-1 entries, exact in bfloat16, with g.rade), i.e. the
// product of the Philox/Box-Muller matrix G (rounded to bfloat16) with the
// element-wise two-slice split of A^T, hi = bf16(a), lo = bf16(a - hi), so
// |a - hi - lo| <= 2^-17 |a| (prepared once by tc_split_t).  One CTA per (128 sketch rows) x
// (256 columns) x (K slice of data rows) tile, 18 warps:
//   warp 0      TMA producer: the hi and lo tiles of A^T (256 x 64 bf16, 128B
//               swizzle) into a 2-stage ring;
//   warp 1      MMA issuer: 8 tcgen05.mma (M=128, N=256, K=16) per stage, both
//               slices into one float32 TMEM accumulator;
//   warps 2-17  generators: 32 rows of the 128 x 64 G tile of the stage
//               from Philox in registers, rounded to bfloat16 and written in
//               the swizzled K-major layout the MMA reads; one thread then
//               sends these rows (one contiguous 4 KB block) to the other 3
//               CTAs of the cluster -- the 4 column tiles that share the G
//               tile -- by bulk copies that complete on their stage barriers
//               (G never goes to global memory); they also drain the
//               accumulator.
// Stage reuse is cluster-wide: every CTA's MMA commit arrives (multicast) on
// the stage barrier of all 4 CTAs.
// The tensor core's float32 accumulation does not round to nearest, so its
// error grows with the number of MMAs summed into one accumulator: every
// group of 4 stages (256 data rows, 32 MMAs) goes to one of two TMEM
// accumulators (ping-pong) and is drained into float32 registers (round to
// nearest) while the next group runs.  Each K slice of <= 16384 data rows
// writes a float32 partial; the partials are summed in a fixed order in
// float64.
constexpr int GBM = 128, GBN = 256, GBK = 64;
constexpr int kGStages = 2;
constexpr int kGTileG = GBM * GBK * 2;                 // 16 KB
constexpr int kGTileA = GBN * GBK * 2;                 // 32 KB
constexpr int kGStageBytes = kGTileG + 2 * kGTileA;    // 80 KB
constexpr int kGGenWarps = 16;
constexpr int kGThreads = (2 + kGGenWarps) * 32;
constexpr uint32_t kGTmemCols = 512;  // two 256-column float32 accumulators
constexpr int kGCluster = 4;           // CTAs along the columns sharing every G tile
constexpr int kGDrain = 4;             // stages per accumulator group
constexpr int kGaussSlice = 16384;    // data rows per K slice
constexpr int kGaussRowChunk = 4096;  // new sketch rows per launch (bounds the partials)

struct GaussArgs {
  int d, m_add, row_base;  // sketch rows [row_base, row_base + m_add)
  long long n;             // data rows
  int Kp, kc;              // padded K; data rows per slice (multiple of 64)
  int tiles_m, tiles_n, ksplits;  // tiles_n: a multiple of the cluster size
  int rade;                        // 1: Rademacher +-1 entries instead of Gaussian ones
  Key key;
  float* part;             // [ksplits][m_add][d]
  const float* scale;      // 8-bit operands: [ksplits][d] column scales of A's slices
  DevStatus* st;
};

// E8: the 8-bit variant -- G rounded to e4m3, A^T an e4m3 operand (mAh) with
// one power-of-two scale per column and K slice, kind::f8f6f4 MMAs (K = 32),
// a stage holding 128 data rows (the same 128 bytes per operand row).
template <bool E8>
__global__ void __cluster_dims__(kGCluster, 1, 1) __launch_bounds__(kGThreads, 1)
    tc_gauss_kernel(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl, GaussArgs g) {
  constexpr int KST = E8 ? 2 * GBK : GBK;  // data rows per stage
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  __shared__ uint64_t tfull[kGStages], gfull[kGStages], empty[kGStages], acc_full[2], acc_empty[2];
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;

  // column tile fastest: the CTAs of a cluster share (row tile, K slice)
  const int tn = blockIdx.x % g.tiles_n;
  const int t2 = blockIdx.x / g.tiles_n;
  const int tm = t2 % g.tiles_m, ks = t2 / g.tiles_m;
  const uint32_t crank = cluster_rank();
  const int rloc0 = tm * GBM;  // first tile row within the m_add new rows
  const int col0 = tn * GBN;
  const int kbeg = ks * g.kc;
  const int kend = min(g.Kp, kbeg + g.kc);
  const int nk = (kend - kbeg) / KST;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < kGStages; ++s) {
      mbar_init(&tfull[s], 1);
      // the local generator warps, plus the peers' rows as transaction bytes
      mbar_init(&gfull[s], kGGenWarps);
      mbar_init(&empty[s], kGCluster);                // the MMAs of every CTA of the cluster
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kGGenWarps);
    }
    fence_mbar_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kGTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers exist before remote arrivals
  tc_fence_after();
  const uint32_t tmem = tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      int issued = 0;
      for (int kk = 0; kk < nk; ++kk) {
        const int s = kk % kGStages;
        const uint32_t ph = (uint32_t)(kk / kGStages) & 1u;
        if (abort_flag || !mbar_wait_cluster(&empty[s], ph ^ 1u, g.st, 51)) {
          abort_flag = 1;
          break;
        }
        unsigned char* st = smem + (size_t)s * kGStageBytes;
        if constexpr (E8) {
          mbar_arrive_expect_tx(&tfull[s], kGTileA);
          tma_load_2d(st + kGTileG, &mAh, &tfull[s], kbeg + kk * KST, col0);
        } else {
          mbar_arrive_expect_tx(&tfull[s], 2 * kGTileA);
          tma_load_2d(st + kGTileG, &mAh, &tfull[s], kbeg + kk * KST, col0);
          tma_load_2d(st + kGTileG + kGTileA, &mAl, &tfull[s], kbeg + kk * KST, col0);
        }
        issued = kk + 1;
      }
      const int first = issued > kGStages ? issued - kGStages : 0;
      for (int k = first; k < issued; ++k) mbar_wait(&tfull[k % kGStages], (uint32_t)(k / kGStages) & 1u, g.st, 52);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = E8 ? idesc_e4m3_f32(GBM, GBN) : idesc_bf16_f32(GBM, GBN);
      const int ngroups = (nk + kGDrain - 1) / kGDrain;
      int committed = -1;
      for (int grp = 0; grp < ngroups && !abort_flag; ++grp) {
        const int buf = grp & 1;
        // the generators have drained this buffer's previous group
        if (!mbar_wait(&acc_empty[buf], ((uint32_t)(grp >> 1) & 1u) ^ 1u, g.st, 58)) {
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc_t = tmem + (uint32_t)(buf * GBN);
        const int k_end = min(nk, (grp + 1) * kGDrain);
        for (int kk = grp * kGDrain; kk < k_end; ++kk) {
          const int s = kk % kGStages;
          const uint32_t ph = (uint32_t)(kk / kGStages) & 1u;
          if (abort_flag || !mbar_wait(&tfull[s], ph, g.st, 53) || !mbar_wait_cluster(&gfull[s], ph, g.st, 54)) {
            abort_flag = 1;
            break;
          }
          tc_fence_after();
          unsigned char* st = smem + (size_t)s * kGStageBytes;
          const uint64_t gd = smem_desc_sw128(st);
          const uint64_t hd = smem_desc_sw128(st + kGTileG);
          const uint64_t ld = smem_desc_sw128(st + kGTileG + kGTileA);
          const bool first = kk == grp * kGDrain;
          // four K steps of 32 bytes per 128-byte operand row (16 bf16 or 32 e4m3 values)
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if constexpr (E8) {
              umma_e4m3(acc_t, gd + (uint64_t)(k * 2), hd + (uint64_t)(k * 2), idesc, (first && k == 0) ? 0u : 1u);
            } else {
              umma_bf16(acc_t, gd + (uint64_t)(k * 2), hd + (uint64_t)(k * 2), idesc, (first && k == 0) ? 0u : 1u);
              umma_bf16(acc_t, gd + (uint64_t)(k * 2), ld + (uint64_t)(k * 2), idesc, 1u);
            }
          }
          umma_commit_multicast(&empty[s], (uint16_t)((1u << kGCluster) - 1u));  // stage free in every CTA
        }
        if (abort_flag) break;
        umma_commit(&acc_full[buf]);
        committed = grp;
      }
      // every issued MMA has finished before the TMEM is freed
      if (committed >= 0) mbar_wait(&acc_full[committed & 1], (uint32_t)(committed >> 1) & 1u, g.st, 55);
    }
  } else {
    // ------------------------------------------------------------ G generators and accumulator drains
    const int gtid = threadIdx.x - 64;  // 0..511
    const int row_base = g.row_base + rloc0;  // global sketch row of tile row 0
    const int row_end = g.row_base + g.m_add;  // first global row past the new rows
    // this CTA generates tile rows [32 crank, 32 crank + 32) for the whole cluster
    constexpr int kRowsPer = GBM / kGCluster;
    const int rl_lo = (int)crank * kRowsPer;
    const int q0 = (row_base + rl_lo) >> 2;
    const int nq = ((row_base + rl_lo + kRowsPer - 1) >> 2) - q0 + 1;
    constexpr uint32_t kRowBytes = kRowsPer * 128;  // this CTA's rows: one contiguous 4 KB block
    constexpr uint32_t kPeerBytes = (kGCluster - 1) * kRowBytes;
    const int quad = warp & 3, cb = (warp - 2) >> 2;  // TMEM lane quadrant, 64-column block
    const int ngroups = (nk + kGDrain - 1) / kGDrain;
    float accr[64];
#pragma unroll
    for (int j = 0; j < 64; ++j) accr[j] = 0.f;
    int drained = 0;
    bool ok = true;
    // adds group `drained` (buffer drained & 1) into the registers and frees the buffer
    auto drain = [&]() -> bool {
      const int buf = drained & 1;
      if (!mbar_wait_warp(&acc_full[buf], (uint32_t)(drained >> 1) & 1u, g.st, 57)) return false;
      tc_fence_after();
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * GBN + cb * 64 + h * 16), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) accr[h * 16 + j] += v[j];
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acc_empty[buf]);
      ++drained;
      return true;
    };
    for (int kk = 0; kk < nk; ++kk) {
      const int s = kk % kGStages;
      const uint32_t ph = (uint32_t)(kk / kGStages) & 1u;
      // the stage is free in every CTA of the cluster (their MMAs have read it)
      const bool got = ok && mbar_wait_cluster_warp(&empty[s], ph ^ 1u, g.st, 56);
      // every generator warp takes the same decision (the named barriers below
      // need all 16): leave together on any timeout or abort
      if (named_bar_or(2, kGGenWarps * 32, !got || abort_flag != 0)) {
        if (lane == 0) abort_flag = 1;
        ok = false;
        break;
      }
      unsigned char* gt = smem + (size_t)s * kGStageBytes;
      const long long i0 = (long long)kbeg + (long long)kk * KST;
      // item = (quad of sketch rows, pair of adjacent data rows): a warp covers
      // the data rows of one quad (two quads for 8-bit values) and stores
      // whole 128-byte tile rows
      for (int it = gtid; it < nq * (KST / 2); it += kGGenWarps * 32) {
        const int qi = E8 ? it >> 6 : it >> 5, kc = E8 ? (it & 63) * 2 : (it & 31) * 2;
        const int Q = q0 + qi;
        const long long i = i0 + kc;
        float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
        if (g.rade) {
          if (i < g.n) rade4_f(g.key, (uint32_t)i, (uint32_t)Q, v0);
          if (i + 1 < g.n) rade4_f(g.key, (uint32_t)(i + 1), (uint32_t)Q, v1);
        } else {
          if (i < g.n) gauss4_f(g.key, (uint32_t)i, (uint32_t)Q, v0);
          if (i + 1 < g.n) gauss4_f(g.key, (uint32_t)(i + 1), (uint32_t)Q, v1);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int R = 4 * Q + t;
          const int rl = R - row_base;
          if (rl < rl_lo || rl >= rl_lo + kRowsPer) continue;
          const bool live = R < row_end;
          if constexpr (E8) {
            // 16 e4m3 values per 16-byte chunk of the swizzled row (data row kc in byte kc)
            const uint32_t off = (uint32_t)rl * 128u + ((((uint32_t)kc >> 4) ^ ((uint32_t)rl & 7u)) << 4) +
                                 ((uint32_t)kc & 15u);
            *(__nv_fp8x2_storage_t*)(gt + off) =
                __nv_cvt_float2_to_fp8x2(make_float2(live ? v0[t] : 0.f, live ? v1[t] : 0.f), __NV_SATFINITE, __NV_E4M3);
          } else {
            const uint32_t off = (uint32_t)rl * 128u + ((((uint32_t)kc >> 3) ^ ((uint32_t)rl & 7u)) << 4) +
                                 (((uint32_t)kc & 7u) << 1);
            *(__nv_bfloat162*)(gt + off) = __floats2bfloat162_rn(live ? v0[t] : 0.f, live ? v1[t] : 0.f);
          }
        }
      }
      fence_proxy_async();  // generic-proxy writes visible to the async proxy (MMA, bulk copies)
      named_bar_sync(1, kGGenWarps * 32);  // this CTA's 32 rows are complete
      if (gtid == 0) {
        // the peers' rows arrive as transaction bytes on the local stage barrier
        mbar_arrive_expect_tx(&gfull[s], kPeerBytes);
        const unsigned char* mine = gt + (size_t)rl_lo * 128;
#pragma unroll
        for (int j = 1; j < kGCluster; ++j) {
          const uint32_t peer = (crank + (uint32_t)j) % kGCluster;
          bulk_copy_to_peer(mapa_shared(smem_addr(mine), peer), mine, kRowBytes,
                            mapa_shared(smem_addr(&gfull[s]), peer));
        }
      } else if (lane == 0) {
        mbar_arrive(&gfull[s]);
      }
      // once the first stage of a group is queued, drain the previous group
      if (kk % kGDrain == 0 && kk > 0 && drained < kk / kGDrain) {
        if (!drain()) {
          if (lane == 0) abort_flag = 1;
          ok = false;
        }
      }
    }
    while (ok && drained < ngroups && !__shfl_sync(0xffffffffu, (int)abort_flag, 0)) {
      if (!drain()) {
        if (lane == 0) abort_flag = 1;
        ok = false;
      }
    }
    const int aborted = __shfl_sync(0xffffffffu, (int)abort_flag, 0);
    if (ok && !aborted) {
      const int r = rloc0 + quad * 32 + lane;  // row within the m_add new rows
      if (r < g.m_add) {
        float* dst = g.part + ((size_t)ks * g.m_add + r) * g.d;
        const int c0 = col0 + cb * 64;
        // 8-bit operands: the slice's column scales (powers of two) bring A back
#pragma unroll
        for (int j = 0; j < 64; ++j)
          if (c0 + j < g.d) dst[c0 + j] = E8 ? accr[j] * g.scale[(size_t)ks * g.d + c0 + j] : accr[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // no CTA leaves while its peers may still write or arrive into it
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kGTmemCols) : "memory");
  }
}

// Y[row0 + r][c] = sum over slices of part[ks][r][c] (fixed order, float64)
__global__ void gauss_reduce_kernel(const float* __restrict__ part, int ksplits, int m_add, int d,
                                    float* __restrict__ Y, long long ldy, int row0) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m_add * d) return;
  const int r = (int)(e / d), c = (int)(e % d);
  double t = 0.0;
  for (int ks = 0; ks < ksplits; ++ks) t += (double)part[((size_t)ks * m_add + r) * d + c];
  Y[(long long)(row0 + r) * ldy + c] = (float)t;
}

// Element-wise split of A^T through 32 x 32 shared-memory tiles: out[c][i]
// for i < Kp (zero past n), hi = bf16(a) and lo = bf16(a - hi) (a - hi is
// exact in float32), both rounded to nearest even.
__global__ void split_t_kernel(const float* __restrict__ A, long long lda, long long n, int d, int Kp,
                               __nv_bfloat16* __restrict__ Hh, __nv_bfloat16* __restrict__ Hl) {
  __shared__ float t[32][33];
  const long long i0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long long i = i0 + j;
    const int c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (i < n && c < d) ? A[i * lda + c] : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j;
    const long long i = i0 + threadIdx.x;
    if (c >= d || i >= Kp) continue;
    const float v = t[threadIdx.x][j];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    Hh[(size_t)c * Kp + i] = h;
    Hl[(size_t)c * Kp + i] = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
  }
}

// 8-bit operand: per (K slice of kc data rows, column c) the largest |a|
// (float bits) and, over everything, sum a^2 (for the noise estimate).
__global__ void e4m3_colmax_kernel(const float* __restrict__ A, long long lda, long long n, int d, long long rows_per,
                                   int kc, unsigned* __restrict__ smax, double* __restrict__ frob2) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  const long long r0 = (long long)blockIdx.y * rows_per;
  const long long r1 = min(n, r0 + rows_per);
  float m = 0.f;
  double s2 = 0.0;
  long long slice = r0 / kc;
  for (long long i = r0; i < r1; ++i) {
    if (i / kc != slice) {
      atomicMax(&smax[(size_t)slice * d + c], __float_as_uint(m));
      m = 0.f;
      slice = i / kc;
    }
    const float v = A[i * lda + c];
    m = fmaxf(m, fabsf(v));
    s2 += (double)v * (double)v;
  }
  if (r0 < r1) atomicMax(&smax[(size_t)slice * d + c], __float_as_uint(m));
  atomicAdd(frob2, s2);
}

// scale = 2^e, e the least integer with max <= 448 2^e: with max = f 2^E
// (f in [0.5, 1)) and 448 = 0.875 2^9, e = E - 9 (+1 when f > 0.875); 1 for 0.
__global__ void e4m3_scale_kernel(int count, const unsigned* __restrict__ smax, float* __restrict__ scale) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= count) return;
  const float mx = __uint_as_float(smax[e]);
  if (!(mx > 0.f)) {
    scale[e] = 1.f;
    return;
  }
  int E;
  const float f = frexpf(mx, &E);
  scale[e] = ldexpf(1.f, E - 9 + (f > 0.875f ? 1 : 0));
}

// The e4m3 operand A8t[c][i] = e4m3(a_ic / scale[i / kc][c]) (exact division
// by a power of two; round to nearest even, finite saturation), zero for
// i >= n up to Kp; 32 x 32 shared-memory tiles for the transpose.
__global__ void split8_t_kernel(const float* __restrict__ A, long long lda, long long n, int d, int Kp, int kc,
                                const float* __restrict__ scale, unsigned char* __restrict__ A8t) {
  __shared__ float t[32][33];
  const long long i0 = (long long)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const long long i = i0 + j;
    const int c = c0 + threadIdx.x;
    t[j][threadIdx.x] = (i < n && c < d) ? A[i * lda + c] / scale[(size_t)(i / kc) * d + c] : 0.f;
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    const int c = c0 + j;
    const long long i = i0 + threadIdx.x;
    if (c >= d || i >= Kp) continue;
    A8t[(size_t)c * Kp + i] = (unsigned char)__nv_cvt_float_to_fp8(t[threadIdx.x][j], __NV_SATFINITE, __NV_E4M3);
  }
}


// ------------------------------------------------------------------ double-float trailing update
// T -= P P^T on the lower part of the trailing matrix of the double-float
// Cholesky (chol.cu), P = the current panel (rest x 64, float32 hi/lo planes).
// Each row of P is split against its own exponent e_i (|P_i.| < 2^e_i) into
// kSySlices bfloat16 slices of integers, P_iq = sum_s q_s 2^(e_i - 8 s) up to
// 2^(e_i - 49), |q_1| <= 256 and |q_s| <= 128 after it.  The products of slices
// s and t of rows i and j are integers times 2^(e_i + e_j - 8 (s + t)); all
// pairs of one level l = s + t (2 .. kSySlices + 1; deeper levels are below
// 2^-54 of the leading one) sum in one float32 TMEM accumulator, exactly
// (< 2^23 for K = 64).  The epilogue scales each level by its power of two,
// adds the levels smallest first with TwoSum and subtracts the double-float
// result from T.
constexpr int kSySlices = 6;
constexpr int kSyLevels = kSySlices;               // levels 2 .. kSySlices + 1
constexpr int kSyM = 128, kSyN = 64, kSyK = 64;
constexpr int kSyATile = kSyM * kSyK * 2;           // 16 KB per slice
constexpr int kSyBTile = kSyN * kSyK * 2;           // 8 KB per slice
constexpr int kSyBytes = kSySlices * (kSyATile + kSyBTile);
constexpr int kSyEpiWarps = 8;
constexpr int kSyThreads = (2 + kSyEpiWarps) * 32;
constexpr uint32_t kSyTmemCols = 512;               // kSyLevels accumulators of kSyN columns

// One warp per row of P: the row exponent and the slices (rows past `rest`,
// up to rest_pad, are zero).  SL: [kSySlices][rest_pad][64] bfloat16.
__global__ void syrk_slice_kernel(int rest, int rest_pad, const float* __restrict__ Ph, const float* __restrict__ Pl,
                                  long long ld, __nv_bfloat16* __restrict__ SL, int* __restrict__ ex) {
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rest_pad; r += nw) {
    float h[2] = {0.f, 0.f}, l[2] = {0.f, 0.f};
    if (r < rest) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        h[u] = Ph[(long long)r * ld + lane + 32 * u];
        l[u] = Pl[(long long)r * ld + lane + 32 * u];
      }
    }
    float mx = fmaxf(fabsf(h[0]), fabsf(h[1]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    if (mx >= 0x1p-100f && mx < 0x1p+100f) frexpf(mx, &e);  // mx < 2^e; tinier rows count as zero
    else mx = 0.f;
    if (lane == 0) ex[r] = mx > 0.f ? e : -1000;
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const float sc = mx > 0.f ? __int_as_float((127 + 8 - e) << 23) : 0.f;  // 2^(8 - e), exact
      float H = h[u] * sc, L = l[u] * sc;
#pragma unroll
      for (int s = 0; s < kSySlices; ++s) {
        const float q = rintf(H);
        // remainder (H - q) + L as an unevaluated pair; H - q is exact
        const float a = __fsub_rn(H, q);
        const float t = __fadd_rn(a, L);
        const float bb = __fsub_rn(t, a);
        const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(t, bb)), __fsub_rn(L, bb));
        SL[((size_t)s * rest_pad + r) * kSyK + lane + 32 * u] = __float2bfloat16_rn(q);  // an integer <= 256: exact
        H = t * 256.f;
        L = err * 256.f;
      }
    }
  }
}

struct SyrkArgs {
  int rest, rest_pad;
  const int* ex;
  float* Th;
  float* Tl;
  long long ldt;
  DevStatus* st;
};

__global__ void __launch_bounds__(kSyThreads, 1) tc_syrk_kernel(const __grid_constant__ CUtensorMap mA,
                                                                const __grid_constant__ CUtensorMap mB, SyrkArgs g) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sa = smem;                                 // kSySlices A tiles (128 rows)
  unsigned char* sb = smem + (size_t)kSySlices * kSyATile;  // kSySlices B tiles (64 rows)
  __shared__ uint64_t full, done;
  __shared__ uint32_t tmem_base;
  __shared__ volatile int abort_flag;
  // lower tiles (tm, tn), tn <= 2 tm + 1, from the linear block index b = tm (tm + 1) + tn
  const int b = (int)blockIdx.x;
  int tm = (int)((sqrtf(4.f * (float)b + 1.f) - 1.f) * 0.5f);
  while ((tm + 1) * (tm + 2) <= b) ++tm;
  while (tm * (tm + 1) > b) --tm;
  const int tn = b - tm * (tm + 1);
  const int row0 = tm * kSyM, col0 = tn * kSyN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    mbar_init(&full, 1);
    mbar_init(&done, 1);
    fence_mbar_init();
    fence_proxy_async();
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                 "r"(kSyTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  if (warp == 0) {
    if (lane == 0) {
      mbar_arrive_expect_tx(&full, (uint32_t)kSyBytes);
#pragma unroll
      for (int s = 0; s < kSySlices; ++s) {
        tma_load_2d(sa + (size_t)s * kSyATile, &mA, &full, 0, s * g.rest_pad + row0);
        tma_load_2d(sb + (size_t)s * kSyBTile, &mB, &full, 0, s * g.rest_pad + col0);
      }
      if (!mbar_wait(&full, 0u, g.st, 47)) abort_flag = 1;  // every copy has landed before exit
    }
  } else if (warp == 1) {
    if (lane == 0) {
      if (mbar_wait(&full, 0u, g.st, 48) && !abort_flag) {
        tc_fence_after();
        constexpr uint32_t idesc = idesc_bf16_f32(kSyM, kSyN);
#pragma unroll 1
        for (int lv = 2; lv <= kSySlices + 1; ++lv) {
          const uint32_t d_tmem = tmem + (uint32_t)((lv - 2) * kSyN);
          bool first = true;
          for (int s = 1; s <= lv - 1; ++s) {
            const int t = lv - s;
            if (s > kSySlices || t > kSySlices) continue;
            const uint64_t ad = smem_desc_sw128(sa + (size_t)(s - 1) * kSyATile);
            const uint64_t bd = smem_desc_sw128(sb + (size_t)(t - 1) * kSyBTile);
#pragma unroll
            for (int k = 0; k < kSyK / 16; ++k) {
              umma_bf16(d_tmem, ad + (uint64_t)(k * 2), bd + (uint64_t)(k * 2), idesc, (first && k == 0) ? 0u : 1u);
            }
            first = false;
          }
        }
        umma_commit(&done);
        if (!mbar_wait(&done, 0u, g.st, 49)) abort_flag = 1;
      } else {
        abort_flag = 1;
      }
    }
  } else {
    const int ew = warp - 2;           // 0..7
    const int quad = warp & 3;         // TMEM lane quadrant this warp may access
    const int cblk = ew >> 2;          // columns [32 cblk, 32 cblk + 32)
    const int row = quad * 32 + lane;  // tile row of this thread
    // the tile's row and column exponents, fetched while the MMAs run
    __shared__ int exr[kSyM], exc[kSyN];
    {
      const int t = threadIdx.x - 64;
      if (t < kSyM) exr[t] = row0 + t < g.rest_pad ? g.ex[row0 + t] : -1000;
      else if (t < kSyM + kSyN) exc[t - kSyM] = col0 + t - kSyM < g.rest_pad ? g.ex[col0 + t - kSyM] : -1000;
    }
    named_bar_sync(1, kSyEpiWarps * 32);
    const bool ok = mbar_wait_warp(&done, 0u, g.st, 50);
    tc_fence_after();
    const int ei = exr[row];
    // per thread (a TMEM lane = a tile row): the double-float update of 32 columns, staged in the
    // operand buffers (free once the MMAs are done) so that the read-modify-write of T below runs
    // along rows (coalesced)
    float* uh = reinterpret_cast<float*>(smem);                 // [kSyM][kSyN + 1]
    float* ul = uh + kSyM * (kSyN + 1);
    const bool live = ok && !abort_flag;
    if (live) {
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        const int c0 = cblk * 32 + half * 16;
        uint32_t vr[kSyLevels][16];
#pragma unroll
        for (int lv = 0; lv < kSyLevels; ++lv)
          tmem_ld16_nowait(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(lv * kSyN + c0), vr[lv]);
        tmem_ld_wait();
        float v[kSyLevels][16];
#pragma unroll
        for (int lv = 0; lv < kSyLevels; ++lv)
#pragma unroll
          for (int i = 0; i < 16; ++i) v[lv][i] = __uint_as_float(vr[lv][i]);
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const int ej = exc[c0 + jj];
          float sh = 0.f, sl = 0.f;
          if (ei > -1000 && ej > -1000) {
            // levels smallest first: term_l = acc_l 2^(e_i + e_j - 8 l), l = 2 .. kSySlices + 1
#pragma unroll
            for (int lv = kSyLevels - 1; lv >= 0; --lv) {
              const int E = ei + ej - 8 * (lv + 2);
              // exact: an integer below 2^24 times a power of two (terms below the float range vanish)
              const float x = (E >= -126 && E <= 127) ? v[lv][jj] * __int_as_float((127 + E) << 23)
                                                       : (E > 127 ? ldexpf(v[lv][jj], E) : 0.f);
              const float t = __fadd_rn(sh, x);
              const float bb = __fsub_rn(t, sh);
              sl = __fadd_rn(sl, __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bb)), __fsub_rn(x, bb)));
              sh = t;
            }
          }
          uh[row * (kSyN + 1) + c0 + jj] = sh;
          ul[row * (kSyN + 1) + c0 + jj] = sl;
        }
      }
    }
    named_bar_sync(1, kSyEpiWarps * 32);
    if (live) {
      // T_ij -= (uh + ul)_ij for the tile's lower part: warp ew takes rows ew, ew + 8, ...; lane = column.
      // All loads of T are issued before any store (independent addresses: one round trip per batch).
      constexpr int kRows = kSyM / kSyEpiWarps;  // 16 rows per warp
      constexpr int kCh = kSyN / 32;             // 2 column chunks
#pragma unroll 1
      for (int half = 0; half < 2; ++half) {
        float th[kRows / 2][kCh], tl[kRows / 2][kCh];
        bool in[kRows / 2][kCh];
#pragma unroll
        for (int q = 0; q < kRows / 2; ++q)
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            const int r = ew + kSyEpiWarps * (half * (kRows / 2) + q);
            const int ri = row0 + r, gj = col0 + c * 32 + lane;
            in[q][c] = ri < g.rest && gj < g.rest && gj <= ri;
            const long long gidx = (long long)ri * g.ldt + gj;
            th[q][c] = in[q][c] ? g.Th[gidx] : 0.f;
            tl[q][c] = in[q][c] ? g.Tl[gidx] : 0.f;
          }
#pragma unroll
        for (int q = 0; q < kRows / 2; ++q)
#pragma unroll
          for (int c = 0; c < kCh; ++c) {
            if (!in[q][c]) continue;
            const int r = ew + kSyEpiWarps * (half * (kRows / 2) + q);
            const int ri = row0 + r, gj = col0 + c * 32 + lane;
            const float sh = uh[r * (kSyN + 1) + c * 32 + lane], sl = ul[r * (kSyN + 1) + c * 32 + lane];
            const float s = __fsub_rn(th[q][c], sh);
            const float bb = __fsub_rn(s, th[q][c]);
            const float err = __fsub_rn(__fsub_rn(th[q][c], __fsub_rn(s, bb)), __fadd_rn(sh, bb));
            const float lo = __fadd_rn(err, __fsub_rn(tl[q][c], sl));
            const float nh = __fadd_rn(s, lo);
            const long long gidx = (long long)ri * g.ldt + gj;
            g.Th[gidx] = nh;
            g.Tl[gidx] = __fsub_rn(lo, __fsub_rn(nh, s));
          }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kSyTmemCols) : "memory");
  }
}

}  // namespace

size_t tc_syrk_ws_bytes(int n) {
  const size_t rp = (size_t)(n + kSyM - 1) / kSyM * kSyM;
  return (size_t)kSySlices * rp * kSyK * sizeof(__nv_bfloat16) + rp * sizeof(int) + 256;
}

sks_status tc_syrk_df32(cudaStream_t stream, int rest, const float* Ph, const float* Pl, long long ld, float* Th,
                        float* Tl, long long ldt, void* ws, size_t ws_bytes, DevStatus* st) {
  if (rest <= 0) return SKS_OK;
  if (ws_bytes < tc_syrk_ws_bytes(rest)) return fail(SKS_ERR_WORKSPACE, "tc_syrk: workspace too small");
  const int rest_pad = (rest + kSyM - 1) / kSyM * kSyM;
  unsigned char* base = (unsigned char*)(((uintptr_t)ws + 127) & ~(uintptr_t)127);
  __nv_bfloat16* SL = (__nv_bfloat16*)base;
  int* ex = (int*)(base + (size_t)kSySlices * rest_pad * kSyK * sizeof(__nv_bfloat16));
  const int sms = device_info().sms > 0 ? device_info().sms : 152;
  syrk_slice_kernel<<<(unsigned)std::min(sms * 8, (rest_pad + 7) / 8), 256, 0, stream>>>(rest, rest_pad, Ph, Pl, ld,
                                                                                          SL, ex);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  CUtensorMap mA, mB;
  SKS_TRY(make_tmap_2d_bf16_sw128(&mA, SL, (uint64_t)kSySlices * rest_pad, kSyK, kSyK, kSyM));
  SKS_TRY(make_tmap_2d_bf16_sw128(&mB, SL, (uint64_t)kSySlices * rest_pad, kSyK, kSyK, kSyN));
  SyrkArgs g;
  g.rest = rest;
  g.rest_pad = rest_pad;
  g.ex = ex;
  g.Th = Th;
  g.Tl = Tl;
  g.ldt = ldt;
  g.st = st;
  const int T = rest_pad / kSyM;
  const size_t smem = (size_t)kSyBytes + 1024;
  static bool attr_set = false;  // the size never changes; set once per process
  if (!attr_set) {
    SKS_CUDA_TRY(cudaFuncSetAttribute(tc_syrk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    attr_set = true;
  }
  tc_syrk_kernel<<<(unsigned)(T * (T + 1)), kSyThreads, smem, stream>>>(mA, mB, g);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

sks_status tc_unsplit(cudaStream_t stream, const __nv_bfloat16* Hh, const __nv_bfloat16* Hl, int rows, int cols,
                      int Kp, const double* sq, double* Y, long long ldy) {
  const long long total = (long long)rows * cols;
  if (total > 0) {
    unsplit_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(Hh, Hl, rows, cols, Kp, sq, Y, ldy);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  return SKS_OK;
}

size_t tc_gram_split_elems(int out_rows, int K) {
  const int Kp = (K + TBK - 1) / TBK * TBK;
  return (size_t)out_rows * Kp;
}

sks_status tc_split(cudaStream_t stream, const float* X, long long ldx, int rows, int cols, bool transpose,
                    const double* colscale, __nv_bfloat16* Hh, __nv_bfloat16* Hl, unsigned* rmax, int* Kp_out,
                    double* colfac) {
  const int out_rows = transpose ? cols : rows;
  const int K = transpose ? rows : cols;
  const int Kp = (K + TBK - 1) / TBK * TBK;
  const long long total = (long long)out_rows * Kp;
  if (colscale && !colfac) return fail(SKS_ERR_INVALID_ARG, "tc_split: column scaling needs colfac");
  const double* isq = nullptr;
  if (colscale && cols > 0) {
    colfac_kernel<<<(cols + 255) / 256, 256, 0, stream>>>(cols, colscale, colfac, colfac + cols);
    note_launch();
    isq = colfac;
  }
  if (total > 0) {
    SKS_CUDA_TRY(cudaMemsetAsync(rmax, 0, (size_t)out_rows * sizeof(unsigned), stream));
    const long long in_total = (long long)rows * cols;
    const unsigned g1 = transpose ? (unsigned)std::max<long long>(1, std::min<long long>((in_total + 255) / 256, 4096))
                                  : (unsigned)std::max<long long>(1, std::min<long long>((rows + 7) / 8, 4096));
    rowmax_kernel<<<g1, 256, 0, stream>>>(X, ldx, rows, cols, transpose ? 1 : 0, isq, rmax);
    note_launch();
    split_scaled_kernel<<<(unsigned)((total + 255) / 256), 256, 0, stream>>>(
        X, ldx, rows, cols, transpose ? 1 : 0, isq, rmax, out_rows, Kp, Hh, Hl);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  *Kp_out = Kp;
  return SKS_OK;
}

sks_status tc_gram(cudaStream_t stream, int M, int N, int Kp, const __nv_bfloat16* Ah, const __nv_bfloat16* Al,
                   const __nv_bfloat16* Bh, const __nv_bfloat16* Bl, double alpha, double beta, double* C,
                   long long ldc, bool lower, DevStatus* st) {
  if (M <= 0 || N <= 0) return SKS_OK;
  if (Kp % TBK != 0) return fail(SKS_ERR_INVALID_ARG, "tc_gram: K must be padded to 64");
  if (Kp == 0) return fail(SKS_ERR_INVALID_ARG, "tc_gram: K = 0");
  CUtensorMap mAh, mAl, mBh, mBl;
  auto mk = [&](CUtensorMap* m, const void* base, int rows) -> sks_status {
    return make_tmap_2d_bf16_sw128(m, base, (uint64_t)rows, (uint64_t)Kp, TBK, TBM);
  };
  SKS_TRY(mk(&mAh, Ah, M));
  SKS_TRY(mk(&mAl, Al, M));
  SKS_TRY(mk(&mBh, Bh, N));
  SKS_TRY(mk(&mBl, Bl, N));
  const int tm = (M + TBM - 1) / TBM, tn = (N + TBN - 1) / TBN;
  GramArgs g;
  g.M = M;
  g.N = N;
  g.Kp = Kp;
  g.tiles_n = tn;
  g.lower = lower ? 1 : 0;
  g.alpha = alpha;
  g.beta = beta;
  g.C = C;
  g.ldc = ldc;
  g.st = st;
  if (lower && tm != tn) return fail(SKS_ERR_INVALID_ARG, "tc_gram: lower needs a square tiling");
  const int tiles = lower ? tm * (tm + 1) / 2 : tm * tn;
  const size_t smem = (size_t)kStagesTC * kStageBytes + 1024;
  SKS_CUDA_TRY(cudaFuncSetAttribute(tc_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  tc_gram_kernel<<<tiles, kTcThreads, smem, stream>>>(mAh, mAl, mBh, mBl, g);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

}  // namespace sks

namespace sks {

// padded to whole 128-row stages of the 8-bit operand (two 64-row bf16 stages)
int tc_gauss_kp(long long n) { return (int)((std::max<long long>(n, 1) + 2 * GBK - 1) / (2 * GBK) * (2 * GBK)); }

int tc_gauss_slices(long long n) { return (tc_gauss_kp(n) + kGaussSlice - 1) / kGaussSlice; }

sks_status tc_split8_t(cudaStream_t stream, const float* A, long long lda, long long n, int d, unsigned char* A8t,
                       float* scale, unsigned* smax, double* frob2) {
  const int Kp = tc_gauss_kp(n);
  const int ks = tc_gauss_slices(n);
  SKS_CUDA_TRY(cudaMemsetAsync(smax, 0, (size_t)ks * d * sizeof(unsigned), stream));
  SKS_CUDA_TRY(cudaMemsetAsync(frob2, 0, sizeof(double), stream));
  if (n > 0) {
    const long long chunks = std::min<long long>((n + 1023) / 1024, 1024);
    const long long per = (n + chunks - 1) / chunks;
    e4m3_colmax_kernel<<<dim3((unsigned)((d + 127) / 128), (unsigned)chunks), 128, 0, stream>>>(A, lda, n, d, per,
                                                                                               kGaussSlice, smax, frob2);
    note_launch();
  }
  e4m3_scale_kernel<<<(unsigned)((ks * d + 255) / 256), 256, 0, stream>>>(ks * d, smax, scale);
  note_launch();
  split8_t_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)((d + 31) / 32)), dim3(32, 8), 0, stream>>>(
      A, lda, n, d, Kp, kGaussSlice, scale, A8t);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

size_t tc_gauss_part_elems(long long n, int d, int max_rows) {
  const int Kp = tc_gauss_kp(n);
  const int kc = kGaussSlice;
  const int ksplits = (Kp + kc - 1) / kc;
  return (size_t)ksplits * (size_t)std::max(1, std::min(max_rows, kGaussRowChunk)) * (size_t)d;
}

sks_status tc_split_t(cudaStream_t stream, const float* A, long long lda, long long n, int d, __nv_bfloat16* Hh,
                      __nv_bfloat16* Hl) {
  const int Kp = tc_gauss_kp(n);
  split_t_kernel<<<dim3((unsigned)(Kp / 32), (unsigned)((d + 31) / 32)), dim3(32, 8), 0, stream>>>(A, lda, n, d, Kp,
                                                                                                   Hh, Hl);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return SKS_OK;
}

sks_status tc_gauss_sketch(cudaStream_t stream, const __nv_bfloat16* Hh, const __nv_bfloat16* Hl, long long n, int d,
                           uint64_t seed, int m_off, int m_add, float* part, size_t part_elems, float* Y,
                           long long ldy, DevStatus* st, bool rademacher, const unsigned char* A8t,
                           const float* scale) {
  if (m_add <= 0) return SKS_OK;
  const int Kp = tc_gauss_kp(n);
  const bool e8 = A8t != nullptr;
  CUtensorMap mh, ml;
  if (e8) {
    if (rademacher) return fail(SKS_ERR_UNSUPPORTED, "the 8-bit sketch is Gaussian only");
    SKS_TRY(make_tmap_2d_u8_sw128(&mh, A8t, (uint64_t)d, (uint64_t)Kp, 2 * GBK, GBN));
    ml = mh;
  } else {
    SKS_TRY(make_tmap_2d_bf16_sw128(&mh, Hh, (uint64_t)d, (uint64_t)Kp, GBK, GBN));
    SKS_TRY(make_tmap_2d_bf16_sw128(&ml, Hl, (uint64_t)d, (uint64_t)Kp, GBK, GBN));
  }
  const size_t smem = (size_t)kGStages * kGStageBytes + 1024;
  auto kern = e8 ? tc_gauss_kernel<true> : tc_gauss_kernel<false>;
  SKS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int kc = kGaussSlice;
  const int ksplits = (Kp + kc - 1) / kc;
  for (int r0 = 0; r0 < m_add; r0 += kGaussRowChunk) {
    const int rows = std::min(kGaussRowChunk, m_add - r0);
    if ((size_t)ksplits * rows * d > part_elems) return fail(SKS_ERR_WORKSPACE, "Gaussian sketch partials too small");
    GaussArgs g;
    g.d = d;
    g.m_add = rows;
    g.row_base = m_off + r0;
    g.n = n;
    g.Kp = Kp;
    g.kc = kc;
    g.tiles_m = (rows + GBM - 1) / GBM;
    g.tiles_n = ((d + GBN - 1) / GBN + kGCluster - 1) / kGCluster * kGCluster;  // whole clusters
    g.ksplits = ksplits;
    g.key = make_key(seed);
    g.rade = rademacher ? 1 : 0;
    g.part = part;
    g.scale = scale;
    g.st = st;
    const long long blocks = (long long)g.tiles_m * g.tiles_n * ksplits;
    if (blocks > 0x7fffffffll) return fail(SKS_ERR_UNSUPPORTED, "Gaussian sketch grid too large");
    kern<<<(unsigned)blocks, kGThreads, smem, stream>>>(mh, ml, g);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
    const long long tot = (long long)rows * d;
    gauss_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, stream>>>(part, ksplits, rows, d, Y, ldy, m_off + r0);
    note_launch();
    SKS_CUDA_TRY(cudaGetLastError());
  }
  return SKS_OK;
}

}  // namespace sks
