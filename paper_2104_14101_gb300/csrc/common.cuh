// common.cuh -- shared device/host utilities of the sks library (sm_103a).
//
// * status plumbing: a device-side status word that kernels raise with
//   atomicCAS (first error wins) and the host reads once per solve step;
// * Philox4x32-10 (Salmon et al., SC'11) and the keyed draws every sketch
//   takes from it -- SRHT signs, the Feistel row permutation, Gaussian
//   variates, SJLT hashes -- defined by (seed, counter, stream id);
// * block reductions;
// * mbarrier / bulk-tensor-copy (TMA) wrappers with time-bounded waits.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sks.h"

#define SKS_DEV __device__ __forceinline__
#define SKS_HD __host__ __device__ __forceinline__

namespace sks {

// ---------------------------------------------------------------- status
// Device status block (lives at the start of every workspace).
struct DevStatus {
  int code;       // sks_status, 0 = OK; first error wins
  int where;      // small integer identifying the raising kernel
  long long aux;  // extra detail (row index, pivot number, ...)
};

SKS_DEV void raise_status(DevStatus* st, int code, int where, long long aux) {
  if (st == nullptr) return;
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->where = where;
    st->aux = aux;
  }
}

// ---------------------------------------------------------------- Philox4x32-10
enum Stream : uint32_t {
  STREAM_GAUSS = 1,
  STREAM_SIGN = 2,
  STREAM_FEISTEL = 3,
  STREAM_SJLT = 4,
  STREAM_SJLT_SIGN = 5,
  STREAM_RADE = 6,
};

constexpr int kFeistelRounds = 6;
constexpr int kFeistelMaxWalk = 64;
constexpr int kSjltMaxAttempts = 256;
constexpr int kSjltMaxS = 16;

SKS_HD uint32_t mulhi32(uint32_t a, uint32_t b) {
  return (uint32_t)(((uint64_t)a * (uint64_t)b) >> 32);
}

// Ten rounds of the Philox4x32 bijection; the key advances by the Weyl
// constants between rounds.
SKS_HD uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t p0h = mulhi32(0xD2511F53u, c.x), p0l = 0xD2511F53u * c.x;
    const uint32_t p1h = mulhi32(0xCD9E8D57u, c.z), p1l = 0xCD9E8D57u * c.z;
    c = make_uint4(p1h ^ c.y ^ k0, p1l, p0h ^ c.w ^ k1, p0l);
  }
  return c;
}

struct Key {
  uint32_t k0, k1;
};
SKS_HD Key make_key(uint64_t seed) { return Key{(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)}; }

// Uniform on (0,1): ((w >> 9) * 2 + 1) * 2^-24, exact in float and double.
SKS_HD double u01_d(uint32_t w) { return (double)(((w >> 9) << 1) | 1u) * 0x1p-24; }
SKS_HD float u01_f(uint32_t w) { return (float)(((w >> 9) << 1) | 1u) * 0x1p-24f; }

// Sign E_i of the SRHT: +1 iff bit 0 of word 0 of Philox(i, 0, 0, SIGN) is 0.
SKS_HD double srht_sign(Key k, uint32_t i) {
  return (philox(make_uint4(i, 0u, 0u, STREAM_SIGN), k.k0, k.k1).x & 1u) ? -1.0 : 1.0;
}

// Feistel permutation of [0, 2^bits) (bits >= 1), 2h-bit network with cycle
// walking.  Returns 0xffffffff if the walk exceeds kFeistelMaxWalk steps.
SKS_HD uint32_t feistel_perm(Key k, uint32_t x, int bits) {
  if (bits <= 0) return 0u;
  const int h = (bits + 1) / 2;
  const uint32_t mask = (1u << h) - 1u;
  const uint32_t n = 1u << bits;
  uint32_t v = x;
  for (int walk = 0; walk < kFeistelMaxWalk; ++walk) {
    uint32_t L = v >> h, R = v & mask;
    for (int j = 0; j < kFeistelRounds; ++j) {
      const uint32_t f = philox(make_uint4(R, (uint32_t)j, 0u, STREAM_FEISTEL), k.k0, k.k1).x & mask;
      const uint32_t t = L ^ f;
      L = R;
      R = t;
    }
    v = (L << h) | R;
    if (v < n) return v;
  }
  return 0xffffffffu;
}

// SJLT hash of data row i: s_eff distinct rows in [0, m) and their signs
// (+1 iff bit k of word 0 of Philox(i, 0, 0, SJLT_SIGN) is 0).  Attempt a
// proposes floor(m * w / 2^32), w = word (a mod 4) of Philox(i, a/4, 0, SJLT);
// duplicates are skipped; after kSjltMaxAttempts attempts the missing slots
// take the smallest unused rows.
SKS_HD int sjlt_hash(Key k, uint32_t i, uint32_t m, int s_eff, uint32_t* rows, float* signs) {
  int filled = 0;
  for (int blk = 0; blk < kSjltMaxAttempts / 4 && filled < s_eff; ++blk) {
    const uint4 w = philox(make_uint4(i, (uint32_t)blk, 0u, STREAM_SJLT), k.k0, k.k1);
    const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
    for (int j = 0; j < 4 && filled < s_eff; ++j) {
      const uint32_t cand = mulhi32(ws[j], m);
      bool dup = false;
      for (int q = 0; q < filled; ++q) dup |= (rows[q] == cand);
      if (!dup) rows[filled++] = cand;
    }
  }
  for (uint32_t r = 0; filled < s_eff; ++r) {
    bool used = false;
    for (int q = 0; q < filled; ++q) used |= (rows[q] == r);
    if (!used) rows[filled++] = r;
  }
  const uint32_t sb = philox(make_uint4(i, 0u, 0u, STREAM_SJLT_SIGN), k.k0, k.k1).x;
  for (int q = 0; q < s_eff; ++q) signs[q] = ((sb >> q) & 1u) ? -1.0f : 1.0f;
  return s_eff;
}

// Rademacher entries of sketch rows 4Q .. 4Q+3 for data row i: bits
// (4Q) % 32 .. +3 of word (4Q % 128) / 32 of Philox at (i, 4Q / 128, 0, 6);
// a set bit is -1.
SKS_DEV void rade4_f(Key k, uint32_t i, uint32_t Q, float g[4]) {
  const uint32_t r0 = 4u * Q;
  const uint4 w = philox(make_uint4(i, r0 >> 7, 0u, STREAM_RADE), k.k0, k.k1);
  const uint32_t sel = (r0 >> 5) & 3u;
  const uint32_t word = sel == 0 ? w.x : (sel == 1 ? w.y : (sel == 2 ? w.z : w.w));
  const uint32_t bits = word >> (r0 & 31u);
#pragma unroll
  for (int t = 0; t < 4; ++t) g[t] = ((bits >> t) & 1u) ? -1.f : 1.f;
}

// Four N(0,1) variates of quad q of data row i (sketch rows 4q..4q+3),
// Box-Muller on two uniform pairs, float64.
SKS_DEV void gauss4_d(Key k, uint32_t i, uint32_t q, double g[4]) {
  const uint4 w = philox(make_uint4(i, q, 0u, STREAM_GAUSS), k.k0, k.k1);
  const double r01 = sqrt(-2.0 * log(u01_d(w.x)));
  const double r23 = sqrt(-2.0 * log(u01_d(w.z)));
  double s1, c1, s3, c3;
  sincospi(2.0 * u01_d(w.y), &s1, &c1);
  sincospi(2.0 * u01_d(w.w), &s3, &c3);
  g[0] = r01 * c1;
  g[1] = r01 * s1;
  g[2] = r23 * c3;
  g[3] = r23 * s3;
}

// Same in float32 arithmetic (the mixed form rounds these to bfloat16).
SKS_DEV void gauss4_f(Key k, uint32_t i, uint32_t q, float g[4]) {
  const uint4 w = philox(make_uint4(i, q, 0u, STREAM_GAUSS), k.k0, k.k1);
  const float r01 = sqrtf(-2.0f * logf(u01_f(w.x)));
  const float r23 = sqrtf(-2.0f * logf(u01_f(w.z)));
  float s1, c1, s3, c3;
  sincospif(2.0f * u01_f(w.y), &s1, &c1);
  sincospif(2.0f * u01_f(w.w), &s3, &c3);
  g[0] = r01 * c1;
  g[1] = r01 * s1;
  g[2] = r23 * c3;
  g[3] = r23 * s3;
}

// ---------------------------------------------------------------- reductions
template <typename T>
SKS_DEV T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the whole block (blockDim.x a multiple of 32, <= 1024); every
// thread receives the result.  `scratch` holds >= 32 T.
template <typename T>
SKS_DEV T block_sum(T v, T* scratch) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) scratch[w] = v;
  __syncthreads();
  T t = (lane < nw) ? scratch[lane] : T(0);
  t = warp_sum(t);
  return t;
}

// ---------------------------------------------------------------- mbarrier / TMA
SKS_DEV uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

SKS_DEV void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

SKS_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
SKS_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

SKS_DEV void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar)) : "memory");
}

SKS_DEV void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

SKS_DEV bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

SKS_DEV uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait: returns false (and raises SKS_ERR_TIMEOUT) once `limit_ns`
// nanoseconds have passed without the phase completing.
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s
SKS_DEV bool mbar_wait(uint64_t* bar, uint32_t parity, DevStatus* st, int where, uint64_t limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) {
      raise_status(st, SKS_ERR_TIMEOUT, where, 0);
      return false;
    }
  }
}

// Warp-uniform bounded wait: every lane polls, lane 0 keeps the clock, and the
// verdict is the same in all 32 lanes (safe before warp shuffles / barriers).
SKS_DEV bool mbar_wait_warp(uint64_t* bar, uint32_t parity, DevStatus* st, int where) {
  const int lane = threadIdx.x & 31;
  uint64_t t0 = 0;
  while (true) {
    const bool ok = mbar_try_wait(bar, parity);
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

// 2-D tiled bulk tensor copy global -> shared, completion counted on `bar`.
SKS_DEV void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_addr(dst)),
      "l"((uint64_t)map), "r"(smem_addr(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16).
SKS_DEV void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
      "l"((uint64_t)src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

SKS_DEV void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Named barrier that also returns the OR of a predicate over its threads.
SKS_DEV bool named_bar_or(int id, int nthreads, bool pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred pi, po;\n\tsetp.ne.b32 pi, %1, 0;\n\tbar.red.or.pred po, %2, %3, pi;\n\t"
      "selp.b32 %0, 1, 0, po;\n\t}"
      : "=r"(r)
      : "r"((int)pred), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

}  // namespace sks
