// sketch.h -- host launchers of the embeddings (Section 2.1).
#pragma once

#include "internal.h"

namespace sks {

int ilog2_ceil(int64_t n);

// B = H_{+-1} E A_pad, B has 2^ceil(log2 n) rows.
template <typename T>
sks_status srht_form(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, T* B, long long ldb,
                     uint64_t seed);

// Y[r] = B[pi(r)], r in [r0, r1).
template <typename TB, typename TY>
sks_status srht_gather(cudaStream_t stream, const TB* B, long long ldb, int d, int64_t n_pad, uint64_t seed, int r0,
                       int r1, TY* Y, long long ldy, DevStatus* st);

// Y[m_off : m_off + m_add] = G[m_off : m_off + m_add, :] A (rademacher: the
// +-1 matrix of the Rademacher embedding instead of G).
template <typename T>
sks_status gaussian_extend(cudaStream_t stream, const T* A, long long lda, int64_t n, int d, uint64_t seed, int m_off,
                           int m_add, T* Y, long long ldy, T* gbuf, size_t gbuf_elems, T* split_ws,
                           size_t split_elems, bool rademacher = false);

// Y (m x d) = S A for the SJLT with s nonzeros per column.  sj_ws (optional,
// sjlt_gather_ws_elems words for float64, sjlt_table_bytes for float32) lets
// larger m gather each sketch row's data rows (float64) or keep the sketch
// rows on chip (float32, s <= 4, m <= 1024) instead of scattering them; st
// receives a timed-out wait of the on-chip kernel.
template <typename TA, typename TY>
sks_status sjlt_form(cudaStream_t stream, const TA* A, long long lda, int64_t n, int d, int m, int s, uint64_t seed,
                     TY* Y, long long ldy, uint32_t* sj_ws = nullptr, size_t sj_ws_elems = 0,
                     DevStatus* st = nullptr);
size_t sjlt_gather_ws_elems(int64_t n, int64_t m_max, int s);
size_t sjlt_table_bytes(int64_t n);

}  // namespace sks
