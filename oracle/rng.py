"""Counter-based random draws used by every sketch (oracle side).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper samples S "uniformly at random" (Section 2.1) without fixing a
generator.  To make the GPU path checkable bit for bit, both sides draw every
random number from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11), keyed by the 64-bit solver seed and
addressed by a 4-word counter whose last word names the stream:

    STREAM_GAUSS   counter (i, r // 4, 0, 1): Gaussian entries G[r, i], four
                   sketch rows per call, Box-Muller on two uniform pairs.
    STREAM_SIGN    counter (i, 0, 0, 2): SRHT sign E_i from the low bit of word 0.
    STREAM_FEISTEL counter (v, round, 0, 3): Feistel round function for the
                   SRHT row permutation pi.
    STREAM_SJLT    counter (i, a // 4, 0, 4): SJLT row candidates of data row i.
    STREAM_SJLT_SIGN counter (i, 0, 0, 5): SJLT signs of data row i (bit k of
                   word 0 for the k-th nonzero).
    STREAM_RADE    counter (i, r // 128, 0, 6): Rademacher entries R[r, i] of
                   sketch rows 128q .. 128q + 127, bit r % 32 of word
                   (r % 128) // 32 (set: -1, clear: +1).

This module implements those definitions in plain integer NumPy (uint64 holds
every 32x32 product exactly).  The GPU side implements the same published
generator independently in CUDA.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_GAUSS = 1
STREAM_SIGN = 2
STREAM_FEISTEL = 3
STREAM_SJLT = 4
STREAM_SJLT_SIGN = 5
STREAM_RADE = 6

FEISTEL_ROUNDS = 6
FEISTEL_MAX_WALK = 64
SJLT_MAX_ATTEMPTS = 256


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit Philox key words (low, high)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds, vectorised over broadcastable counters.

    One round maps (c0, c1, c2, c3) with key (k0, k1) to
        (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
    and the key is advanced by the Weyl constants (W0, W1) between rounds.
    Returns four uint32 arrays.
    """
    c0, c1, c2, c3 = [np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3)]
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return tuple(np.asarray(c, dtype=np.uint32) for c in (c0, c1, c2, c3))


def uniform_open01(word):
    """Uniform in (0, 1) from a uint32: ((w >> 9) * 2 + 1) * 2^-24.

    Exactly representable in float32 and float64, so both sides agree bit for
    bit on the uniforms; never 0 or 1, so log() below is finite.
    """
    w = np.asarray(word, dtype=np.uint64)
    return ((w >> np.uint64(9)) * np.uint64(2) + np.uint64(1)).astype(np.float64) * 2.0 ** -24


def rademacher_block(n_rows_data, m_rows, seed):
    """Matrix R (m_rows x n_rows_data) of +-1 entries, R[r, i] from bit r % 32
    of word (r % 128) // 32 of Philox at counter (i, r // 128, 0, STREAM_RADE)
    (set bit: -1).  Row r depends only on (seed, r): nested like the Gaussian."""
    k0, k1 = seed_key(seed)
    nq = (m_rows + 127) // 128
    i = np.arange(n_rows_data, dtype=np.uint64)[None, :]
    q = np.arange(nq, dtype=np.uint64)[:, None]
    words = philox4x32_10(i, q, 0, STREAM_RADE, k0, k1)  # 4 arrays of shape (nq, n)
    R = np.empty((128 * nq, n_rows_data), dtype=np.float64)
    for w in range(4):
        for b in range(32):
            bit = (words[w] >> np.uint64(b)) & np.uint64(1)
            R[128 * np.arange(nq) + 32 * w + b] = 1.0 - 2.0 * bit.astype(np.float64)
    return R[:m_rows]


def gaussian_block(n_rows_data, m_rows, seed):
    """Matrix G (m_rows x n_rows_data) of standard normals, G[r, i].

    Counter (i, r // 4, 0, STREAM_GAUSS); the four words (w0, w1, w2, w3) give
    u_j = uniform_open01(w_j) and
        G[4q+0] = sqrt(-2 ln u0) cos(2 pi u1),  G[4q+1] = sqrt(-2 ln u0) sin(2 pi u1),
        G[4q+2] = sqrt(-2 ln u2) cos(2 pi u3),  G[4q+3] = sqrt(-2 ln u2) sin(2 pi u3).
    Row r of G depends only on (seed, r), so growing m appends rows (nested
    sketches).
    """
    k0, k1 = seed_key(seed)
    nq = (m_rows + 3) // 4
    i = np.arange(n_rows_data, dtype=np.uint64)[None, :]
    q = np.arange(nq, dtype=np.uint64)[:, None]
    w0, w1, w2, w3 = philox4x32_10(i, q, 0, STREAM_GAUSS, k0, k1)
    u0, u1, u2, u3 = (uniform_open01(w) for w in (w0, w1, w2, w3))
    r01 = np.sqrt(-2.0 * np.log(u0))
    r23 = np.sqrt(-2.0 * np.log(u2))
    G = np.empty((4 * nq, n_rows_data), dtype=np.float64)
    G[0::4] = r01 * np.cos(2.0 * np.pi * u1)
    G[1::4] = r01 * np.sin(2.0 * np.pi * u1)
    G[2::4] = r23 * np.cos(2.0 * np.pi * u3)
    G[3::4] = r23 * np.sin(2.0 * np.pi * u3)
    return G[:m_rows]


def srht_signs(n_pad, seed):
    """Rademacher diagonal E of the SRHT: E_i = +1 iff bit 0 of word 0 of
    Philox(i, 0, 0, STREAM_SIGN) is 0."""
    k0, k1 = seed_key(seed)
    w0, _, _, _ = philox4x32_10(np.arange(n_pad, dtype=np.uint64), 0, 0, STREAM_SIGN, k0, k1)
    return np.where((w0 & np.uint32(1)) == 0, 1.0, -1.0)


def _feistel_round_value(v, rnd, k0, k1, half_bits):
    w0, _, _, _ = philox4x32_10(v, rnd, 0, STREAM_FEISTEL, k0, k1)
    return np.asarray(w0, dtype=np.uint64) & np.uint64((1 << half_bits) - 1)


def feistel_permute(x, n_pad, seed):
    """Pseudorandom bijection pi of [0, n_pad) (n_pad a power of two), applied to x.

    Balanced Feistel network (Luby-Rackoff) on 2h bits, h = ceil(log2(n_pad)/2),
    FEISTEL_ROUNDS rounds (L, R) -> (R, L xor F_j(R)) with F_j(R) = word 0 of
    Philox(R, j, 0, STREAM_FEISTEL) masked to h bits; values that land outside
    [0, n_pad) are re-encrypted (cycle walking, Black & Rogaway 2002) until they
    fall inside.  Used for the SRHT's row subsampling R: the sketch of size m
    takes rows pi(0), ..., pi(m-1), so a larger m keeps the previous rows.
    """
    x = np.asarray(x, dtype=np.uint64)
    if n_pad <= 1:
        return np.zeros_like(x)
    k = int(n_pad).bit_length() - 1
    assert (1 << k) == n_pad, "n_pad must be a power of two"
    h = (k + 1) // 2
    mask = np.uint64((1 << h) - 1)
    k0, k1 = seed_key(seed)

    def enc(v):
        L = v >> np.uint64(h)
        R = v & mask
        for j in range(FEISTEL_ROUNDS):
            L, R = R, L ^ _feistel_round_value(R, j, k0, k1, h)
        return (L << np.uint64(h)) | R

    v = enc(x)
    for _ in range(FEISTEL_MAX_WALK * 1024):  # the walk ends: enc is a bijection
        out = v >= np.uint64(n_pad)
        if not out.any():
            return v
        v = np.where(out, enc(v), v)
    raise RuntimeError("cycle walk did not terminate")


def sjlt_rows_signs(n_rows_data, m, s, seed):
    """Hash table of the SJLT with s nonzeros per column (Section 2.1).

    For data row i, attempt a uses word (a mod 4) of Philox(i, a // 4, 0,
    STREAM_SJLT) as w and proposes sketch row floor(m * w / 2^32); proposals
    already taken by data row i are skipped until s_eff = min(s, m) distinct
    rows are found (uniform sampling without replacement).  After
    SJLT_MAX_ATTEMPTS attempts any missing slots take the smallest unused rows
    (probability below 1e-30 for s <= 8).  The k-th nonzero has sign + iff bit k
    of word 0 of Philox(i, 0, 0, STREAM_SJLT_SIGN) is 0.
    Returns rows (n, s_eff) int64 and signs (n, s_eff) float64.
    """
    s_eff = min(int(s), int(m))
    k0, k1 = seed_key(seed)
    rows = np.full((n_rows_data, s_eff), -1, dtype=np.int64)
    # Draw candidate words in blocks of 4 attempts, vectorised over data rows.
    i_all = np.arange(n_rows_data, dtype=np.uint64)
    filled = np.zeros(n_rows_data, dtype=np.int64)
    for blk in range(SJLT_MAX_ATTEMPTS // 4):
        todo = filled < s_eff
        if not todo.any():
            break
        w = philox4x32_10(i_all, blk, 0, STREAM_SJLT, k0, k1)
        for j in range(4):
            cand = ((np.asarray(w[j], dtype=np.uint64) * np.uint64(m)) >> np.uint64(32)).astype(np.int64)
            todo = filled < s_eff
            dup = (rows == cand[:, None]).any(axis=1)
            take = todo & ~dup
            idx = np.nonzero(take)[0]
            rows[idx, filled[idx]] = cand[idx]
            filled[idx] += 1
    for i in np.nonzero(filled < s_eff)[0]:
        used = set(rows[i, : filled[i]].tolist())
        r = 0
        while filled[i] < s_eff:
            if r not in used:
                rows[i, filled[i]] = r
                filled[i] += 1
            r += 1
    ws, _, _, _ = philox4x32_10(i_all, 0, 0, STREAM_SJLT_SIGN, k0, k1)
    ws = np.asarray(ws, dtype=np.uint64)
    bits = (ws[:, None] >> np.arange(s_eff, dtype=np.uint64)[None, :]) & np.uint64(1)
    signs = np.where(bits == 0, 1.0, -1.0)
    return rows, signs
