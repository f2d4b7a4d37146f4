// tile.cuh -- device routines for one segment ("tile") of the residue bitmaps.
//
// A CTA owns one tile at a time; its two bitmaps (class 1 and class 5, one bit
// per candidate) live in shared memory (Sections 2.1-2.3: each worker sieves
// its own contiguous chunk in private memory, so no two workers write the same
// address).
//
// Bit-sliced layout: a tile of L = 32 W indices per class (W a power of two)
// stores index k in word (k mod W), bit (k div W).  Shared-memory word w sits
// in bank w mod 32 = k mod 32, so the 32 lanes of a warp that strike one prime
// P at k, k + P, ..., k + 31 P always touch 32 different banks (P is odd): the
// warp-cooperative strikes are free of bank conflicts for every P.  Row b of
// the tile (bit b of every word) is the contiguous index run [b W, b W + W).
#pragma once

#include "sieve_internal.cuh"

namespace sieve {

// device copy of kPatternPrimes (one per translation unit)
static __constant__ uint32_t c_pattern_primes[kNumPatterns][6] = {
    {5, 7, 11, 13, 17, 19}, {23, 29, 31, 0, 0, 0},    {37, 41, 43, 0, 0, 0},
    {47, 53, 59, 0, 0, 0},  {61, 67, 71, 0, 0, 0},    {73, 79, 83, 0, 0, 0},
    {89, 97, 101, 0, 0, 0}, {103, 107, 109, 0, 0, 0}, {113, 127, 131, 0, 0, 0}};

__device__ __forceinline__ uint32_t rotl32(uint32_t x, uint32_t s) { return __funnelshift_l(x, x, s); }

// floor(sqrt(n)) for n < 2^63: a double estimate, then integer correction.
__device__ __forceinline__ uint64_t isqrt_dev(uint64_t n) {
  uint64_t r = (uint64_t)sqrt((double)n);
  while (r * r > n) r--;
  while ((r + 1) * (r + 1) <= n) r++;
  return r;
}

// Number of entries <= s in the increasing array a[0..n); warp-collective
// 32-ary search (every lane returns the answer).
__device__ __forceinline__ uint32_t warp_count_le(const uint32_t *a, uint32_t n, uint64_t s) {
  const uint32_t lane = threadIdx.x & 31;
  uint32_t lo = 0, hi = n;  // answer in [lo, hi]
  while (hi - lo > 32) {
    uint32_t step = (hi - lo + 31) / 32;
    uint32_t idx = lo + lane * step;
    bool le = idx < hi && (uint64_t)__ldg(a + idx) <= s;
    uint32_t c = __popc(__ballot_sync(kFullMask, le));
    if (c == 0) return lo;
    uint32_t nlo = lo + (c - 1) * step + 1;
    uint32_t nhi = lo + c * step;
    lo = nlo;
    hi = nhi < hi ? nhi : hi;
  }
  uint32_t idx = lo + lane;
  bool le = idx < hi && (uint64_t)__ldg(a + idx) <= s;
  return lo + __popc(__ballot_sync(kFullMask, le));
}

// Tile geometry shared by the phases.
struct TileGeom {
  uint32_t W;     // words per class (power of two, multiple of 32)
  uint32_t logW;  // log2(W)
  uint32_t len;   // indices in use (<= 32 W)
};

// K0 mod period of pattern g (the tile's offset into it).
__device__ __forceinline__ uint32_t pattern_offset(uint64_t K0, const PatternDesc &pd) {
  return (uint32_t)(K0 - div_invariant(K0, pd.period, pd.magic) * pd.period);
}

// Presieve copy.  For pattern g (period P_g), the sliced pattern T_g holds, at
// word j, bit b = pattern bit (j + b W) mod P_g; so tile word w is
// T_g[(K0 mod P_g) + w], a contiguous, coalesced copy.  Words of all patterns
// in use are ANDed.  `o_given`, when given, holds the tile's offsets K0 mod
// P_g (computed ahead by the caller); else every thread computes them.
template <int BLOCK>
__device__ __forceinline__ void presieve_copy(uint32_t *s1, uint32_t *s5, const TileGeom &tg, uint64_t K0,
                                              const uint32_t *__restrict__ sliced, const PatternDesc *pd,
                                              int npat, const uint32_t *o_given = nullptr) {
  uint32_t o[kNumPatterns];
#pragma unroll
  for (int g = 0; g < kNumPatterns; g++)
    if (g < npat) o[g] = o_given ? o_given[g] : pattern_offset(K0, pd[g]);
  for (uint32_t w = threadIdx.x; w < tg.W; w += BLOCK) {
    uint32_t v1 = 0xFFFFFFFFu, v5 = 0xFFFFFFFFu;
#pragma unroll
    for (int g = 0; g < kNumPatterns; g++) {
      if (g < npat) {
        v1 &= __ldg(sliced + pd[g].off1 + o[g] + w);
        v5 &= __ldg(sliced + pd[g].off5 + o[g] + w);
      }
    }
    s1[w] = v1;
    s5[w] = v5;
  }
}

// Strike indices k = k0, k0 + step, ... < len in bitmap s (Section 3: the
// index advances by P, the value by 6P).  Clearing is an atomic AND in shared
// memory because several lanes may clear bits of one word.  Eight strikes
// per loop trip (measured better than four) and a short tail keep the branch
// count low.  step < 2^29.
__device__ __forceinline__ void strike_one(uint32_t *s, uint32_t k, uint32_t wmask, uint32_t logW) {
  atomicAnd(s + (k & wmask), rotl32(0xFFFFFFFEu, k >> logW));
}

__device__ __forceinline__ void strike(uint32_t *s, uint32_t k, uint32_t step, uint32_t len, uint32_t wmask,
                                       uint32_t logW) {
  if (step < len) {
    const uint32_t s2 = 2 * step, s3 = 3 * step, s4 = 4 * step, s8 = 8 * step;
    for (; k + s4 + s3 < len; k += s8) {
      strike_one(s, k, wmask, logW);
      strike_one(s, k + step, wmask, logW);
      strike_one(s, k + s2, wmask, logW);
      strike_one(s, k + s3, wmask, logW);
      strike_one(s, k + s4, wmask, logW);
      strike_one(s, k + s4 + step, wmask, logW);
      strike_one(s, k + s4 + s2, wmask, logW);
      strike_one(s, k + s4 + s3, wmask, logW);
    }
    if (k + s3 < len) {
      strike_one(s, k, wmask, logW);
      strike_one(s, k + step, wmask, logW);
      strike_one(s, k + s2, wmask, logW);
      strike_one(s, k + s3, wmask, logW);
      k += s4;
    }
    if (k + s2 < len) strike_one(s, k + s2, wmask, logW);
    if (k + step < len) strike_one(s, k + step, wmask, logW);
  }
  if (k < len) strike_one(s, k, wmask, logW);
}

// Start indices of the warp-band primes [i_first, i_split) for the tile with
// base B (the inverse-of-6 form where P^2 <= B, else Table 1 with the P^2
// clamp), one prime per thread, into shared memory (as 32-bit indices; a
// start >= len means no hit, kept as len).
template <int BLOCK>
__device__ __forceinline__ void warp_band_starts(uint2 *starts, uint64_t B, uint32_t len,
                                                 const uint32_t *__restrict__ primes,
                                                 const uint64_t *__restrict__ magic,
                                                 const uint2 *__restrict__ cinv, uint32_t i_first,
                                                 uint32_t i_split) {
  for (uint32_t i = i_first + threadIdx.x; i < i_split; i += BLOCK) {
    const uint32_t P = __ldg(primes + i);
    uint64_t k1, k5;
    if ((uint64_t)P * P <= B && P < 0x80000000u) {  // the inverse-of-6 start (= Table 1's)
      uint32_t a1, a5;
      starts_from_inverse(B / 6, P, __ldg(magic + i), __ldg(cinv + i), a1, a5);
      k1 = a1;
      k5 = a5;
    } else {
      tile_starts(B, P, __ldg(magic + i), k1, k5);
    }
    starts[i - i_first] = make_uint2(k1 < len ? (uint32_t)k1 : len, k5 < len ? (uint32_t)k5 : len);
  }
}

// Strike every base prime with index in [i_first, np) into the tile whose
// index 0 is value B.  Primes with index below i_split are struck by a whole
// warp (lane l takes hits l, l + 32, ... of the prime; bank-conflict free in
// the sliced layout) from the starts precomputed in shared memory, handed out
// one at a time through a shared counter so that warps finish together; the
// rest by one lane each, which locates the prime's first hits from its
// inverse-of-6 constants (cinv; the Table 1 start, see starts_from_inverse)
// or, where the P^2 clamp can apply, with Table 1 itself (K0 = B / 6; all_sq: the caller
// knows that every prime below np has P^2 <= B and P < 2^31, so the test per
// prime is skipped).  (Loading the
// constants only for primes below the tile span, so that larger ones keep a
// one-remainder miss test, was slower: the load then waits for the prime.)
template <int BLOCK, bool PREFETCH = false>
__device__ __forceinline__ void strike_lane_band(uint32_t *s1, uint32_t *s5, uint64_t B, const TileGeom &tg,
                                                 const uint32_t *__restrict__ primes,
                                                 const uint64_t *__restrict__ magic,
                                                 const uint2 *__restrict__ cinv, uint32_t i_lo, uint32_t np,
                                                 bool all_sq, uint64_t K0);

template <int BLOCK, bool PREFETCH = false>
__device__ __forceinline__ void strike_primes(uint32_t *s1, uint32_t *s5, uint64_t B, const TileGeom &tg,
                                              const uint32_t *__restrict__ primes,
                                              const uint64_t *__restrict__ magic, const uint2 *__restrict__ cinv,
                                              const uint2 *starts, uint32_t i_first, uint32_t i_split, uint32_t np,
                                              bool all_sq, uint32_t *next, uint64_t K0,
                                              uint32_t lane_end = 0xFFFFFFFFu) {
  const uint32_t lane = threadIdx.x & 31;
  const uint32_t split = i_split < np ? i_split : np;
  const uint32_t len = tg.len, wmask = tg.W - 1, logW = tg.logW;
  for (;;) {
    uint32_t i = 0;
    if (lane == 0) i = atomicAdd(next, 1u);
    i = __shfl_sync(kFullMask, i, 0);
    if (i >= split) break;
    const uint32_t P = __ldg(primes + i);
    const uint2 st = starts[i - i_first];
    const uint32_t k1 = st.x + lane * P, k5 = st.y + lane * P;
    if (k1 < len) strike(s1, k1, 32u * P, len, wmask, logW);
    if (k5 < len) strike(s5, k5, 32u * P, len, wmask, logW);
  }
  // primes from the warp band's end up to np (or lane_end: above it the
  // bucket sieve applies them) by one lane each
  strike_lane_band<BLOCK, PREFETCH>(s1, s5, B, tg, primes, magic, cinv, split > i_first ? split : i_first,
                                    np < lane_end ? np : lane_end, all_sq, K0);
}

// L2 prefetch (TMA bulk prefetch, a hint: no data moves to the SM) of the
// table entries [a, b) of the primes, their reciprocals and their inverse-of-6
// constants; the spans are cut to 16-byte boundaries inside each array.
__device__ __forceinline__ void prefetch_table_l2(const uint32_t *primes, const uint64_t *magic, const uint2 *cinv,
                                                  uint32_t a, uint32_t b) {
  if (b <= a) return;
  auto pf = [](const void *base, uint32_t elem, uint32_t a, uint32_t b) {
    const uintptr_t s = ((uintptr_t)base + (uintptr_t)a * elem + 15) & ~(uintptr_t)15;
    const uintptr_t e = ((uintptr_t)base + (uintptr_t)b * elem) & ~(uintptr_t)15;
    if (e > s) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s), "r"((uint32_t)(e - s)) : "memory");
  };
  pf(primes, 4, a, b);
  pf(magic, 8, a, b);
  pf(cinv, 8, a, b);
}

// Blocks of BLOCK primes by which thread 0 keeps the table ahead of the
// one-lane band: far up a lane's prime costs a few dozen instructions, far
// less than a table line's trip from DRAM.  Only entries from index
// kLanePrefetchFirst on (primes above about 3.5e7, 40 MB of table below them)
// are prefetched: those stream from DRAM, while the table below stays in L2,
// where the prefetches only cost (the 4096-query batch, whose primes stop
// below it: 12.4 -> 13.6 ms with them; serving requests up to 1e18: 24.2 ->
// 22.4 ms per 512).  Only the batch kernel, which serves the far requests,
// is compiled with them: in the range kernel the untaken test alone cost 2 %
// at the headline.
constexpr uint32_t kLanePrefetchBlocks = 4;
constexpr uint32_t kLanePrefetchFirst = 1u << 21;

// Strike the primes with table index in [i_lo, np) into the tile whose index
// 0 is value B (K0 = B / 6), one lane per prime: each lane locates its prime's
// first hits from the inverse-of-6 constants (the Table 1 start, see
// starts_from_inverse) or, where the P^2 clamp can apply, with Table 1 itself
// (all_sq: the caller knows that every prime below np has P^2 <= B and
// P < 2^31, so the test per prime is skipped).  PREFETCH: thread 0 keeps the
// far part of the table (see kLanePrefetchFirst) in L2 ahead of the lanes.
template <int BLOCK, bool PREFETCH>
__device__ __forceinline__ void strike_lane_band(uint32_t *s1, uint32_t *s5, uint64_t B, const TileGeom &tg,
                                                 const uint32_t *__restrict__ primes,
                                                 const uint64_t *__restrict__ magic,
                                                 const uint2 *__restrict__ cinv, uint32_t i_lo, uint32_t np,
                                                 bool all_sq, uint64_t K0) {
  const uint32_t len = tg.len, wmask = tg.W - 1, logW = tg.logW, span6 = 6 * tg.len;
  // one lane per prime; the next prime's table entries are loaded before the
  // current prime is struck so that their latency overlaps the strikes.  The
  // loop is unrolled by two with the prefetched entries alternating between
  // two register sets (fewer moves than rotating one set; measured).
  auto lane_loop = [&](auto &&one) {
    uint32_t i = i_lo + threadIdx.x;
    uint32_t P = 0;
    uint64_t m = 0;
    uint2 c = make_uint2(0, 0);
    constexpr uint32_t kAhead = kLanePrefetchBlocks * BLOCK;
    const bool far = PREFETCH && np > kLanePrefetchFirst;  // the stream reaches the table kept in DRAM
    auto ahead = [&](uint32_t a, uint32_t b) {  // [a, b) within [kLanePrefetchFirst, np)
      prefetch_table_l2(primes, magic, cinv, a > kLanePrefetchFirst ? a : kLanePrefetchFirst, b < np ? b : np);
    };
    if (far && threadIdx.x == 0) ahead(i_lo, i_lo + kAhead);
    if (i < np) {
      P = __ldg(primes + i);
      m = __ldg(magic + i);
      c = __ldg(cinv + i);
    }
    while (i < np) {
      // thread 0 (at i = i_lo + 2 k BLOCK) requests the two blocks that come
      // into the prefetch window as the CTA moves on by two blocks
      if (far && threadIdx.x == 0) ahead(i + kAhead, i + kAhead + 2 * BLOCK);
      const uint32_t in = i + BLOCK;
      uint32_t Pb = 0;
      uint64_t mb = 0;
      uint2 cb = make_uint2(0, 0);
      if (in < np) {
        Pb = __ldg(primes + in);
        mb = __ldg(magic + in);
        cb = __ldg(cinv + in);
      }
      one(P, m, c);
      if (in >= np) break;
      const uint32_t in2 = in + BLOCK;
      if (in2 < np) {
        P = __ldg(primes + in2);
        m = __ldg(magic + in2);
        c = __ldg(cinv + in2);
      }
      one(Pb, mb, cb);
      i = in2;
    }
  };
  // a plain loop per class: one-lane primes have few hits per tile, so the
  // unrolled loop's set-up costs more than it saves (measured); k + P < 2^32
  auto strike_from = [&](uint32_t Pq, uint32_t k1, uint32_t k5) {
    for (uint32_t k = k1; k < len; k += Pq) strike_one(s1, k, wmask, logW);
    for (uint32_t k = k5; k < len; k += Pq) strike_one(s5, k, wmask, logW);
  };
  if (all_sq) {  // every prime has P^2 <= B and P < 2^31: no clamp to test for
    lane_loop([&](uint32_t Pq, uint64_t mq, uint2 cq) {
      uint32_t k1, k5;
      starts_from_inverse(K0, Pq, mq, cq, k1, k5);
      strike_from(Pq, k1, k5);
    });
  } else {
    lane_loop([&](uint32_t Pq, uint64_t mq, uint2 cq) {
      uint32_t k1 = len, k5 = len;
      if ((uint64_t)Pq * Pq <= B && Pq < 0x80000000u) {
        starts_from_inverse(K0, Pq, mq, cq, k1, k5);
      } else {
        uint64_t a1, a5;
        if (tile_starts_within(B, Pq, mq, span6, a1, a5)) {
          k1 = a1 < len ? (uint32_t)a1 : len;
          k5 = a5 < len ? (uint32_t)a5 : len;
        }
      }
      strike_from(Pq, k1, k5);
    });
  }
}

// ceil(a / 6) for signed a.
__device__ __forceinline__ int64_t ceil_div6(int64_t a) { return -floor_div6(-a); }

// Low n bits (n clamped to [0, 32]).
__device__ __forceinline__ uint32_t low_bits(int64_t n) {
  return n <= 0 ? 0u : (n >= 32 ? 0xFFFFFFFFu : ((1u << n) - 1u));
}

// Bits b of word w whose index w + b W lies below t: b < ceil((t - w) / W).
__device__ __forceinline__ uint32_t below_mask(int64_t t, uint32_t w, uint32_t logW, uint32_t W) {
  const int64_t d = t - (int64_t)w;
  return d <= 0 ? 0u : low_bits((d + W - 1) >> logW);
}

// Valid indices of class r in a tile with base B: lo <= B + 6 k + r < hi.
struct ValidRange {
  int64_t kl1, kh1, kl5, kh5;
};

__device__ __forceinline__ ValidRange valid_range(uint64_t lo, uint64_t hi, uint64_t B, uint32_t len) {
  ValidRange v;
  const int64_t dl = (int64_t)lo - (int64_t)B, dh = (int64_t)hi - (int64_t)B;
  v.kl1 = ceil_div6(dl - 1);
  v.kl5 = ceil_div6(dl - 5);
  v.kh1 = ceil_div6(dh - 1);
  v.kh5 = ceil_div6(dh - 5);
  v.kl1 = v.kl1 < 0 ? 0 : v.kl1;
  v.kl5 = v.kl5 < 0 ? 0 : v.kl5;
  v.kh1 = v.kh1 > (int64_t)len ? (int64_t)len : (v.kh1 < 0 ? 0 : v.kh1);
  v.kh5 = v.kh5 > (int64_t)len ? (int64_t)len : (v.kh5 < 0 ? 0 : v.kh5);
  return v;
}

// Fix-ups after striking (Section 2.1: the arrays hold candidates > 3):
//   * tiles holding values up to the largest presieved prime: clear the value
//     1 and restore the presieved primes themselves (their patterns removed
//     them together with their multiples);
//   * edge tiles: clear the bits outside [lo, hi) and past len.
template <int BLOCK>
__device__ __forceinline__ void fixup_tile(uint32_t *s1, uint32_t *s5, const TileGeom &tg, uint64_t K0,
                                           const ValidRange &v, int npat) {
  // Nothing to fix in a tile above the presieved primes that lies inside the
  // range (most tiles): return at once, without the barriers.  The condition
  // is the same for every thread of the block.  Otherwise the tile is ready
  // when this returns (it ends with a barrier).
  const int64_t full = 32 * (int64_t)tg.W;
  const bool small = 6 * K0 <= 131;
  const bool edge = v.kl1 > 0 || v.kl5 > 0 || v.kh1 < full || v.kh5 < full;
  if (!small && !edge) return;
  if (threadIdx.x == 0 && small) {
    if (K0 == 0) s1[0] &= ~1u;  // 1 is not a prime (index 0: word 0, bit 0)
    for (int g = 0; g < npat; g++) {
      for (int q = 0; q < 6; q++) {
        const uint32_t wv = c_pattern_primes[g][q];
        if (wv == 0) continue;
        const uint32_t r = wv % 6, k = wv / 6;
        if (k >= K0 && k - K0 < tg.len) {
          const uint32_t kk = (uint32_t)(k - K0);
          (r == 1 ? s1 : s5)[kk & (tg.W - 1)] |= 1u << (kk >> tg.logW);
        }
      }
    }
  }
  __syncthreads();
  if (edge) {
    for (uint32_t w = threadIdx.x; w < tg.W; w += BLOCK) {
      s1[w] &= below_mask(v.kh1, w, tg.logW, tg.W) & ~below_mask(v.kl1, w, tg.logW, tg.W);
      s5[w] &= below_mask(v.kh5, w, tg.logW, tg.W) & ~below_mask(v.kl5, w, tg.logW, tg.W);
    }
  }
  __syncthreads();
}

// Sum over the set bits b of x of b.
__device__ __forceinline__ uint32_t bit_index_sum(uint32_t x) {
  return __popc(x & 0xAAAAAAAAu) + (__popc(x & 0xCCCCCCCCu) << 1) + (__popc(x & 0xF0F0F0F0u) << 2) +
         (__popc(x & 0xFF00FF00u) << 3) + (__popc(x & 0xFFFF0000u) << 4);
}

// Carry-save bit-plane counters (Harley-Seal): after words x_1 .. x_n (n <
// 256) are added, bit b of plane k is bit k of the number of words with bit
// b set, so index_sum() = sum over all set bits of their positions b = the
// sum of bit_index_sum(x_i).  Eight words cost seven full adders (two
// three-input logic operations each) and a ripple of the top carry, about
// three operations per word against fourteen for bit_index_sum.
struct BitPlanes {
  uint32_t p[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  // a + b + c = 2 h + l, bitwise
  __device__ __forceinline__ static void csa(uint32_t &h, uint32_t &l, uint32_t a, uint32_t b, uint32_t c) {
    const uint32_t u = a ^ b;
    h = (a & b) | (u & c);
    l = u ^ c;
  }
  __device__ __forceinline__ void carry_from(int k, uint32_t x) {
#pragma unroll
    for (int j = 0; j < 8; j++) {
      if (j >= k) {
        const uint32_t c = p[j] & x;
        p[j] ^= x;
        x = c;
      }
    }
  }
  __device__ __forceinline__ void add1(uint32_t x) { carry_from(0, x); }
  __device__ __forceinline__ void add8(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t w3, uint32_t w4,
                                       uint32_t w5, uint32_t w6, uint32_t w7) {
    uint32_t ta, tb, tc, td, fa, fb, e;
    csa(ta, p[0], p[0], w0, w1);
    csa(tb, p[0], p[0], w2, w3);
    csa(tc, p[0], p[0], w4, w5);
    csa(td, p[0], p[0], w6, w7);
    csa(fa, p[1], p[1], ta, tb);
    csa(fb, p[1], p[1], tc, td);
    csa(e, p[2], p[2], fa, fb);
    carry_from(3, e);
  }
  __device__ __forceinline__ uint32_t index_sum() const {
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++)
      if (p[k]) s += bit_index_sum(p[k]) << k;  // the top planes are mostly empty
    return s;
  }
};

// As block_sum3, for values that lane 0 of each warp already holds summed
// over its warp: only the sum over the warps remains (result in thread 0).
template <int BLOCK>
__device__ __forceinline__ void block_sum3_warps(uint64_t &a, uint64_t &b, uint64_t &c, uint64_t *red) {
  constexpr int NWARPS = BLOCK / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[warp] = a;
    red[NWARPS + warp] = b;
    red[2 * NWARPS + warp] = c;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < NWARPS ? red[lane] : 0;
    b = lane < NWARPS ? red[NWARPS + lane] : 0;
    c = lane < NWARPS ? red[2 * NWARPS + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(kFullMask, a, o);
      b += __shfl_down_sync(kFullMask, b, o);
      c += __shfl_down_sync(kFullMask, c, o);
    }
  }
}

template <int BLOCK>
__device__ __forceinline__ void block_sum3(uint64_t &a, uint64_t &b, uint64_t &c, uint64_t *red) {
  constexpr int NWARPS = BLOCK / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(kFullMask, a, o);
    b += __shfl_down_sync(kFullMask, b, o);
    c += __shfl_down_sync(kFullMask, c, o);
  }
  if (lane == 0) {
    red[warp] = a;
    red[NWARPS + warp] = b;
    red[2 * NWARPS + warp] = c;
  }
  __syncthreads();
  if (warp == 0) {
    a = lane < NWARPS ? red[lane] : 0;
    b = lane < NWARPS ? red[NWARPS + lane] : 0;
    c = lane < NWARPS ? red[2 * NWARPS + lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(kFullMask, a, o);
      b += __shfl_down_sync(kFullMask, b, o);
      c += __shfl_down_sync(kFullMask, c, o);
    }
  }
}

// 32 x 32 bit transpose across a warp: on return, bit j of lane i's word is
// bit i of lane j's input word.  Five exchange stages; at stage s a lane
// keeps the half of each 2s-bit block that stays on its side and takes the
// other half from lane ^ s.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, uint32_t lane) {
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) {
    const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu : s == 2 ? 0x33333333u
                                                                                                   : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(kFullMask, x, s);
    x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

// Staging for compact_tile's emission: per warp and row, up to ROW (>= 64:
// one chunk's row holds at most 64 candidates) 16-bit codes ((chunk - c0) << 6
// | j << 1 | class, in value order); rows are ROW + 2 codes apart so that the
// 32 lanes' rows start in different banks.  A deeper staging row flushes less
// often but holds fewer CTAs per SM.
__host__ __device__ constexpr size_t compact_stage_bytes(int block, uint32_t row) {
  return (size_t)(block / 32) * 32 * (row + 2) * sizeof(uint16_t);
}

// Bit i of x to bit 2 i.
__device__ __forceinline__ uint64_t spread_bits(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

// Write the survivors of one tile, in value order, to out[off, ...).  The
// tile's bitmap bm holds W = 2^logW (class-1 word, class-5 word) pairs in the
// sliced layout: index k = b W + w is bit b of word w, so row b (bit b of
// every word) is the index run [b W, b W + W), and value order is row-major.
// With SBUF the bitmap is first staged in shared memory (sbuf, W pairs; bm
// 16-byte aligned), else it is read from global memory in both passes.
// Warp g takes the word chunks [g C / NWARPS, (g+1) C / NWARPS) of every row
// (C = W / 32).  For a chunk, each lane loads one word pair and the warp
// transposes the two 32 x 32 bit blocks, after which lane b holds row b's 32
// candidates of each class for that chunk.  Pass 1: each lane counts its
// row's survivors over the warp's chunks (warp_cnt[g][b], NWARPS x 32
// entries), and the offsets follow from a row-major prefix sum.  Pass 2
// (below) writes the values.  Bits outside the valid range must already be
// clear.
template <int BLOCK, typename OutT, bool SBUF, uint32_t ROW>
__device__ __forceinline__ void compact_tile(const uint2 *__restrict__ bm, uint32_t logW, uint64_t K0, uint64_t off,
                                             OutT *out, uint32_t *warp_cnt, uint2 *sbuf, uint16_t *stage) {
  constexpr int NWARPS = BLOCK / 32;
  constexpr uint32_t kPitch = ROW + 2;
  static_assert(ROW >= 64, "a staging row must hold one chunk's row");
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t W = 1u << logW, C = W / 32;
  if (SBUF) {
    const uint4 *src = (const uint4 *)bm;
    uint4 *dst = (uint4 *)sbuf;
    for (uint32_t i = threadIdx.x; i < W / 2; i += BLOCK) dst[i] = __ldg(src + i);
    __syncthreads();
  }
  auto pair = [&](uint32_t c) -> uint2 { return SBUF ? sbuf[(c << 5) + lane] : __ldg(bm + (c << 5) + lane); };
  const uint32_t c_begin = (uint32_t)((uint64_t)warp * C / NWARPS);
  const uint32_t c_end = (uint32_t)((uint64_t)(warp + 1) * C / NWARPS);
  uint32_t cnt = 0;
  for (uint32_t c = c_begin; c < c_end; c++) {
    const uint2 x = pair(c);
    cnt += __popc(warp_transpose32(x.x, lane)) + __popc(warp_transpose32(x.y, lane));
  }
  warp_cnt[warp * 32 + lane] = cnt;
  __syncthreads();
  if (warp == 0) {  // row-major prefix: rows in order, within a row the warps in order
    uint32_t row = 0;
    for (int g = 0; g < NWARPS; g++) row += warp_cnt[g * 32 + lane];
    uint32_t incl = row;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    uint32_t run = incl - row;
    for (int g = 0; g < NWARPS; g++) {
      const uint32_t cg = warp_cnt[g * 32 + lane];
      warp_cnt[g * 32 + lane] = run;
      run += cg;
    }
  }
  __syncthreads();
  // Pass 2.  The warp's outputs of row b form one run, starting at pos (lane
  // b's register).  Lane b extracts its row's survivors of each chunk, in
  // value order, as codes into its staging row; before a chunk would overflow
  // a row, the warp flushes: row by row, consecutive lanes write consecutive
  // outputs, so the stores coalesce and use all lanes.
  uint32_t pos = warp_cnt[warp * 32 + lane];
  uint16_t *const wst = stage + (size_t)warp * 32 * kPitch;
  uint16_t *const row = wst + lane * kPitch;
  const uint64_t v0 = 6 * K0;
  uint32_t n = 0, c0 = c_begin;
  auto flush = [&]() {
    __syncwarp();
    for (uint32_t r = 0; r < 32; r++) {
      const uint32_t nr = __shfl_sync(kFullMask, n, r), pr = __shfl_sync(kFullMask, pos, r);
      const uint16_t *rs = wst + r * kPitch;
      const uint64_t vr = v0 + 6ull * (((uint64_t)r << logW) + ((uint64_t)c0 << 5));
      for (uint32_t i = lane; i < nr; i += 32) {
        const uint32_t code = rs[i];
        out[off + pr + i] = (OutT)(vr + 6ull * (code >> 1) + 1 + 4 * (code & 1));
      }
    }
    __syncwarp();
    pos += n;
    n = 0;
  };
  for (uint32_t c = c_begin; c < c_end; c++) {
    const uint2 x = pair(c);
    const uint32_t t1 = warp_transpose32(x.x, lane), t5 = warp_transpose32(x.y, lane);
    const uint32_t rn = __popc(t1) + __popc(t5);
    if (__any_sync(kFullMask, n + rn > ROW) || c - c0 >= 1024) {  // codes hold c - c0 < 1024
      flush();
      c0 = c;
    }
    uint64_t m = spread_bits(t1) | (spread_bits(t5) << 1);
    const uint32_t cb = (c - c0) << 6;
    while (m) {
      row[n++] = (uint16_t)(cb + (uint32_t)(__ffsll((long long)m) - 1));
      m &= m - 1;
    }
  }
  flush();
}

// Staging bytes of compact_tile_smem for BLOCK threads: per warp 32 rows of
// kFusedRow one-byte codes, rows kFusedPitch bytes apart (17 words: the 32
// lanes' rows start in 32 different banks).
constexpr uint32_t kFusedRow = 64;
constexpr uint32_t kFusedPitch = 68;
__host__ __device__ constexpr size_t fused_stage_bytes(int block) {
  return (size_t)(block / 32) * 32 * kFusedPitch;
}

// compact_tile for a tile whose bitmaps are still in shared memory (s1, s5:
// W words each, sliced layout): writes its survivors, in value order, to
// out[off, ...), skipping every position >= cap.  Same two passes as
// compact_tile (warp transposes give lane b row b's candidates of a 32-word
// chunk; pass 1 counts per warp and row, a row-major prefix gives the
// positions), but the staging codes are one byte, (chunk - c0) << 6 | j << 1
// | class, so a warp flushes after at most four chunks or when a row would
// overflow kFusedRow codes.  Bits outside the range must already be clear.
template <int BLOCK, typename OutT>
__device__ __forceinline__ void compact_tile_smem(const uint32_t *s1, const uint32_t *s5, uint32_t logW, uint64_t K0,
                                                  uint64_t off, OutT *out, uint64_t cap, uint32_t *warp_cnt,
                                                  uint8_t *stage) {
  constexpr int NWARPS = BLOCK / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t W = 1u << logW, C = W / 32;
  const uint32_t c_begin = (uint32_t)((uint64_t)warp * C / NWARPS);
  const uint32_t c_end = (uint32_t)((uint64_t)(warp + 1) * C / NWARPS);
  uint32_t cnt = 0;
  for (uint32_t c = c_begin; c < c_end; c++)
    cnt += __popc(warp_transpose32(s1[(c << 5) + lane], lane)) + __popc(warp_transpose32(s5[(c << 5) + lane], lane));
  warp_cnt[warp * 32 + lane] = cnt;
  __syncthreads();
  if (warp == 0) {  // row-major prefix: rows in order, within a row the warps in order
    uint32_t row = 0;
    for (int g = 0; g < NWARPS; g++) row += warp_cnt[g * 32 + lane];
    uint32_t incl = row;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    uint32_t run = incl - row;
    for (int g = 0; g < NWARPS; g++) {
      const uint32_t cg = warp_cnt[g * 32 + lane];
      warp_cnt[g * 32 + lane] = run;
      run += cg;
    }
  }
  __syncthreads();
  uint32_t pos = warp_cnt[warp * 32 + lane];
  uint8_t *const wst = stage + (size_t)warp * 32 * kFusedPitch;
  uint8_t *const row = wst + lane * kFusedPitch;
  const uint64_t v0 = 6 * K0;
  uint32_t n = 0, c0 = c_begin;
  auto flush = [&]() {
    __syncwarp();
    for (uint32_t r = 0; r < 32; r++) {
      const uint32_t nr = __shfl_sync(kFullMask, n, r), pr = __shfl_sync(kFullMask, pos, r);
      const uint8_t *rs = wst + r * kFusedPitch;
      const uint64_t vr = v0 + 6ull * (((uint64_t)r << logW) + ((uint64_t)c0 << 5));
      for (uint32_t i = lane; i < nr; i += 32) {
        const uint32_t code = rs[i];
        const uint64_t o = off + pr + i;
        if (o < cap) out[o] = (OutT)(vr + 6ull * (code >> 1) + 1 + 4 * (code & 1));
      }
    }
    __syncwarp();
    pos += n;
    n = 0;
  };
  for (uint32_t c = c_begin; c < c_end; c++) {
    const uint32_t t1 = warp_transpose32(s1[(c << 5) + lane], lane), t5 = warp_transpose32(s5[(c << 5) + lane], lane);
    const uint32_t rn = __popc(t1) + __popc(t5);
    if (__any_sync(kFullMask, n + rn > kFusedRow) || c - c0 >= 4) {  // codes hold c - c0 < 4
      flush();
      c0 = c;
    }
    uint64_t m = spread_bits(t1) | (spread_bits(t5) << 1);
    const uint32_t cb = (c - c0) << 6;
    while (m) {
      row[n++] = (uint8_t)(cb + (uint32_t)(__ffsll((long long)m) - 1));
      m &= m - 1;
    }
  }
  flush();
}

}  // namespace sieve
