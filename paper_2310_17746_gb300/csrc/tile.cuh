// tile.cuh -- device routines for one segment ("tile") of the residue bitmaps.
//
// A CTA owns one tile at a time; its two bitmaps (class 1 and class 5, one bit
// per candidate, bit j of word w = index 32 w + j) live in shared memory
// (Sections 2.1-2.3: each worker sieves its own contiguous chunk in private
// memory, so no two workers write the same address).
#pragma once

#include "sieve_internal.cuh"

namespace sieve {

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

// Wheel presieve copy: word w of the tile receives the pattern bits
// [o0 + 32 w, o0 + 32 w + 32) with o0 = K0 mod period.  A warp copies 32
// consecutive words per step: one coalesced load per lane, the neighbour's
// word by shuffle, a funnel shift for the bit phase.  Needs len <= period.
template <int NWARPS>
__device__ __forceinline__ void presieve_copy(uint32_t *s1, uint32_t *s5, uint32_t nwords,
                                              uint64_t K0, const uint32_t *__restrict__ pat) {
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t o0 = (uint32_t)(K0 % kWheelPeriod);
  for (uint32_t c = warp; c * 32 < nwords; c += NWARPS) {
    uint32_t o = o0 + c * 1024u;
    if (o >= kWheelPeriod) o -= kWheelPeriod;
    const uint32_t wi = o >> 5, sh = o & 31;
    const uint32_t w = c * 32 + lane;
    uint32_t a1 = __ldg(pat + wi + lane);
    uint32_t a5 = __ldg(pat + kPatternWords + wi + lane);
    uint32_t b1 = __shfl_down_sync(kFullMask, a1, 1);
    uint32_t b5 = __shfl_down_sync(kFullMask, a5, 1);
    if (lane == 31) {
      b1 = __ldg(pat + wi + 32);
      b5 = __ldg(pat + kPatternWords + wi + 32);
    }
    if (w < nwords) {
      s1[w] = __funnelshift_r(a1, b1, sh);
      s5[w] = __funnelshift_r(a5, b5, sh);
    }
  }
}

// Strike indices k = id, id + step, ... < len in bitmap s (Section 3: the
// index advances by P, the value by 6P).  Clearing is an atomic AND in shared
// memory because several lanes may clear bits of one word.
__device__ __forceinline__ void strike(uint32_t *s, uint32_t k, uint32_t step, uint32_t len) {
#pragma unroll 4
  for (; k < len; k += step) atomicAnd(s + (k >> 5), rotl32(0xFFFFFFFEu, k));
}

// Strike every base prime with index in [i_first, np) into the tile whose
// index 0 is value B and which holds len indices per class.  Primes with index
// below i_split are struck by a whole warp (lane l takes hits l, l + 32, ...
// of the prime); the rest by one lane each.
template <int BLOCK>
__device__ __forceinline__ void strike_primes(uint32_t *s1, uint32_t *s5, uint64_t B, uint32_t len,
                                              const uint32_t *__restrict__ primes,
                                              const uint64_t *__restrict__ magic, uint32_t i_first,
                                              uint32_t i_split, uint32_t np) {
  constexpr int NWARPS = BLOCK / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t split = i_split < np ? i_split : np;
  for (uint32_t i = i_first + warp; i < split; i += NWARPS) {
    const uint32_t P = __ldg(primes + i);
    const StartIndex st = table1_start(B, B, P, __ldg(magic + i));
    const uint64_t k1 = (uint64_t)st.id1 + (uint64_t)lane * P;
    const uint64_t k5 = (uint64_t)st.id5 + (uint64_t)lane * P;
    if (k1 < len) strike(s1, (uint32_t)k1, 32u * P, len);
    if (k5 < len) strike(s5, (uint32_t)k5, 32u * P, len);
  }
  const uint32_t start = split > i_first ? split : i_first;
  for (uint32_t i = start + threadIdx.x; i < np; i += BLOCK) {
    const uint32_t P = __ldg(primes + i);
    const StartIndex st = table1_start(B, B, P, __ldg(magic + i));
    if ((uint64_t)st.id1 < len) strike(s1, (uint32_t)st.id1, P, len);
    if ((uint64_t)st.id5 < len) strike(s5, (uint32_t)st.id5, P, len);
  }
}

// ceil(a / 6) for signed a.
__device__ __forceinline__ int64_t ceil_div6(int64_t a) { return -floor_div6(-a); }

// Bits [lo_bit, hi_bit) of a word, bounds clamped to [0, 32].
__device__ __forceinline__ uint32_t bit_range_mask(int64_t lo_bit, int64_t hi_bit) {
  lo_bit = lo_bit < 0 ? 0 : (lo_bit > 32 ? 32 : lo_bit);
  hi_bit = hi_bit < 0 ? 0 : (hi_bit > 32 ? 32 : hi_bit);
  if (hi_bit <= lo_bit) return 0u;
  uint32_t upto_hi = hi_bit == 32 ? 0xFFFFFFFFu : ((1u << hi_bit) - 1u);
  uint32_t below_lo = lo_bit == 32 ? 0xFFFFFFFFu : ((1u << lo_bit) - 1u);
  return upto_hi & ~below_lo;
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
//   * tiles holding values below 24: clear the value 1, restore the wheel
//     primes 5..19 (the presieve pattern removed them with their multiples);
//   * edge tiles: clear the bits outside [lo, hi) and past len.
template <int BLOCK>
__device__ __forceinline__ void fixup_tile(uint32_t *s1, uint32_t *s5, uint32_t len, uint32_t nwords,
                                           uint64_t K0, const ValidRange &v) {
  if (K0 < 4 && threadIdx.x == 0) {  // the tile holds values below 24
    if (K0 == 0) s1[0] &= ~1u;       // 1 is not a prime
    const uint32_t wheel[6] = {5, 7, 11, 13, 17, 19};
    for (int q = 0; q < 6; q++) {
      const uint32_t wv = wheel[q], r = wv % 6, k = wv / 6;
      if (k >= K0 && k - K0 < len) (r == 1 ? s1 : s5)[(k - K0) >> 5] |= 1u << ((k - K0) & 31);
    }
  }
  __syncthreads();
  const int64_t full = 32 * (int64_t)nwords;
  if (v.kl1 > 0 || v.kl5 > 0 || v.kh1 < full || v.kh5 < full) {
    for (uint32_t w = threadIdx.x; w < nwords; w += BLOCK) {
      const int64_t base = 32 * (int64_t)w;
      s1[w] &= bit_range_mask(v.kl1 - base, v.kh1 - base);
      s5[w] &= bit_range_mask(v.kl5 - base, v.kh5 - base);
    }
  }
}

// Sum over the set bits j of x of j (x's bits are indices 32 w + j).
__device__ __forceinline__ uint32_t bit_index_sum(uint32_t x) {
  return __popc(x & 0xAAAAAAAAu) + (__popc(x & 0xCCCCCCCCu) << 1) + (__popc(x & 0xF0F0F0F0u) << 2) +
         (__popc(x & 0xFF00FF00u) << 3) + (__popc(x & 0xFFFF0000u) << 4);
}

// Interleave: bit 2j of the result is bit j of a, bit 2j+1 is bit j of b.
// With a = class 1 and b = class 5 of one word, bit order = value order
// (6k+1 < 6k+5 < 6(k+1)+1).
__device__ __forceinline__ uint64_t spread_bits(uint32_t x) {
  uint64_t v = x;
  v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
  v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
  v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
  v = (v | (v << 2)) & 0x3333333333333333ull;
  v = (v | (v << 1)) & 0x5555555555555555ull;
  return v;
}

__device__ __forceinline__ uint64_t interleave_classes(uint32_t a, uint32_t b) {
  return spread_bits(a) | (spread_bits(b) << 1);
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

}  // namespace sieve
