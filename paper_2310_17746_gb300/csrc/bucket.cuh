// bucket.cuh -- the bucket sieve for base primes much larger than a tile.
//
// A prime P above the tile length L hits each residue class of a tile at most
// once, and a prime near the top of a far range (P ~ 1e7 against L ~ 5e5)
// hits a given tile's class only about L / P ~ 5 % of the time.  Locating
// every such prime in every tile (Table 1, or the inverse-of-6 form of its
// start) is then mostly wasted work.  Section 2.4's incremental sieve acts
// with a prime only where it hits; the bucket sieve does that on the GPU:
//
//   * The tiles of a range are taken in waves of `ntl` consecutive tiles.
//   * Scatter (bucket_scatter_kernel): each large prime is located once per
//     wave (its first class-1 and class-5 index at or after max(wave start,
//     P^2)) and walked through the wave by steps of P (Section 3: +P in index
//     is +6P in value).  Every hit is an entry (offset in its tile, class)
//     for the bucket of the tile it falls in.  A CTA counting-sorts the hits
//     of a round in shared memory by target tile, so that each bucket is
//     written in contiguous runs (coalesced), into its own sub-bucket per
//     target tile: no global atomics.
//   * Drain (bucket_drain, inside the tile kernel): a tile reads its buckets
//     (one per scatter CTA) and clears the entries' bits in shared memory.
//
// Sub-buckets have a fixed capacity computed on the host from the expected
// number of hits.  An entry that does not fit sets the target tile's overflow
// flag, and that tile then also locates every large prime itself (the plain
// per-tile method): a strike applied twice is harmless, so the result never
// depends on the capacity.
#pragma once

#include "tile.cuh"

namespace sieve {

// Entry layout: bit 0 = class (0: 6k+1, 1: 6k+5), bits 1..19 = index in the
// tile (< L <= 2^19); in the scatter's shared-memory sort, bits 20..31 hold
// the target tile of the wave (< 4096).
constexpr uint32_t kBucketKeyShift = 20;
constexpr uint32_t kBucketMaxWaveTiles = 1u << (32 - kBucketKeyShift);

struct BucketParams {
  uint32_t *entries;    // [ntl][ncta][cap]
  uint32_t *counts;     // [ntl][ncta]: entries the scatter CTA wrote for the tile
  uint32_t *overflow;   // [ntl]: nonzero when a sub-bucket of the tile overflowed
  uint32_t cap;         // entries per (target tile, scatter CTA)
  uint32_t ncta;        // scatter CTAs
  uint32_t i_large;     // table indices [i_large, i_end) go through the buckets
  uint32_t i_end;
  uint32_t t_begin;     // first tile of the wave (tile index within the range)
  uint32_t ntl;         // tiles in the wave
  uint32_t wave_id;     // index of the wave in the call
  // range geometry and base table (as the tile kernel sees them)
  uint64_t k_begin, k_end;
  uint32_t L, logW;
  const uint32_t *primes;
  const uint64_t *magic;
  const uint2 *cinv;
};

// Dynamic shared memory of bucket_scatter_kernel<SB, H> for a wave of ntl tiles.
__host__ __device__ constexpr size_t bucket_scatter_smem(int sb, int h, uint32_t ntl) {
  return (size_t)4 * ntl * sizeof(uint32_t) + (size_t)sb * h * (2 * sizeof(uint32_t) + sizeof(uint16_t));
}

// Exclusive prefix of a[0..n) into out[0..n) by the whole block; returns the
// total in every thread.  Each thread sums a contiguous run of entries, the
// runs' sums are scanned across warps, then each thread writes its run.
template <int SB>
__device__ __forceinline__ uint32_t block_exclusive_scan(const uint32_t *a, uint32_t *out, uint32_t n,
                                                         uint32_t *warp_tot) {
  constexpr int NW = SB / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t per = (n + SB - 1) / SB;
  const uint32_t i0 = threadIdx.x * per;
  uint32_t s = 0;
  for (uint32_t i = i0; i < i0 + per && i < n; i++) s += a[i];
  uint32_t incl = s;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(kFullMask, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    uint32_t t = lane < (uint32_t)NW ? warp_tot[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(kFullMask, t, o);
      if (lane >= (uint32_t)o) t += y;
    }
    if (lane < (uint32_t)NW) warp_tot[lane] = t;  // inclusive over warps
  }
  __syncthreads();
  uint32_t run = (warp ? warp_tot[warp - 1] : 0) + incl - s;
  for (uint32_t i = i0; i < i0 + per && i < n; i++) {
    out[i] = run;
    run += a[i];
  }
  const uint32_t total = warp_tot[NW - 1];
  __syncthreads();
  return total;
}

// Scatter of one wave.  CTA c owns the large primes with table index
// i_large + c + ncta * m, m = 0, 1, ...; its threads take the next m from a
// shared counter whenever their prime is used up, so that the threads stay
// busy until the CTA's primes are done (a prime near the threshold hits a wave
// ten times as often as one near the top).  Each thread walks its prime's hits
// in the wave, up to H hits per round.  A round: the hits go to shared memory
// with their rank among the round's hits for the same target tile (a
// shared-memory histogram), the histogram is scanned, the hits are placed in
// target order, and the block writes them out in that order, each target's
// run contiguous in its sub-bucket.  Requires ntl * L < 2^31 and every prime
// < 2^31 (the host checks), so that wave indices and index + P fit in 32 bits.
template <int SB, int H>
__global__ void __launch_bounds__(SB) bucket_scatter_kernel(const BucketParams b) {
  static_assert(SB * H <= 65536, "ranks are 16-bit");
  extern __shared__ uint32_t bsm[];
  __shared__ uint32_t warp_tot[SB / 32];
  __shared__ uint32_t next_m;
  const uint32_t ntl = b.ntl;
  uint32_t *hist = bsm;            // hits of this round per target tile
  uint32_t *offs = hist + ntl;     // exclusive prefix of hist
  uint32_t *gbase = offs + ntl;    // where this round's run starts in each sub-bucket
  uint32_t *sub = gbase + ntl;     // entries this CTA produced so far per target tile
  uint32_t *raw = sub + ntl;       // [SB * H] this round's hits, in thread order
  uint32_t *sorted = raw + SB * H; // [SB * H] the same, in target order
  uint16_t *rank = (uint16_t *)(sorted + SB * H);
  if (threadIdx.x == 0) next_m = 0;
  for (uint32_t i = threadIdx.x; i < ntl; i += SB) {
    hist[i] = 0;
    sub[i] = 0;
  }
  const uint64_t Kw = b.k_begin + (uint64_t)b.t_begin * b.L;
  const uint64_t wl64 = b.k_end - Kw < (uint64_t)ntl * b.L ? b.k_end - Kw : (uint64_t)ntl * b.L;
  const uint32_t wlen = (uint32_t)wl64;
  const uint32_t logL = b.logW + 5, lmask = b.L - 1;
  uint32_t P = 0, k1 = wlen, k5 = wlen;
  bool more = true;
  __syncthreads();
  for (;;) {
    uint32_t n = 0;
    while (n < (uint32_t)H) {
      if (k1 >= wlen && k5 >= wlen) {  // next prime of this CTA that hits the wave
        while (more) {
          const uint64_t i = (uint64_t)b.i_large + blockIdx.x + (uint64_t)b.ncta * atomicAdd(&next_m, 1u);
          if (i >= b.i_end) {
            more = false;
            break;
          }
          P = __ldg(b.primes + i);
          const uint64_t Kc = ((uint64_t)P * P - 1) / 6;  // P^2 = 6 Kc + 1: no hit below P^2
          const uint64_t K0 = Kw > Kc ? Kw : Kc;
          if (K0 >= Kw + wl64) continue;
          uint32_t a1, a5;
          starts_from_inverse(K0, P, __ldg(b.magic + i), __ldg(b.cinv + i), a1, a5);
          const uint32_t base = (uint32_t)(K0 - Kw);
          k1 = base + a1;
          k5 = base + a5;
          if (k1 < wlen || k5 < wlen) break;
        }
        if (k1 >= wlen && k5 >= wlen) break;  // no prime left
      }
      uint32_t k, cls;
      if (k1 <= k5) {
        k = k1;
        cls = 0;
        k1 += P;
      } else {
        k = k5;
        cls = 1;
        k5 += P;
      }
      const uint32_t key = k >> logL;
      const uint32_t slot = n * SB + threadIdx.x;  // n-major: a warp's lanes on consecutive words
      raw[slot] = (key << kBucketKeyShift) | ((k & lmask) << 1) | cls;
      rank[slot] = (uint16_t)atomicAdd(hist + key, 1u);
      n++;
    }
    if (!__syncthreads_or(n > 0)) break;
    const uint32_t total = block_exclusive_scan<SB>(hist, offs, ntl, warp_tot);
    for (uint32_t i = threadIdx.x; i < ntl; i += SB) {
      gbase[i] = sub[i];
      sub[i] += hist[i];
      hist[i] = 0;
    }
    for (uint32_t q = 0; q < n; q++) {
      const uint32_t slot = q * SB + threadIdx.x;
      const uint32_t e = raw[slot];
      sorted[offs[e >> kBucketKeyShift] + rank[slot]] = e;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < total; i += SB) {
      const uint32_t e = sorted[i];
      const uint32_t key = e >> kBucketKeyShift;
      const uint32_t dst = gbase[key] + (i - offs[key]);
      if (dst < b.cap)
        b.entries[((size_t)key * b.ncta + blockIdx.x) * b.cap + dst] = e & ((1u << kBucketKeyShift) - 1);
      else
        b.overflow[key] = 1;
    }
    __syncthreads();
  }
  for (uint32_t i = threadIdx.x; i < ntl; i += SB)
    b.counts[(size_t)i * b.ncta + blockIdx.x] = sub[i] < b.cap ? sub[i] : b.cap;
}

// The same scatter without the shared-memory sort: each hit takes its slot in
// the CTA's sub-bucket of its target tile from a shared-memory counter and is
// stored at once.  No rounds and no barriers, at the price of stores that a
// warp spreads over many sub-buckets (L2 merges them into sectors).
template <int SB>
__global__ void __launch_bounds__(SB) bucket_scatter_direct_kernel(const BucketParams b) {
  extern __shared__ uint32_t bsm[];
  __shared__ uint32_t next_m;
  const uint32_t ntl = b.ntl;
  uint32_t *sub = bsm;  // entries this CTA produced per target tile
  if (threadIdx.x == 0) next_m = 0;
  for (uint32_t i = threadIdx.x; i < ntl; i += SB) sub[i] = 0;
  const uint64_t Kw = b.k_begin + (uint64_t)b.t_begin * b.L;
  const uint64_t wl64 = b.k_end - Kw < (uint64_t)ntl * b.L ? b.k_end - Kw : (uint64_t)ntl * b.L;
  const uint32_t wlen = (uint32_t)wl64;
  const uint32_t logL = b.logW + 5, lmask = b.L - 1;
  uint32_t *const ent = b.entries + (size_t)blockIdx.x * b.cap;
  const size_t key_stride = (size_t)b.ncta * b.cap;
  __syncthreads();
  auto emit = [&](uint32_t k, uint32_t cls) {
    const uint32_t key = k >> logL;
    const uint32_t pos = atomicAdd(sub + key, 1u);
    if (pos < b.cap)
      ent[key * key_stride + pos] = ((k & lmask) << 1) | cls;
    else
      b.overflow[key] = 1;
  };
  // one prime at a time per thread; the next prime's index and table entries
  // are fetched before the current prime is walked, so that their latency
  // (the table streams from L2 or DRAM) overlaps its hits
  auto take = [&]() -> uint64_t {
    return (uint64_t)b.i_large + blockIdx.x + (uint64_t)b.ncta * atomicAdd(&next_m, 1u);
  };
  uint64_t i = take();
  uint32_t P = 0;
  uint64_t m = 0;
  uint2 c = make_uint2(0, 0);
  if (i < b.i_end) {
    P = __ldg(b.primes + i);
    m = __ldg(b.magic + i);
    c = __ldg(b.cinv + i);
  }
  while (i < b.i_end) {
    const uint64_t in = take();
    uint32_t Pn = 0;
    uint64_t mn = 0;
    uint2 cn = make_uint2(0, 0);
    if (in < b.i_end) {
      Pn = __ldg(b.primes + in);
      mn = __ldg(b.magic + in);
      cn = __ldg(b.cinv + in);
    }
    const uint64_t Kc = ((uint64_t)P * P - 1) / 6;  // P^2 = 6 Kc + 1: no hit below P^2
    const uint64_t K0 = Kw > Kc ? Kw : Kc;
    if (K0 < Kw + wl64) {
      uint32_t a1, a5;
      starts_from_inverse(K0, P, m, c, a1, a5);
      const uint32_t base = (uint32_t)(K0 - Kw);
      // four hits per trip: their slot atomics are independent, so they are
      // in flight together instead of one at a time (64-bit index: k + 3P may
      // pass 2^32 before the test ends the loop)
      auto walk = [&](uint64_t k, uint32_t cls) {
        for (; k + 3ull * P < wlen; k += 4ull * P) {
          emit((uint32_t)k, cls);
          emit((uint32_t)(k + P), cls);
          emit((uint32_t)(k + 2ull * P), cls);
          emit((uint32_t)(k + 3ull * P), cls);
        }
        for (; k < wlen; k += P) emit((uint32_t)k, cls);
      };
      walk(base + a1, 0);
      walk(base + a5, 1);
    }
    P = Pn;
    m = mn;
    c = cn;
    i = in;
  }
  __syncthreads();
  for (uint32_t j = threadIdx.x; j < ntl; j += SB)
    b.counts[(size_t)j * b.ncta + blockIdx.x] = sub[j] < b.cap ? sub[j] : b.cap;
}

constexpr int kDrainUnroll = 8;

// Drain the buckets of wave tile `tl` into the tile's bitmaps: warp w takes
// the sub-buckets w, w + NWARPS, ...; its lanes read consecutive entries.
template <int BLOCK>
__device__ __forceinline__ void bucket_drain(uint32_t *s1, uint32_t *s5, const TileGeom &tg, const BucketParams &b,
                                             uint32_t tl) {
  constexpr int NWARPS = BLOCK / 32;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t wmask = tg.W - 1, logW = tg.logW, len = tg.len;
  const uint32_t *cnt = b.counts + (size_t)tl * b.ncta;
  const uint32_t *ent = b.entries + (size_t)tl * b.ncta * b.cap;
  // kDrainUnroll loads in flight per lane before the strikes (the entries
  // come from L2 or DRAM; one at a time the loop waits on each); a slot past
  // the sub-bucket's count reads as an index >= len and strikes nothing
  auto hit = [&](uint32_t v) {
    const uint32_t k = v >> 1;
    if (k < len) strike_one((v & 1) ? s5 : s1, k, wmask, logW);
  };
  for (uint32_t c = warp; c < b.ncta; c += NWARPS) {
    const uint32_t n = __ldg(cnt + c);
    const uint32_t *e = ent + (size_t)c * b.cap;
    for (uint32_t q = lane; q < n; q += 32 * kDrainUnroll) {  // read once: streaming loads
      uint32_t v[kDrainUnroll];
#pragma unroll
      for (int u = 0; u < kDrainUnroll; u++) v[u] = q + 32 * u < n ? __ldcs(e + q + 32 * u) : 0xFFFFFFFFu;
#pragma unroll
      for (int u = 0; u < kDrainUnroll; u++) hit(v[u]);
    }
  }
}

}  // namespace sieve
