// range.cu -- sieve of one range [lo, hi): count / checksum / per-segment
// counts, or the full increasing list.
//
// Kernel structure (Section 4, Figure 4, mapped to a GPU): the range is cut
// into tiles of L indices per residue class; CTAs take tiles in grid-stride
// order.  Per tile: presieve copy -> start indices (Table 1, or the equal
// inverse-of-6 form) and strikes for every base prime above the presieved
// ones up to isqrt(tile end) -> fix-ups -> popcount,
// checksum and per-segment counts (count mode) or bitmap write-out (list mode,
// followed by a scan of per-tile counts and a compaction kernel).
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include <cuda/atomic>

#include "bucket.cuh"
#include "cluster.cuh"
#include "tile.cuh"

namespace sieve {

struct RangeKernelParams {
  uint64_t lo, hi;          // [lo, hi)
  uint64_t k_begin;         // class index of tile 0's index 0
  uint64_t k_end;           // ceil((hi - 1) / 6): indices below it can hold a value < hi
  uint32_t L;               // indices per class per tile (32 W, W a power of two)
  uint32_t logW;            // log2(L / 32)
  uint32_t ntiles;
  const uint32_t *primes;
  const uint64_t *magic;
  const uint2 *cinv;
  uint32_t nprimes;         // primes[0..nprimes) cover isqrt(hi - 1)
  uint32_t i_first;         // first prime index struck (after the presieved ones)
  uint32_t i_split;         // primes with index < i_split are struck by a warp
  const uint32_t *sliced;   // presieve patterns in the sliced layout for this W
  PatternDesc pd[kNumPatterns];
  int npat;                 // patterns in use (wheel + groups)
  // count-mode outputs (atomically accumulated)
  unsigned long long *count;
  unsigned long long *checksum;
  uint64_t seg_width;       // 0: no per-segment counts
  uint64_t first_seg;       // floor(lo / seg_width)
  unsigned long long *bins;
  // list mode with bitmap write-out (kModeListBitmap)
  uint32_t *tile_counts;    // per tile
  uint2 *bitmap;            // per tile L/32 (class-1 word, class-5 word) pairs
  // single-pass list mode (kModeListFused)
  unsigned long long *tile_state;  // per tile: look-back word (flag << 62 | count), zeroed per call
  uint32_t *tile_counter;          // per launch (bucket wave): next tile to take, zeroed per call
  unsigned long long *error;       // set to 1 when a look-back gave up (the call reports TIMEOUT)
  void *out;                       // device output, uint32 or uint64 per out_bytes
  uint64_t cap;                    // elements of out; positions >= cap are not written
  uint32_t out_bytes;
  uint32_t stage_off;              // words from the start of dynamic shared memory to the staging
  // cluster segments (kLargeCluster)
  uint32_t cluster;                // CTAs per cluster: C consecutive tiles form one segment
  uint32_t i_cluster;              // primes with table index >= i_cluster: located once per segment
};

// What the tile kernel produces: counts only; counts plus each tile's bitmap
// in global memory (for scan_tile_counts_kernel and compact_kernel); or
// counts plus the list itself, each tile compacted straight from shared
// memory at an offset found by decoupled look-back (one pass).
constexpr int kModeCount = 0;
constexpr int kModeListBitmap = 1;
constexpr int kModeListFused = 2;

// How the tile kernel applies the primes far above the tile length: located
// in every tile; drained from the buckets of a wave (bucket.cuh); or located
// once per cluster segment and struck through distributed shared memory
// (cluster.cuh).
constexpr int kLargeTiles = 0;
constexpr int kLargeBuckets = 1;
constexpr int kLargeCluster = 2;

// Decoupled look-back (Merrill & Garland, "Single-pass Parallel Prefix Scan
// with Decoupled Look-back", 2016) over per-tile words flag << 62 | value:
// flag 1 = the tile's own count is known, 2 = its inclusive prefix is known,
// 3 = a look-back before it failed.  Tiles are taken from an atomic counter,
// so every tile before the current one is held by a running CTA that
// publishes without waiting on later tiles; each poll that finds no flag
// counts against kLookbackPolls (about a second of polling), after which the
// tile publishes flag 3, as do all tiles after it, and the call fails.
constexpr uint64_t kLookbackFlagShift = 62;
constexpr uint64_t kLookbackValueMask = (1ull << kLookbackFlagShift) - 1;
constexpr uint32_t kLookbackPolls = 1u << 23;

__device__ __forceinline__ void lookback_publish(unsigned long long *w, uint64_t flag, uint64_t value) {
  cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(*w);
  a.store((flag << kLookbackFlagShift) | (value & kLookbackValueMask), cuda::memory_order_release);
}

// Exclusive prefix of tile t's count, by warp 0 (every lane returns it); false
// if it failed.  Each step reads the 32 words before the window's end at once
// (lane l: tile j - l), and stops at the nearest one carrying an inclusive
// prefix: the prefix is that value plus the counts of the tiles after it.
// When one of the 32 still has no flag, the warp polls the same window again.
__device__ __forceinline__ bool lookback_prefix_warp(unsigned long long *state, uint32_t t, uint64_t cnt,
                                                     uint64_t *excl) {
  const uint32_t lane = threadIdx.x & 31;
  if (t == 0) {
    if (lane == 0) lookback_publish(state, 2, cnt);
    *excl = 0;
    return true;
  }
  if (lane == 0) lookback_publish(state + t, 1, cnt);
  uint64_t sum = 0;
  uint32_t polls = 0;
  bool ok = true;
  int64_t j = (int64_t)t - 1;  // the window is tiles j - 31 .. j
  while (j >= 0) {
    const int64_t mine = j - (int64_t)lane;
    uint64_t w = (2ull << kLookbackFlagShift);  // below tile 0: an inclusive prefix of 0
    if (mine >= 0) {
      cuda::atomic_ref<unsigned long long, cuda::thread_scope_device> a(state[mine]);
      w = a.load(cuda::memory_order_acquire);
    }
    const uint32_t f = (uint32_t)(w >> kLookbackFlagShift);
    const uint32_t has_p = __ballot_sync(kFullMask, f == 2), bad = __ballot_sync(kFullMask, f == 3);
    const uint32_t empty = __ballot_sync(kFullMask, f == 0);
    // lanes up to the nearest inclusive prefix (the lowest lane with f == 2)
    const uint32_t stop = has_p ? (uint32_t)(__ffs(has_p) - 1) : 31u;
    const uint32_t upto = stop == 31 ? 0xFFFFFFFFu : ((2u << stop) - 1u);
    if (bad & upto) {
      ok = false;
      break;
    }
    if (empty & upto) {  // a tile in the window has not published its count yet
      if (++polls > kLookbackPolls) {
        ok = false;
        break;
      }
      __nanosleep(100);
      continue;
    }
    uint64_t v = lane <= stop ? (w & kLookbackValueMask) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFullMask, v, o);
    sum += __shfl_sync(kFullMask, v, 0);
    if (has_p) break;
    j -= 32;
  }
  if (lane == 0) lookback_publish(state + t, ok ? 2 : 3, sum + cnt);
  *excl = sum;
  return ok;
}

// LARGE = kLargeBuckets: the launch sieves the tiles of one bucket wave,
// [b.t_begin, b.t_begin + b.ntl); the primes with table index >= b.i_large
// are applied by draining the wave's buckets (bucket.cuh) instead of being
// located in every tile.  LARGE = kLargeCluster: the launch is made of
// clusters of p.cluster CTAs; the CTAs of a cluster take consecutive tiles
// (one segment) in each step of the grid-stride loop, and the primes with
// table index >= p.i_cluster are located once per segment (cluster.cuh).  A
// member whose tile lies past the range's end still takes its share of the
// segment's primes and both cluster barriers.  Otherwise the launch sieves
// every tile and b is unused.
template <int BLOCK, int MODE, int LARGE>
__global__ void __launch_bounds__(BLOCK, 1536 / BLOCK) range_tiles_kernel(const RangeKernelParams p,
                                                                          const BucketParams b) {
  constexpr bool LIST = MODE == kModeListBitmap;
  constexpr bool FUSED = MODE == kModeListFused;
  constexpr bool BUCKET = LARGE == kLargeBuckets;
  constexpr bool CLUSTER = LARGE == kLargeCluster;
  static_assert(!(CLUSTER && FUSED), "cluster segments take tiles in grid-stride order, not from a counter");
  constexpr int NWARPS = BLOCK / 32;
  extern __shared__ uint32_t smem[];
  const uint32_t W = p.L / 32;
  uint32_t *s1 = smem;
  uint32_t *s5 = smem + W;
  uint2 *starts = (uint2 *)(smem + 2 * W);  // warp-band start indices
  __shared__ uint32_t sh_np, sh_next, sh_allsq;
  __shared__ uint32_t sh_poff[kNumPatterns];  // pattern offsets of the tile about to be sieved
  __shared__ uint64_t sh_bin0;
  __shared__ int64_t sh_t1, sh_t5;
  __shared__ int sh_has_boundary;
  __shared__ uint32_t sh_overflow;
  __shared__ uint32_t sh_tile;                // FUSED: the tile taken next
  __shared__ uint64_t sh_excl;                // FUSED: the tile's output offset
  __shared__ int sh_lb_ok;
  __shared__ uint32_t sh_np_seg;              // CLUSTER: primes the segment needs
  __shared__ uint64_t red[3 * NWARPS];
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t t_begin = BUCKET ? b.t_begin : 0u;
  const uint32_t t_end = BUCKET ? b.t_begin + b.ntl : p.ntiles;
  uint32_t *const counter = FUSED ? p.tile_counter + (BUCKET ? b.wave_id : 0u) : nullptr;
  uint32_t np_prev = 0;  // warp 0: the previous tile's prime count
  const uint32_t crank = CLUSTER ? cluster_rank() : 0u;
  // tiles in grid-stride order, or (FUSED) from the counter, in increasing
  // order over the CTAs, as the look-back needs
  uint32_t t = t_begin + blockIdx.x;
  if (FUSED) {
    if (threadIdx.x == 0) sh_tile = t_begin + atomicAdd(counter, 1u);
    __syncthreads();
    t = sh_tile;
  }
  // the pattern offsets K0 mod period: computed once per tile by a few
  // threads (for the next tile at the end of this one), not by every thread
  if (threadIdx.x < (uint32_t)p.npat && t < t_end)
    sh_poff[threadIdx.x] = pattern_offset(p.k_begin + (uint64_t)t * p.L, p.pd[threadIdx.x]);
  __syncthreads();

  // (a cluster's members share the loop: t - crank is its segment's first tile)
  while ((CLUSTER ? t - crank : t) < t_end) {
    const bool active = !CLUSTER || t < t_end;  // CTA-uniform
    const uint64_t K0 = p.k_begin + (uint64_t)t * p.L;
    const uint64_t left = p.k_end - K0;
    TileGeom tg;
    tg.W = W;
    tg.logW = p.logW;
    tg.len = left < p.L ? (uint32_t)left : p.L;
    const uint64_t B = 6 * K0;
    const uint64_t tile_end = B + 6ull * tg.len;
    const uint64_t vend = tile_end < p.hi ? tile_end : p.hi;

    if (warp == 0 && active) {
      // base primes needed: P <= isqrt(vend - 1).  A CTA's tiles go up, so
      // the count of the previous tile stays right unless the next prime
      // joins (then search again).
      const uint64_t s = vend >= 2 ? isqrt_dev(vend - 1) : 0;
      const bool grows = np_prev < p.nprimes && (uint64_t)__ldg(p.primes + np_prev) <= s;
      const bool shrinks = np_prev > 0 && (uint64_t)__ldg(p.primes + np_prev - 1) > s;
      if (grows || shrinks) np_prev = warp_count_le(p.primes, p.nprimes, s);
      const uint32_t np = np_prev;
      // every needed prime is below sqrt(B) (and 2^31): no P^2 clamp in this tile
      const uint64_t Plast = np ? __ldg(p.primes + np - 1) : 0;
      if (lane == 0) {
        sh_np = np;
        sh_allsq = Plast * Plast <= B && Plast < 0x80000000ull;
        sh_next = p.i_first;
        sh_has_boundary = 0;
        if (BUCKET) {  // read and re-arm the tile's overflow flag
          sh_overflow = b.overflow[t - t_begin];
          if (sh_overflow) b.overflow[t - t_begin] = 0;
        }
        if (p.seg_width) {
          const uint64_t v0 = B > p.lo ? B : p.lo;
          const uint64_t sg = v0 / p.seg_width;
          sh_bin0 = sg - p.first_seg;
          const uint64_t X = (sg + 1) * p.seg_width;
          if (X < vend) {
            sh_has_boundary = 1;
            int64_t t1 = ceil_div6((int64_t)(X - B) - 1), t5 = ceil_div6((int64_t)(X - B) - 5);
            sh_t1 = t1 < 0 ? 0 : (t1 > (int64_t)tg.len ? (int64_t)tg.len : t1);
            sh_t5 = t5 < 0 ? 0 : (t5 > (int64_t)tg.len ? (int64_t)tg.len : t5);
          }
        }
      }
    }
    // CLUSTER: the segment (the cluster's C tiles from t - crank) and the
    // primes it needs, by warp 1 of every member
    uint64_t Ks = 0;
    uint32_t slen = 0;
    if (CLUSTER) {
      Ks = p.k_begin + (uint64_t)(t - crank) * p.L;
      const uint64_t sleft = p.k_end - Ks, scap = (uint64_t)p.cluster * p.L;
      slen = (uint32_t)(sleft < scap ? sleft : scap);
      if (warp == 1) {
        const uint64_t send = 6 * (Ks + slen), svend = send < p.hi ? send : p.hi;
        const uint32_t nps = warp_count_le(p.primes, p.nprimes, svend >= 2 ? isqrt_dev(svend - 1) : 0);
        if (lane == 0) sh_np_seg = nps;
      }
    }
    if (active) {
      presieve_copy<BLOCK>(s1, s5, tg, K0, p.sliced, p.pd, p.npat, sh_poff);
      warp_band_starts<BLOCK>(starts, B, tg.len, p.primes, p.magic, p.cinv, p.i_first, p.i_split);
    }
    __syncthreads();
    if (CLUSTER) cluster_sync_all();  // every member's tile is presieved before any remote strike

    if (CLUSTER) {
      // primes below i_cluster in the tile itself, the rest once per segment
      if (active)
        strike_primes<BLOCK>(s1, s5, B, tg, p.primes, p.magic, p.cinv, starts, p.i_first, p.i_split, sh_np,
                             sh_allsq != 0, &sh_next, K0, p.i_cluster);
      cluster_strike<BLOCK>(s1, s5, p.logW, Ks, slen, crank, p.cluster, p.primes, p.magic, p.cinv, p.i_cluster,
                            sh_np_seg);
    } else if (BUCKET) {
      // primes below i_large as usual, the rest from the buckets; a tile whose
      // buckets overflowed also locates the large primes itself (a strike
      // applied twice is harmless)
      strike_primes<BLOCK>(s1, s5, B, tg, p.primes, p.magic, p.cinv, starts, p.i_first, p.i_split, sh_np,
                           sh_allsq != 0, &sh_next, K0, b.i_large);
      bucket_drain<BLOCK>(s1, s5, tg, b, t - t_begin);
      if (sh_overflow && sh_np > b.i_large)
        strike_lane_band<BLOCK>(s1, s5, B, tg, p.primes, p.magic, p.cinv, b.i_large, sh_np, sh_allsq != 0, K0);
    } else {
      strike_primes<BLOCK>(s1, s5, B, tg, p.primes, p.magic, p.cinv, starts, p.i_first, p.i_split, sh_np,
                           sh_allsq != 0, &sh_next, K0);
    }
    __syncthreads();
    if (CLUSTER) cluster_sync_all();  // every remote strike into this tile has landed
    if (active) {
      // a full tile above the presieved primes and inside [lo, hi) needs no
      // fix-up (valid_range would give [0, 32 W) in both classes)
      const bool interior = 6 * K0 > 131 && p.lo <= B + 1 && p.hi >= B + 6ull * 32 * W && tg.len == 32 * W;
      if (!interior)  // ends with a barrier when it changes the tile
        fixup_tile<BLOCK>(s1, s5, tg, K0, valid_range(p.lo, p.hi, B, tg.len), p.npat);

      // popcount, checksum, and the count below the segment boundary (if any).
      // Word w holds indices w + b W: their values sum to
      // popc * (6 (K0 + w) + r) + 6 w popc + 6 W * (sum of the set bit positions b),
      // so a thread accumulates, in 32 bits, the class counts c1 / c5, the
      // word-weighted count sw and the bit-position sum bs of its words
      // (sw < 2^15 * 64 * (W / BLOCK) < 2^32), and forms the 64-bit sum once.
      uint32_t c1 = 0, c5 = 0, sw = 0, below32 = 0;
      BitPlanes planes;  // the bit-position sum, four word pairs at a time
      const int has_b = sh_has_boundary;
      const int64_t t1 = has_b ? sh_t1 : 0, t5 = has_b ? sh_t5 : 0;
      auto pair = [&](uint32_t w, uint32_t a, uint32_t b) {
        if (LIST) p.bitmap[(uint64_t)t * W + w] = make_uint2(a, b);
        const uint32_t ca = __popc(a), cb = __popc(b);
        c1 += ca;
        c5 += cb;
        sw += w * (ca + cb);
        if (has_b)
          below32 += __popc(a & below_mask(t1, w, tg.logW, W)) + __popc(b & below_mask(t5, w, tg.logW, W));
      };
      uint32_t w = threadIdx.x;
      for (; w + 3 * BLOCK < W; w += 4 * BLOCK) {
        const uint32_t a0 = s1[w], b0 = s5[w], a1 = s1[w + BLOCK], b1 = s5[w + BLOCK];
        const uint32_t a2 = s1[w + 2 * BLOCK], b2 = s5[w + 2 * BLOCK], a3 = s1[w + 3 * BLOCK], b3 = s5[w + 3 * BLOCK];
        pair(w, a0, b0);
        pair(w + BLOCK, a1, b1);
        pair(w + 2 * BLOCK, a2, b2);
        pair(w + 3 * BLOCK, a3, b3);
        planes.add8(a0, b0, a1, b1, a2, b2, a3, b3);
      }
      for (; w < W; w += BLOCK) {
        const uint32_t a = s1[w], b = s5[w];
        pair(w, a, b);
        planes.add1(a);
        planes.add1(b);
      }
      const uint32_t bs = planes.index_sum();
      // the sums over the warp in 32 bits (a warp's c1, c5 < 2^17, sw < 2^31,
      // bs < 2^23: they fit), then the 64-bit count and checksum once per warp
      uint32_t wc1 = c1, wc5 = c5, wsw = sw, wbs = bs, wbl = below32;
  #pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        wc1 += __shfl_down_sync(kFullMask, wc1, o);
        wc5 += __shfl_down_sync(kFullMask, wc5, o);
        wsw += __shfl_down_sync(kFullMask, wsw, o);
        wbs += __shfl_down_sync(kFullMask, wbs, o);
        wbl += __shfl_down_sync(kFullMask, wbl, o);
      }
      uint64_t cnt = (uint64_t)wc1 + wc5, below = wbl;
      uint64_t sum = (uint64_t)wc1 * (6 * K0 + 1) + (uint64_t)wc5 * (6 * K0 + 5) + 6ull * wsw + 6ull * W * wbs;
      if (FUSED && threadIdx.x == 0) sh_tile = t_begin + atomicAdd(counter, 1u);  // read after the next barrier
      block_sum3_warps<BLOCK>(cnt, sum, below, red);
      if (threadIdx.x == 0) {
        if (K0 == 0) {  // 2 and 3 are outside the residue arrays (Section 2.1)
          const uint64_t e2 = (p.lo <= 2 && 2 < p.hi), e3 = (p.lo <= 3 && 3 < p.hi);
          cnt += e2 + e3;
          below += e2 + e3;
          sum += 2 * e2 + 3 * e3;
        }
        if (LIST) {
          p.tile_counts[t] = (uint32_t)cnt;
        }
        if (p.count) atomicAdd(p.count, (unsigned long long)cnt);
        if (p.checksum) atomicAdd(p.checksum, (unsigned long long)sum);
        if (p.seg_width && cnt) {
          if (has_b) {
            if (below) atomicAdd(p.bins + sh_bin0, (unsigned long long)below);
            if (cnt - below) atomicAdd(p.bins + sh_bin0 + 1, (unsigned long long)(cnt - below));
          } else {
            atomicAdd(p.bins + sh_bin0, (unsigned long long)cnt);
          }
        }
      }
      if (FUSED) {
        // the tile's output offset, then its survivors straight from shared memory
        if (warp == 0) {
          const uint64_t c = __shfl_sync(kFullMask, cnt, 0);  // thread 0 holds the tile's count
          uint64_t excl = 0;
          const bool ok = lookback_prefix_warp(p.tile_state, t, c, &excl);
          if (lane == 0) {
            sh_lb_ok = ok;
            if (!ok) atomicExch(p.error, 1ull);
            sh_excl = excl;
          }
        }
        __syncthreads();
        if (sh_lb_ok) {
          uint64_t off = sh_excl;
          uint32_t *stage_w = smem + p.stage_off;
          uint32_t *warp_cnt = stage_w + fused_stage_bytes(BLOCK) / sizeof(uint32_t);
          if (K0 == 0 && threadIdx.x == 0) {  // 2 and 3 first
            uint64_t o = off;
            const bool e2 = p.lo <= 2 && 2 < p.hi, e3 = p.lo <= 3 && 3 < p.hi;
            if (p.out_bytes == 4) {
              if (e2 && o < p.cap) ((uint32_t *)p.out)[o] = 2;
              o += e2;
              if (e3 && o < p.cap) ((uint32_t *)p.out)[o] = 3;
            } else {
              if (e2 && o < p.cap) ((uint64_t *)p.out)[o] = 2;
              o += e2;
              if (e3 && o < p.cap) ((uint64_t *)p.out)[o] = 3;
            }
          }
          if (K0 == 0) off += (p.lo <= 2 && 2 < p.hi) + (p.lo <= 3 && 3 < p.hi);
          if (p.out_bytes == 4)
            compact_tile_smem<BLOCK, uint32_t>(s1, s5, tg.logW, K0, off, (uint32_t *)p.out, p.cap, warp_cnt,
                                               (uint8_t *)stage_w);
          else
            compact_tile_smem<BLOCK, uint64_t>(s1, s5, tg.logW, K0, off, (uint64_t *)p.out, p.cap, warp_cnt,
                                               (uint8_t *)stage_w);
        }
      }
    }  // active
    // the next tile and its pattern offsets (a warp other than thread 0's)
    const uint32_t tn = FUSED ? sh_tile : t + gridDim.x;
    if (threadIdx.x >= 32 && threadIdx.x < 32 + (uint32_t)p.npat && tn < t_end)
      sh_poff[threadIdx.x - 32] = pattern_offset(p.k_begin + (uint64_t)tn * p.L, p.pd[threadIdx.x - 32]);
    __syncthreads();
    t = tn;
  }
}

// Exclusive scan of per-tile counts into 64-bit offsets; total at offsets[n].
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) scan_tile_counts_kernel(const uint32_t *__restrict__ counts,
                                                                 uint64_t *__restrict__ offsets,
                                                                 uint32_t n) {
  constexpr int NWARPS = BLOCK / 32;
  __shared__ uint64_t warp_tot[NWARPS];
  __shared__ uint64_t carry;
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += BLOCK) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t x = i < n ? counts[i] : 0;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint64_t y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t wt = lane < NWARPS ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(kFullMask, wt, o);
        if (lane >= (uint32_t)o) wt += y;
      }
      if (lane < NWARPS) warp_tot[lane] = wt;  // inclusive over warps
    }
    __syncthreads();
    const uint64_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (i < n) offsets[i] = before + incl - x;
    __syncthreads();
    if (threadIdx.x == BLOCK - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n] = carry;
}

struct CompactParams {
  uint64_t lo, hi, k_begin, k_end;
  uint32_t L, logW, ntiles;
  const uint2 *bitmap;      // per tile W (class-1 word, class-5 word) pairs, sliced layout
  const uint64_t *offsets;  // ntiles + 1 entries; offsets[ntiles] = total
  void *out;
  uint64_t cap;
};

// List compaction of a range in value order: one tile per CTA iteration
// (compact_tile), after 2 and 3.
// Whether the list compaction stages a tile's bitmap in shared memory (it
// then needs W * 8 bytes of dynamic shared memory before the emission
// staging) or reads it from global memory in both passes.
constexpr bool kRangeCompactSbuf = false;
constexpr uint32_t kRangeStageRow = 96;  // measured best of 64 / 96 / 128

template <int BLOCK, typename OutT>
__global__ void __launch_bounds__(BLOCK) compact_kernel(const CompactParams p) {
  constexpr int NWARPS = BLOCK / 32;
  __shared__ uint32_t warp_cnt[NWARPS * 32];
  extern __shared__ __align__(16) uint2 sbuf[];  // [one tile's bitmap (W pairs)] [emission staging]
  if (p.offsets[p.ntiles] > p.cap) return;  // capacity: the host reports it
  OutT *out = (OutT *)p.out;
  const uint32_t W = p.L / 32;
  uint16_t *stage = (uint16_t *)(sbuf + (kRangeCompactSbuf ? W : 0));
  for (uint32_t t = blockIdx.x; t < p.ntiles; t += gridDim.x) {
    const uint64_t K0 = p.k_begin + (uint64_t)t * p.L;
    const uint2 *bm = p.bitmap + (uint64_t)t * W;
    uint64_t off = p.offsets[t];
    if (K0 == 0) {  // 2 and 3 first
      if (threadIdx.x == 0) {
        uint64_t o = off;
        if (p.lo <= 2 && 2 < p.hi) out[o++] = (OutT)2;
        if (p.lo <= 3 && 3 < p.hi) out[o++] = (OutT)3;
      }
      off += (p.lo <= 2 && 2 < p.hi) + (p.lo <= 3 && 3 < p.hi);
    }
    compact_tile<BLOCK, OutT, kRangeCompactSbuf, kRangeStageRow>(bm, p.logW, K0, off, out, warp_cnt, sbuf, stage);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host side

constexpr int kCompactBlock = 512;

// Dynamic shared memory of compact_kernel for tiles of L indices per class.
static size_t compact_smem_bytes(uint32_t L) {
  return (kRangeCompactSbuf ? (size_t)(L / 32) * sizeof(uint2) : 0) + compact_stage_bytes(kCompactBlock, kRangeStageRow);
}

namespace {

template <int BLOCK, int MODE>
void launch_mode(sieve_ctx *ctx, const RangeKernelParams &p, const BucketParams *b, int grid, size_t smem) {
  if (b) {
    range_tiles_kernel<BLOCK, MODE, kLargeBuckets><<<grid, BLOCK, smem, ctx->stream>>>(p, *b);
  } else {
    BucketParams none;
    memset(&none, 0, sizeof(none));
    range_tiles_kernel<BLOCK, MODE, kLargeTiles><<<grid, BLOCK, smem, ctx->stream>>>(p, none);
  }
}

// The cluster-segment kernel for MODE (count or list bitmap) and BLOCK.
template <int BLOCK>
const void *cluster_kernel(int mode) {
  return mode == kModeListBitmap ? (const void *)range_tiles_kernel<BLOCK, kModeListBitmap, kLargeCluster>
                                 : (const void *)range_tiles_kernel<BLOCK, kModeCount, kLargeCluster>;
}

const void *dispatch_cluster_kernel(int threads, int mode) {
  switch (threads) {
    case 256: return cluster_kernel<256>(mode);
    case 512: return cluster_kernel<512>(mode);
    default: return cluster_kernel<1024>(mode);
  }
}

// Launch configuration of a cluster-segment launch: `grid` CTAs (a multiple
// of C) in one-dimensional clusters of C.
struct ClusterLaunch {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute attr[1];
  ClusterLaunch(int threads, uint32_t C, int grid, size_t smem, cudaStream_t st) {
    memset(&cfg, 0, sizeof(cfg));
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
};

// Clusters of C CTAs that can be resident at once for this kernel (0: none).
int cluster_capacity(int threads, int mode, uint32_t C, size_t smem, int *nclusters) {
  ClusterLaunch cl(threads, C, (int)C, smem, nullptr);
  *nclusters = 0;
  SIEVE_CUDA_TRY(cudaOccupancyMaxActiveClusters(nclusters, dispatch_cluster_kernel(threads, mode), &cl.cfg));
  return SIEVE_OK;
}

int launch_cluster(sieve_ctx *ctx, int threads, const RangeKernelParams &p, int mode, int grid, size_t smem) {
  ClusterLaunch cl(threads, p.cluster, grid, smem, ctx->stream);
  BucketParams none;
  memset(&none, 0, sizeof(none));
  const void *fn = dispatch_cluster_kernel(threads, mode);
  void *args[] = {(void *)&p, (void *)&none};
  SIEVE_CUDA_TRY(cudaLaunchKernelExC(&cl.cfg, fn, args));
  ctx->launches++;
  return SIEVE_OK;
}

template <int BLOCK>
int launch_range_tiles(sieve_ctx *ctx, const RangeKernelParams &p, const BucketParams *b, int mode, int grid,
                       size_t smem) {
  if (mode == kModeListFused) {
    if (BLOCK == 256) {
      set_error("the single-pass list kernel needs 512 or 1024 threads");
      return SIEVE_ERR_INVALID;
    }
    launch_mode<BLOCK, kModeListFused>(ctx, p, b, grid, smem);
  } else if (mode == kModeListBitmap) {
    launch_mode<BLOCK, kModeListBitmap>(ctx, p, b, grid, smem);
  } else {
    launch_mode<BLOCK, kModeCount>(ctx, p, b, grid, smem);
  }
  ctx->launches++;
  SIEVE_CUDA_TRY(cudaGetLastError());
  return SIEVE_OK;
}

template <int BLOCK>
int occupancy(int *blocks, bool list, size_t smem) {
  cudaError_t e = list ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             blocks, range_tiles_kernel<BLOCK, kModeListBitmap, kLargeTiles>, BLOCK, smem)
                       : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                             blocks, range_tiles_kernel<BLOCK, kModeCount, kLargeTiles>, BLOCK, smem);
  SIEVE_CUDA_TRY(e);
  return SIEVE_OK;
}

template <int BLOCK, int MODE>
int set_smem_attr_mode(int bytes) {
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(range_tiles_kernel<BLOCK, MODE, kLargeTiles>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(range_tiles_kernel<BLOCK, MODE, kLargeBuckets>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  if constexpr (MODE != kModeListFused) {
    SIEVE_CUDA_TRY(cudaFuncSetAttribute(range_tiles_kernel<BLOCK, MODE, kLargeCluster>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    // clusters of 16 CTAs are beyond the portable size of 8; a device that
    // refuses them reports no capacity for them later
    if (cudaFuncSetAttribute(range_tiles_kernel<BLOCK, MODE, kLargeCluster>,
                             cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
      cudaGetLastError();
  }
  return SIEVE_OK;
}

template <int BLOCK>
int set_smem_attr(int bytes) {
  int rc;
  if ((rc = set_smem_attr_mode<BLOCK, kModeCount>(bytes)) != SIEVE_OK) return rc;
  if ((rc = set_smem_attr_mode<BLOCK, kModeListBitmap>(bytes)) != SIEVE_OK) return rc;
  if (BLOCK != 256) return set_smem_attr_mode<BLOCK, kModeListFused>(bytes);
  return SIEVE_OK;
}

int dispatch_occupancy(int threads, int *blocks, bool list, size_t smem) {
  switch (threads) {
    case 256: return occupancy<256>(blocks, list, smem);
    case 512: return occupancy<512>(blocks, list, smem);
    default: return occupancy<1024>(blocks, list, smem);
  }
}

int dispatch_launch(sieve_ctx *ctx, int threads, const RangeKernelParams &p, int mode, int grid, size_t smem,
                    const BucketParams *b = nullptr) {
  switch (threads) {
    case 256: return launch_range_tiles<256>(ctx, p, b, mode, grid, smem);
    case 512: return launch_range_tiles<512>(ctx, p, b, mode, grid, smem);
    default: return launch_range_tiles<1024>(ctx, p, b, mode, grid, smem);
  }
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

int range_set_smem_attributes(int bytes) {
  int rc;
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(compact_kernel<kCompactBlock, uint32_t>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(compact_kernel<kCompactBlock, uint64_t>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
  if ((rc = set_smem_attr<256>(bytes)) != SIEVE_OK) return rc;
  if ((rc = set_smem_attr<512>(bytes)) != SIEVE_OK) return rc;
  return set_smem_attr<1024>(bytes);
}

// Largest power of two <= x (x >= 1).
static uint32_t floor_pow2(uint64_t x) {
  uint32_t r = 1;
  while ((uint64_t)r * 2 <= x && r < (1u << 30)) r *= 2;
  return r;
}

// Records phase-timing event i on the context's stream when timing is on.
static void phase_event(sieve_ctx *ctx, int i) {
  if (!ctx->phase_timing) return;
  if (cudaEventRecord(ctx->ph_ev[i], ctx->stream) == cudaSuccess) ctx->ph_recorded |= 1u << i;
}

static uint32_t log2u(uint32_t x) {
  uint32_t r = 0;
  while ((1u << r) < x) r++;
  return r;
}

// Tile geometry of a single-range call (shared by run_range and the routing
// decision of sieve_range): tile length L (tile_bits, at most one segment
// boundary per tile when per-segment counts are asked for, smaller tiles when
// the range gives fewer than one full tile per CTA slot), tile count, grid,
// base primes needed and the warp/lane split (a warp takes a prime while it
// has >= group_hits hits per lane in a tile, i.e. P <= L / (32 group_hits)),
// and the dynamic shared memory of the tile kernel.
struct RangeGeom {
  uint64_t k_begin, k_end;  // class indices [k_begin, k_end) cover [lo, hi)
  uint32_t L, ntiles, np, i_first, i_split;
  int threads, grid;
  size_t smem;
};

static int range_geometry(const sieve_ctx *ctx, const DeviceTable &table, uint64_t lo, uint64_t hi,
                          uint64_t seg_width, bool list, RangeGeom *g) {
  g->k_begin = lo / 6;
  g->k_end = (hi + 4) / 6;  // ceil((hi - 1) / 6)
  const uint64_t span = g->k_end > g->k_begin ? g->k_end - g->k_begin : 0;
  g->threads = (int)ctx->opt.block_threads;
  uint32_t L = ctx->opt.tile_bits;
  if (seg_width) {  // at most one segment boundary per tile: 6 L <= seg_width
    const uint32_t lw = floor_pow2(seg_width / 6);
    if (lw < L) L = lw;
  }
  int per_sm = 0;
  const int ti = g->threads == 256 ? 0 : (g->threads == 512 ? 1 : 2);
  const uint32_t lg = log2u(L) & 31;
  int *cached = const_cast<int *>(&ctx->occ_cache[ti][list ? 1 : 0][lg]);
  if (*cached > 0) {
    per_sm = *cached;
  } else {
    int rc = dispatch_occupancy(g->threads, &per_sm, list, (size_t)L / 4);
    if (rc != SIEVE_OK) return rc;
    if (per_sm > 0) *cached = per_sm;
  }
  if (per_sm < 1) {
    set_error("tile of %u bits does not fit on an SM", L);
    return SIEVE_ERR_INVALID;
  }
  if (ctx->opt.ctas_per_sm && (int)ctx->opt.ctas_per_sm < per_sm) per_sm = (int)ctx->opt.ctas_per_sm;
  const uint64_t slots = (uint64_t)ctx->num_sms * (uint64_t)per_sm;
  // small ranges: shrink tiles so that every CTA slot gets work
  if (span > 0 && span < (uint64_t)L * slots) {
    const uint64_t want = (span + slots - 1) / slots;
    uint32_t lw = floor_pow2(want);
    if (lw < want) lw *= 2;
    if (lw < 1024) lw = 1024;
    if (lw < L) L = lw;
  }
  const uint64_t ntiles64 = span ? (span + L - 1) / L : 0;
  if (ntiles64 > 0xFFFFFFF0ull) {
    set_error("range needs too many tiles");
    return SIEVE_ERR_INVALID;
  }
  g->L = L;
  g->ntiles = (uint32_t)ntiles64;
  g->grid = (int)std::min<uint64_t>(g->ntiles ? g->ntiles : 1, slots);
  const uint64_t s = hi >= 2 ? isqrt_u64(hi - 1) : 0;
  g->np = host_prime_count_le_table(table, s);
  const uint64_t gmax = L / (32ull * std::max<uint32_t>(1u, ctx->opt.group_hits));
  g->i_first = first_struck_prime_index((int)ctx->opt.presieve_groups);
  g->i_split = std::min(host_prime_count_le_table(table, gmax), g->np);
  if (g->i_split < g->i_first) g->i_split = g->i_first;
  g->smem = (size_t)L / 4 + (size_t)(g->i_split - g->i_first) * sizeof(uint2);
  if (g->smem > (size_t)ctx->smem_optin) {
    set_error("tile of %u bits with %u warp-band primes needs %zu bytes of shared memory", L,
              g->i_split - g->i_first, g->smem);
    return SIEVE_ERR_INVALID;
  }
  return SIEVE_OK;
}

constexpr int kScatterBlock = 512;  // threads of bucket_scatter_kernel
constexpr uint32_t kBucketPresieveGroups = 4;  // presieve groups copied when the bucket sieve runs
constexpr int kScatterHits = 16;    // hits per thread per round

// Upper bound on the sum of 1/p over the primes p in (a, b], a >= 286: with
// Rosser & Schoenfeld's bound |sum_{p <= x} 1/p - ln ln x - B| < 1 / (2 ln^2 x)
// ("Approximate formulas for some functions of prime numbers", 1962, (3.18)).
static double prime_reciprocal_sum_bound(double a, double b) {
  if (b <= a) return 0.0;
  const double la = std::log(a), lb = std::log(b);
  return std::log(lb) - std::log(la) + 0.5 / (la * la) + 0.5 / (lb * lb);
}

// Which scatter kernel and how many bytes of bucket entries a wave of one
// tile per CTA holds, above which the sorted scatter (coalesced writes, waves
// of at least four tiles per CTA) beats the direct one (measured: the direct
// scatter's scattered stores are cheap while the wave's entries stay in L2).
constexpr double kBucketDirectMaxBytes = 96e6;

static size_t scatter_smem(bool sorted, uint32_t ntl) {
  return sorted ? bucket_scatter_smem(kScatterBlock, kScatterHits, ntl) : (size_t)ntl * sizeof(uint32_t);
}

// Scatter CTAs per SM for a wave of ntl tiles (occupancy of the scatter kernel).
static int scatter_ctas_per_sm(bool sorted, uint32_t ntl) {
  int blocks = 0;
  const size_t smem = scatter_smem(sorted, ntl);
  const void *fn = sorted ? (const void *)bucket_scatter_kernel<kScatterBlock, kScatterHits>
                          : (const void *)bucket_scatter_direct_kernel<kScatterBlock>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kScatterBlock, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return blocks;
}

// Whether a range's large primes go through the bucket sieve, and its layout:
// the primes above bucket_threshold x L (table indices [i_large, np)) when
// there are many of them and each hits a tile's two classes rarely.  The mean
// hits per prime per tile, h = 2 L sum(1/p) / N, must stay below
// kBucketMaxHits: a bucket entry costs about four per-tile locations
// (measured break-even near h = 0.28 at [1e14, 1e14 + 1e11)).  Waves of
// bucket_wave x grid tiles (at least four per CTA for the sorted scatter);
// sub-bucket capacity from the expected hits per (tile, scatter CTA) with a
// margin of six standard deviations (overflow is handled by the tile, see
// bucket.cuh).  With plan == nullptr only the decision is made (no device
// calls); else *plan receives the layout (without t_begin / ntl).
struct BucketPlan {
  BucketParams b;
  uint32_t wave;
  bool sorted;
};

static bool plan_buckets(const sieve_ctx *ctx, const DeviceTable &table, const RangeGeom &g, BucketPlan *plan) {
  constexpr uint32_t kBucketMinPrimes = 8192;
  constexpr double kBucketMaxHits = 0.25;
  const sieve_options &o = ctx->opt;
  if (!o.bucket_threshold || g.ntiles < 2 || g.np == 0) return false;
  const uint32_t Pmax = table.host_primes[g.np - 1];
  if (Pmax >= 0x80000000u) return false;
  // bucket_threshold x L is the lowest threshold; while the primes above it
  // hit a tile too often, raise it by a quarter (a range whose top primes sit
  // just above 4 L keeps its buckets for the primes above 5 L: [5e13, +1e11)
  // 43.8 ms without them, 40.8 with the primes above 6 L)
  uint64_t T = (uint64_t)o.bucket_threshold * g.L;
  uint32_t i_large = 0;
  double e_tile = 0.0;
  for (;;) {
    i_large = host_prime_count_le_table(table, T);
    if (i_large < g.i_split) i_large = g.i_split;
    if (g.np < i_large + kBucketMinPrimes) return false;
    const uint32_t Plo = table.host_primes[i_large];
    const double S = prime_reciprocal_sum_bound(std::max<double>(Plo - 1, 286.0), (double)Pmax);
    const double n_large = (double)(g.np - i_large);
    e_tile = 2.0 * g.L * S;  // expected bucket entries per tile
    if (e_tile / n_large <= kBucketMaxHits) break;
    T += T / 4;
  }
  if (!plan) return true;
  const bool sorted = o.bucket_scatter == 2 ||
                      (o.bucket_scatter == 0 && e_tile * g.grid * sizeof(uint32_t) > kBucketDirectMaxBytes);
  uint32_t per_cta = std::max<uint32_t>(1u, o.bucket_wave);
  if (sorted && o.bucket_scatter == 0) per_cta = std::max<uint32_t>(per_cta, 4u);
  uint64_t ntl = (uint64_t)per_cta * g.grid;
  ntl = std::min<uint64_t>(ntl, g.ntiles);
  ntl = std::min<uint64_t>(ntl, kBucketMaxWaveTiles - 1);
  while (ntl > 1 && ntl * g.L >= (1ull << 31)) ntl--;
  const int scatter_ctas = scatter_ctas_per_sm(sorted, (uint32_t)ntl) * ctx->num_sms;
  if (scatter_ctas < 1) return false;
  const double e = e_tile / scatter_ctas;
  uint32_t cap = ((uint32_t)(e + 6.0 * std::sqrt(e) + 64.0) + 31u) & ~31u;
  // SIEVE_BUCKET_CAP overrides the capacity (tests use a small one to make
  // sub-buckets overflow and so exercise the tiles' fallback)
  if (const char *env = std::getenv("SIEVE_BUCKET_CAP")) {
    const long v = std::strtol(env, nullptr, 10);
    if (v >= 1 && v < (long)cap) cap = (uint32_t)v;
  }
  BucketParams &b = plan->b;
  memset(&b, 0, sizeof(b));
  b.cap = cap;
  b.ncta = (uint32_t)scatter_ctas;
  b.i_large = i_large;
  b.i_end = g.np;
  b.k_begin = g.k_begin;
  b.k_end = g.k_end;
  b.L = g.L;
  b.logW = log2u(g.L / 32);
  b.primes = table.primes;
  b.magic = table.magic;
  b.cinv = table.cinv;
  plan->wave = (uint32_t)ntl;
  plan->sorted = sorted;
  return true;
}

bool range_prefers_buckets(sieve_ctx *ctx, uint64_t lo, uint64_t hi) {
  if (hi <= lo || hi > (1ull << 63) || isqrt_u64(hi - 1) > ctx->table.limit) return false;
  RangeGeom g;
  if (range_geometry(ctx, ctx->table, lo, hi, 0, false, &g) != SIEVE_OK) return false;
  return plan_buckets(ctx, ctx->table, g, nullptr);
}

// Bucket buffers of the context (kept across calls, grown on demand).
static int ensure_buckets(sieve_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->bucket_bytes) return SIEVE_OK;
  if (ctx->d_bucket) {
    SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_bucket);
    ctx->d_bucket = nullptr;
    ctx->bucket_bytes = 0;
  }
  SIEVE_CUDA_TRY(cudaMalloc(&ctx->d_bucket, bytes));
  ctx->bucket_bytes = bytes;
  return SIEVE_OK;
}

int run_range(sieve_ctx *ctx, const DeviceTable &table, const RangeRequest &req, size_t *n_out) {
  if (n_out) *n_out = 0;
  if (req.lo > req.hi) {
    set_error("lo (%llu) > hi (%llu)", (unsigned long long)req.lo, (unsigned long long)req.hi);
    return SIEVE_ERR_INVALID;
  }
  if (req.hi > (1ull << 63)) {
    set_error("hi must be <= 2^63");
    return SIEVE_ERR_RANGE;
  }
  if (req.seg_width) {
    if (req.seg_width < 6144) {
      set_error("seg_width must be >= 6144");
      return SIEVE_ERR_INVALID;
    }
    const size_t need = req.hi > req.lo ? (size_t)((req.hi - 1) / req.seg_width - req.lo / req.seg_width + 1) : 0;
    if (req.nbins != need) {
      set_error("ncounts must be %zu for this range and seg_width", need);
      return SIEVE_ERR_INVALID;
    }
  }
  const bool dev_out = req.out_on_device != 0;
  cudaStream_t st = ctx->stream;

  // empty range: zero every output
  if (req.lo == req.hi) {
    if (req.total) {
      if (dev_out) {
        SIEVE_CUDA_TRY(cudaMemsetAsync(req.total, 0, sizeof(sieve_count_result), st));
      } else {
        req.total->count = 0;
        req.total->checksum = 0;
      }
    }
    if (!req.async) SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIEVE_OK;
  }
  const uint64_t s = isqrt_u64(req.hi - 1);
  if (s > table.limit) {
    set_error("isqrt(hi - 1) = %llu exceeds the base table limit %llu (context max_hi too small)",
              (unsigned long long)s, (unsigned long long)table.limit);
    return SIEVE_ERR_RANGE;
  }

  RangeGeom g;
  int rc = range_geometry(ctx, table, req.lo, req.hi, req.seg_width, req.list != 0, &g);
  if (rc != SIEVE_OK) return rc;
  const uint64_t k_begin = g.k_begin, k_end = g.k_end;
  const int threads = g.threads;
  const uint32_t L = g.L, ntiles = g.ntiles, np = g.np, i_first = g.i_first, i_split = g.i_split;
  const int grid = g.grid;
  size_t smem = g.smem;

  RangeKernelParams p;
  memset(&p, 0, sizeof(p));
  p.lo = req.lo;
  p.hi = req.hi;
  p.k_begin = k_begin;
  p.k_end = k_end;
  p.L = L;
  p.logW = log2u(L / 32);
  p.ntiles = ntiles;
  p.primes = table.primes;
  p.magic = table.magic;
  p.cinv = table.cinv;
  p.nprimes = np;
  p.i_split = i_split;
  p.i_first = i_first;
  p.npat = 1 + (int)ctx->opt.presieve_groups;
  rc = sliced_patterns(ctx, p.logW, &p.sliced, p.pd);
  if (rc != SIEVE_OK) return rc;
  p.seg_width = req.seg_width;
  p.first_seg = req.seg_width ? req.lo / req.seg_width : 0;

  // where count / checksum / bins accumulate
  unsigned long long *acc = ctx->d_acc;  // [0] count, [1] checksum
  const bool total_direct = dev_out && req.total && !req.list;
  if (total_direct) {
    p.count = (unsigned long long *)&req.total->count;
    p.checksum = (unsigned long long *)&req.total->checksum;
    SIEVE_CUDA_TRY(cudaMemsetAsync(req.total, 0, sizeof(sieve_count_result), st));
  } else {
    p.count = acc;
    p.checksum = acc + 1;
    SIEVE_CUDA_TRY(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), st));
  }

  // single-pass list: device output, 512 or 1024 threads, and room in shared
  // memory for the emission staging (it reuses the warp-band starts' space)
  const int nwarps = threads / 32;
  const size_t fused_smem =
      (size_t)L / 4 + std::max(align_up((size_t)(i_split - i_first) * sizeof(uint2), 16),
                               fused_stage_bytes(threads) + (size_t)nwarps * 32 * sizeof(uint32_t));
  const bool fused = req.list && dev_out && threads != 256 && ctx->opt.list_single_pass &&
                     fused_smem <= (size_t)ctx->smem_optin;
  // cluster segments (option cluster_ctas): not with the single-pass list,
  // and only while every needed prime is below 2^31 (the inverse-of-6 start)
  const uint32_t C = ctx->opt.cluster_ctas;
  const bool use_cluster = C >= 2 && ntiles && !fused && np && table.host_primes[np - 1] < 0x80000000u;
  BucketPlan plan;
  const bool use_buckets = !use_cluster && ntiles && plan_buckets(ctx, table, g, &plan);
  const uint32_t nwaves = use_buckets ? (ntiles + plan.wave - 1) / plan.wave : 1;
  size_t fused_smem_used = fused_smem;
  if (use_buckets && ctx->opt.presieve_groups > kBucketPresieveGroups) {
    // with the bucket sieve at most kBucketPresieveGroups groups are copied:
    // a wave's bucket entries (tens of MB) and the larger groups' patterns
    // then compete for L2, and those patterns cost more than the strikes
    // they save ([1e14, +1e11): 39.2 ms with 4 groups, 42.5 with 7, 45.6
    // with 8; the headline, without buckets, is fastest with 7)
    p.npat = 1 + kBucketPresieveGroups;
    p.i_first = first_struck_prime_index(kBucketPresieveGroups);
    const size_t starts_bytes = (size_t)(i_split - p.i_first) * sizeof(uint2);
    smem = (size_t)L / 4 + starts_bytes;
    fused_smem_used = (size_t)L / 4 + std::max(align_up(starts_bytes, 16), fused_stage_bytes(threads) +
                                                                             (size_t)nwarps * 32 * sizeof(uint32_t));
    if (std::max(smem, fused ? fused_smem_used : 0) > (size_t)ctx->smem_optin) {
      set_error("tile of %u bits with %u warp-band primes needs %zu bytes of shared memory", L,
                i_split - p.i_first, smem);
      return SIEVE_ERR_INVALID;
    }
  }

  // scratch layout: [bins (host-output case)] [tile counts] [offsets] [bitmap]
  // (two-pass list) or [tile states] [tile counters] [error word] (single pass)
  size_t off_bins = 0, off_counts = 0, off_offsets = 0, off_bitmap = 0, need = 0;
  size_t off_state = 0, off_ctr = 0, off_err = 0;
  const bool bins_direct = dev_out;
  if (req.seg_width && !bins_direct) {
    off_bins = need;
    need = align_up(need + req.nbins * sizeof(uint64_t), 256);
  }
  if (fused) {
    off_state = need;
    need = align_up(need + (size_t)ntiles * sizeof(uint64_t), 256);
    off_ctr = need;
    need = align_up(need + (size_t)nwaves * sizeof(uint32_t), 256);
    off_err = need;
    need = align_up(need + sizeof(uint64_t), 256);
  } else if (req.list) {
    off_counts = need;
    need = align_up(need + (size_t)ntiles * sizeof(uint32_t), 256);
    off_offsets = need;
    need = align_up(need + ((size_t)ntiles + 1) * sizeof(uint64_t), 256);
    off_bitmap = need;
    need = align_up(need + (size_t)ntiles * (L / 32) * sizeof(uint2), 256);
  }
  if (need) {
    rc = ensure_scratch(ctx, need);
    if (rc != SIEVE_OK) return rc;
  }
  char *scr = (char *)ctx->d_scratch;
  if (req.seg_width) {
    p.bins = bins_direct ? (unsigned long long *)req.bins : (unsigned long long *)(scr + off_bins);
    SIEVE_CUDA_TRY(cudaMemsetAsync(p.bins, 0, req.nbins * sizeof(uint64_t), st));
  }
  if (fused) {
    p.tile_state = (unsigned long long *)(scr + off_state);
    p.tile_counter = (uint32_t *)(scr + off_ctr);
    p.error = (unsigned long long *)(scr + off_err);
    SIEVE_CUDA_TRY(cudaMemsetAsync(scr + off_state, 0, off_err + sizeof(uint64_t) - off_state, st));
    p.out = req.out;
    p.cap = req.cap;
    p.out_bytes = (uint32_t)req.out_bytes;
    p.stage_off = 2 * (L / 32);
    smem = fused_smem_used;
  } else if (req.list) {
    p.tile_counts = (uint32_t *)(scr + off_counts);
    p.bitmap = (uint2 *)(scr + off_bitmap);
  }
  const int mode = fused ? kModeListFused : (req.list ? kModeListBitmap : kModeCount);

  if (ctx->phase_timing) {
    ctx->ph = sieve_phase_times{};
    ctx->ph.tiles = ntiles;
    ctx->ph.tile_len = L;
    ctx->ph_recorded = 0;
    phase_event(ctx, 0);
  }
  if (ntiles) {
    if (use_cluster) {
      // one launch of clusters of C CTAs, each cluster taking segments of C
      // consecutive tiles in grid-stride order
      p.cluster = C;
      p.i_cluster = std::max(host_prime_count_le_table(table, (uint64_t)ctx->opt.cluster_threshold * L), i_split);
      int ncl = 0;
      rc = cluster_capacity(threads, mode, C, smem, &ncl);
      if (rc != SIEVE_OK) return rc;
      if (ncl < 1) {
        set_error("no cluster of %u CTAs of %d threads and %zu bytes of shared memory fits on the device", C,
                  threads, smem);
        return SIEVE_ERR_INVALID;
      }
      const uint64_t nseg = (ntiles + C - 1) / C;
      rc = launch_cluster(ctx, threads, p, mode, (int)(std::min<uint64_t>(nseg, (uint64_t)ncl) * C), smem);
      if (rc != SIEVE_OK) return rc;
      if (ctx->phase_timing) ctx->ph.cluster_ctas = C;
    } else if (use_buckets) {
      // the bucket sieve: per wave, the scatter, then the wave's tiles
      BucketParams &bk = plan.b;
      const uint32_t wave = plan.wave;
      const size_t n_sub = (size_t)wave * bk.ncta;
      const size_t off_counts = align_up(n_sub * bk.cap * sizeof(uint32_t), 256);
      const size_t off_ovf = align_up(off_counts + n_sub * sizeof(uint32_t), 256);
      rc = ensure_buckets(ctx, off_ovf + (size_t)wave * sizeof(uint32_t));
      if (rc != SIEVE_OK) return rc;
      char *bb = (char *)ctx->d_bucket;
      bk.entries = (uint32_t *)bb;
      bk.counts = (uint32_t *)(bb + off_counts);
      bk.overflow = (uint32_t *)(bb + off_ovf);
      SIEVE_CUDA_TRY(cudaMemsetAsync(bk.overflow, 0, (size_t)wave * sizeof(uint32_t), st));
      const size_t ssmem = scatter_smem(plan.sorted, wave);
      for (uint32_t t0 = 0; t0 < ntiles; t0 += wave) {
        bk.t_begin = t0;
        bk.ntl = std::min(wave, ntiles - t0);
        bk.wave_id = t0 / wave;
        if (plan.sorted)
          bucket_scatter_kernel<kScatterBlock, kScatterHits><<<bk.ncta, kScatterBlock, ssmem, st>>>(bk);
        else
          bucket_scatter_direct_kernel<kScatterBlock><<<bk.ncta, kScatterBlock, ssmem, st>>>(bk);
        ctx->launches++;
        SIEVE_CUDA_TRY(cudaGetLastError());
        rc = dispatch_launch(ctx, threads, p, mode, (int)std::min<uint32_t>(grid, bk.ntl), smem, &bk);
        if (rc != SIEVE_OK) return rc;
      }
      if (ctx->phase_timing) ctx->ph.bucket_waves = (ntiles + wave - 1) / wave;
    } else {
      rc = dispatch_launch(ctx, threads, p, mode, grid, smem);
      if (rc != SIEVE_OK) return rc;
    }
  }
  phase_event(ctx, 1);

  if (fused) {  // the list is written: read the total (the last tile's inclusive prefix) and the error word
    ctx->h_acc[2] = 0;
    ctx->h_acc[3] = 0;
    if (ntiles) {
      SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc + 2, p.tile_state + (ntiles - 1), sizeof(uint64_t),
                                     cudaMemcpyDeviceToHost, st));
      SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc + 3, p.error, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
    }
    SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
    SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    if (ctx->h_acc[3] || (ntiles && (ctx->h_acc[2] >> kLookbackFlagShift) != 2)) {
      set_error("single-pass list: a tile's look-back gave up waiting for an earlier tile");
      return SIEVE_ERR_TIMEOUT;
    }
    const uint64_t total = ctx->h_acc[2] & kLookbackValueMask;
    if (n_out) *n_out = (size_t)total;
    if (ctx->phase_timing) ctx->ph.listed = total < req.cap ? total : req.cap;
    if (req.total) {
      sieve_count_result r{ctx->h_acc[0], ctx->h_acc[1]};
      SIEVE_CUDA_TRY(cudaMemcpy(req.total, &r, sizeof(r), cudaMemcpyHostToDevice));
    }
    if (total > req.cap) {
      set_error("output capacity %zu is below the %llu primes found", req.cap, (unsigned long long)total);
      return SIEVE_ERR_CAPACITY;
    }
    return SIEVE_OK;
  }

  if (!req.list) {
    if (!dev_out) {
      SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
      if (req.seg_width)
        SIEVE_CUDA_TRY(cudaMemcpyAsync(req.bins, p.bins, req.nbins * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
      SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
      if (req.total) {
        req.total->count = ctx->h_acc[0];
        req.total->checksum = ctx->h_acc[1];
      }
    } else if (!req.async) {
      SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return SIEVE_OK;
  }

  // list mode: scan, read the total, compact
  uint64_t *offsets = (uint64_t *)(scr + off_offsets);
  if (ntiles) {
    scan_tile_counts_kernel<1024><<<1, 1024, 0, st>>>(p.tile_counts, offsets, ntiles);
    ctx->launches++;
    SIEVE_CUDA_TRY(cudaGetLastError());
    phase_event(ctx, 2);
    SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc + 2, offsets + ntiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  } else {
    ctx->h_acc[2] = 0;
  }
  SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  const uint64_t total = ctx->h_acc[2];
  if (n_out) *n_out = (size_t)total;
  if (req.total) {
    sieve_count_result r{ctx->h_acc[0], ctx->h_acc[1]};
    if (dev_out)
      SIEVE_CUDA_TRY(cudaMemcpyAsync(req.total, &r, sizeof(r), cudaMemcpyHostToDevice, st));
    else
      *req.total = r;
  }
  if (total > req.cap) {
    set_error("output capacity %zu is below the %llu primes found", req.cap, (unsigned long long)total);
    if (dev_out) SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIEVE_ERR_CAPACITY;
  }
  if (total == 0) {
    if (dev_out) SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIEVE_OK;
  }
  void *dst = req.out;
  if (!dev_out) {  // stage on the device, then copy to the caller's host buffer
    rc = ensure_stage(ctx, (size_t)total * req.out_bytes);
    if (rc != SIEVE_OK) return rc;
    dst = ctx->d_stage;
  }
  CompactParams cp;
  cp.lo = req.lo;
  cp.hi = req.hi;
  cp.k_begin = k_begin;
  cp.k_end = k_end;
  cp.L = L;
  cp.logW = p.logW;
  cp.ntiles = ntiles;
  cp.bitmap = p.bitmap;
  cp.offsets = offsets;
  cp.out = dst;
  cp.cap = req.cap;
  const size_t csmem = compact_smem_bytes(L);
  const int cgrid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 4);
  phase_event(ctx, 3);
  if (req.out_bytes == 4)
    compact_kernel<kCompactBlock, uint32_t><<<cgrid, kCompactBlock, csmem, st>>>(cp);
  else
    compact_kernel<kCompactBlock, uint64_t><<<cgrid, kCompactBlock, csmem, st>>>(cp);
  ctx->launches++;
  SIEVE_CUDA_TRY(cudaGetLastError());
  phase_event(ctx, 4);
  if (ctx->phase_timing) ctx->ph.listed = total;
  if (!dev_out)
    SIEVE_CUDA_TRY(cudaMemcpyAsync(req.out, dst, (size_t)total * req.out_bytes, cudaMemcpyDeviceToHost, st));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  return SIEVE_OK;
}

}  // namespace sieve

namespace sieve {

// Tile length and count of a list-mode range of `span` indices per class on
// `slots` CTA slots with tiles of at most L indices (the rule run_range
// applies: a range smaller than one full tile per slot gets smaller tiles,
// down to 1024), and the scratch bytes its per-tile counts, offsets and
// bitmaps take in the layout of run_range_list_into.
static size_t list_scratch_need(uint64_t span, uint32_t L, uint64_t slots, uint32_t *L_used, uint64_t *ntiles) {
  if (span > 0 && span < (uint64_t)L * slots) {
    const uint64_t want = (span + slots - 1) / slots;
    uint32_t lw = floor_pow2(want);
    if (lw < want) lw *= 2;
    if (lw < 1024) lw = 1024;
    if (lw < L) L = lw;
  }
  const uint64_t n = span ? (span + L - 1) / L : 0;
  if (L_used) *L_used = L;
  if (ntiles) *ntiles = n;
  const size_t off_offsets = align_up((size_t)n * sizeof(uint32_t), 256);
  const size_t off_bitmap = align_up(off_offsets + ((size_t)n + 1) * sizeof(uint64_t), 256);
  return off_bitmap + (size_t)n * (L / 32) * sizeof(uint2);
}

// The widest range whose list scratch fits in `bytes` wherever it starts: the
// largest span S (indices per class) that fits, found by bisection over the
// same layout (the need grows with the span), turned into a width: a range of
// w numbers covers at most floor((w + 9) / 6) indices per class, which is
// <= S for every w <= 6 S - 4.
static uint64_t list_scratch_max_width(uint32_t L, uint64_t slots, size_t bytes) {
  uint64_t lo = 0, hi = (uint64_t)bytes * 8;  // a span of 8 indices per byte never fits
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    (list_scratch_need(mid, L, slots, nullptr, nullptr) <= bytes ? lo : hi) = mid;
  }
  return lo >= 1 ? 6 * lo - 4 : 0;
}

// List-mode sieve of [lo, hi) into the device buffer `out` using caller-given
// scratch and no allocation of any kind: no presieve patterns (every base
// prime from 5 on is struck), the context's preallocated accumulators, and
// `scratch` for the per-tile counts, offsets and bitmaps.  Used by the
// entry point that allocates nothing (noalloc.cu).
int run_range_list_into(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out, size_t cap, size_t *n_out,
                        sieve_count_result *cnt, void *scratch, size_t scratch_bytes) {
  if (n_out) *n_out = 0;
  if (cnt) {
    cnt->count = 0;
    cnt->checksum = 0;
  }
  if (lo > hi) {
    set_error("lo (%llu) > hi (%llu)", (unsigned long long)lo, (unsigned long long)hi);
    return SIEVE_ERR_INVALID;
  }
  if (hi > (1ull << 63)) {
    set_error("hi must be <= 2^63");
    return SIEVE_ERR_RANGE;
  }
  if (lo == hi) return SIEVE_OK;
  const DeviceTable &table = ctx->table;
  const uint64_t s = isqrt_u64(hi - 1);
  if (s > table.limit) {
    set_error("isqrt(hi - 1) = %llu exceeds the base table limit %llu", (unsigned long long)s,
              (unsigned long long)table.limit);
    return SIEVE_ERR_RANGE;
  }
  cudaStream_t st = ctx->stream;
  const uint64_t k_begin = lo / 6;
  const uint64_t k_end = (hi + 4) / 6;
  const uint64_t span = k_end > k_begin ? k_end - k_begin : 0;
  const int threads = (int)ctx->opt.block_threads;
  uint32_t L = ctx->opt.tile_bits;
  size_t smem = (size_t)L / 4;
  int per_sm = 0;
  int rc = dispatch_occupancy(threads, &per_sm, true, smem);
  if (rc != SIEVE_OK) return rc;
  if (per_sm < 1) {
    set_error("tile of %u bits does not fit on an SM", L);
    return SIEVE_ERR_INVALID;
  }
  if (ctx->opt.ctas_per_sm && (int)ctx->opt.ctas_per_sm < per_sm) per_sm = (int)ctx->opt.ctas_per_sm;
  const uint64_t slots = (uint64_t)ctx->num_sms * (uint64_t)per_sm;
  uint64_t ntiles64 = 0;
  const size_t need = list_scratch_need(span, L, slots, &L, &ntiles64);
  smem = (size_t)L / 4;
  // scratch layout: [tile counts][offsets][bitmaps]
  const size_t off_offsets = align_up((size_t)ntiles64 * sizeof(uint32_t), 256);
  const size_t off_bitmap = align_up(off_offsets + ((size_t)ntiles64 + 1) * sizeof(uint64_t), 256);
  if (ntiles64 > 0xFFFFFFF0ull || need > scratch_bytes) {
    set_error("range [%llu, %llu) needs %zu bytes of scratch; the fixed scratch holds %zu, enough for "
              "ranges of up to %llu numbers with this context's tile length",
              (unsigned long long)lo, (unsigned long long)hi, need, scratch_bytes,
              (unsigned long long)list_scratch_max_width(ctx->opt.tile_bits, slots, scratch_bytes));
    return SIEVE_ERR_INVALID;
  }
  const uint32_t ntiles = (uint32_t)ntiles64;
  const int grid = (int)std::min<uint64_t>(ntiles ? ntiles : 1, slots);
  const uint32_t np = host_prime_count_le_table(table, s);
  const uint32_t i_first = 2;  // no presieve: strike from 5 on
  const uint64_t gmax = L / (32ull * std::max<uint32_t>(1u, ctx->opt.group_hits));
  uint32_t i_split = std::min(host_prime_count_le_table(table, gmax), np);
  if (i_split < i_first) i_split = i_first;
  smem += (size_t)(i_split - i_first) * sizeof(uint2);
  if (smem > (size_t)ctx->smem_optin) {
    set_error("tile of %u bits needs %zu bytes of shared memory", L, smem);
    return SIEVE_ERR_INVALID;
  }
  char *scr = (char *)scratch;
  RangeKernelParams p;
  memset(&p, 0, sizeof(p));
  p.lo = lo;
  p.hi = hi;
  p.k_begin = k_begin;
  p.k_end = k_end;
  p.L = L;
  p.logW = log2u(L / 32);
  p.ntiles = ntiles;
  p.primes = table.primes;
  p.magic = table.magic;
  p.cinv = table.cinv;
  p.nprimes = np;
  p.i_first = i_first;
  p.i_split = i_split;
  p.npat = 0;
  p.sliced = nullptr;
  p.count = ctx->d_acc;
  p.checksum = ctx->d_acc + 1;
  p.tile_counts = (uint32_t *)scr;
  p.bitmap = (uint2 *)(scr + off_bitmap);
  uint64_t *offsets = (uint64_t *)(scr + off_offsets);
  SIEVE_CUDA_TRY(cudaMemsetAsync(ctx->d_acc, 0, 2 * sizeof(unsigned long long), st));
  if (ntiles) {
    rc = dispatch_launch(ctx, threads, p, kModeListBitmap, grid, smem);
    if (rc != SIEVE_OK) return rc;
    scan_tile_counts_kernel<1024><<<1, 1024, 0, st>>>(p.tile_counts, offsets, ntiles);
    ctx->launches++;
    SIEVE_CUDA_TRY(cudaGetLastError());
    SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc + 2, offsets + ntiles, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  } else {
    ctx->h_acc[2] = 0;
  }
  SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->h_acc, ctx->d_acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  const uint64_t total = ctx->h_acc[2];
  if (n_out) *n_out = (size_t)total;
  if (cnt) {
    cnt->count = ctx->h_acc[0];
    cnt->checksum = ctx->h_acc[1];
  }
  if (total > cap) {
    set_error("output capacity %zu is below the %llu primes found", cap, (unsigned long long)total);
    return SIEVE_ERR_CAPACITY;
  }
  if (total == 0) return SIEVE_OK;
  CompactParams cp;
  cp.lo = lo;
  cp.hi = hi;
  cp.k_begin = k_begin;
  cp.k_end = k_end;
  cp.L = L;
  cp.logW = p.logW;
  cp.ntiles = ntiles;
  cp.bitmap = p.bitmap;
  cp.offsets = offsets;
  cp.out = out;
  cp.cap = cap;
  const int cgrid = (int)std::min<uint64_t>(ntiles, (uint64_t)ctx->num_sms * 4);
  compact_kernel<kCompactBlock, uint64_t><<<cgrid, kCompactBlock, compact_smem_bytes(L), st>>>(cp);
  ctx->launches++;
  SIEVE_CUDA_TRY(cudaGetLastError());
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  return SIEVE_OK;
}

}  // namespace sieve
