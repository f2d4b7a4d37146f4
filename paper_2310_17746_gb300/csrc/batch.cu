// batch.cu -- the batched range sieve: kernels, host planner, CUDA-graph runner
// and the public sieve_range_batch call.  The data layout and the two kinds of
// work items are described in batch.cuh.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <new>

#include "batch.cuh"
#include "tile.cuh"

namespace sieve {

// ---------------------------------------------------------------- kernels

// Zero the per-batch state and accumulators; set the merge bitmaps to all ones
// (a merged tile starts with every candidate alive; items only clear bits).
__global__ void batch_init_kernel(const BatchArena a) {
  const BatchHeader *hdr = (const BatchHeader *)a.plan;
  const uint32_t nq = hdr->nq;
  const uint64_t words = hdr->slot_words;
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t nth = (uint64_t)gridDim.x * blockDim.x;
  if (tid == 0) {
    a.state->next_item = 0;
    a.state->status = 0;
  }
  for (uint64_t i = tid; i < 2ull * nq; i += nth) a.acc[i] = 0;
  uint4 *bm4 = (uint4 *)a.slot_bm;  // slot bitmaps are allocated in 16-byte units
  const uint4 ones = make_uint4(~0u, ~0u, ~0u, ~0u);
  for (uint64_t i = tid; i < words / 4; i += nth) bm4[i] = ones;
}

// L2 cache policies (PTX createpolicy): strips stream the base table once per
// query, which would push the query's bitmap -- the target of their atomics --
// out of L2.  Table loads are marked evict-first and the atomics evict-last.
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint32_t ld_hint_u32(const uint32_t *a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ uint64_t ld_hint_u64(const uint64_t *a, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.nc.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void red_and_hint(uint32_t *a, uint32_t v, uint64_t pol) {
  asm volatile("red.global.and.L2::cache_hint.b32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}

// Clear index k (query-relative) of class c in a merged query's bitmap: tile
// k >> logL, in-tile index kk, word kk mod W of that class, bit kk div W.
__device__ __forceinline__ void strike_merged(uint32_t *gq, uint64_t k, uint32_t c, uint32_t logL, uint32_t logW,
                                              uint64_t pol) {
  const uint64_t t = k >> logL;
  const uint32_t kk = (uint32_t)k & ((1u << logL) - 1u);
  const uint32_t W = 1u << logW;
  red_and_hint(gq + t * 2ull * W + (uint64_t)c * W + (kk & (W - 1u)), rotl32(0xFFFFFFFEu, kk >> logW), pol);
}

// Count / checksum a finished tile held in s1 / s5 (fix-ups applied), write
// its list bitmap, and add to its query's accumulators.
template <int BLOCK>
__device__ __forceinline__ void emit_tile(const BatchArena &a, const BatchQuery &qd, uint32_t q, uint32_t t,
                                          const uint32_t *s1, const uint32_t *s5, uint32_t W, uint32_t logW,
                                          uint64_t K0, uint64_t *red) {
  const bool list = (qd.flags & kQueryList) != 0;
  uint2 *bm = list ? a.list_bm + qd.bitmap_off + (uint64_t)t * W : nullptr;
  // 32-bit per-thread sums (as in the range kernel): class counts, the
  // word-weighted count and the bit-position sum; the 64-bit checksum once
  uint32_t c1 = 0, c5 = 0, sw = 0;
  BitPlanes planes;  // the bit-position sum, four word pairs at a time
  auto pair = [&](uint32_t w, uint32_t x, uint32_t y) {
    if (list) bm[w] = make_uint2(x, y);
    const uint32_t cx = __popc(x), cy = __popc(y);
    c1 += cx;
    c5 += cy;
    sw += w * (cx + cy);
  };
  uint32_t w = threadIdx.x;
  for (; w + 3 * BLOCK < W; w += 4 * BLOCK) {
    const uint32_t x0 = s1[w], y0 = s5[w], x1 = s1[w + BLOCK], y1 = s5[w + BLOCK];
    const uint32_t x2 = s1[w + 2 * BLOCK], y2 = s5[w + 2 * BLOCK], x3 = s1[w + 3 * BLOCK], y3 = s5[w + 3 * BLOCK];
    pair(w, x0, y0);
    pair(w + BLOCK, x1, y1);
    pair(w + 2 * BLOCK, x2, y2);
    pair(w + 3 * BLOCK, x3, y3);
    planes.add8(x0, y0, x1, y1, x2, y2, x3, y3);
  }
  for (; w < W; w += BLOCK) {
    const uint32_t x = s1[w], y = s5[w];
    pair(w, x, y);
    planes.add1(x);
    planes.add1(y);
  }
  const uint32_t bs = planes.index_sum();
  uint64_t cnt = (uint64_t)c1 + c5, unused = 0;
  uint64_t sum = (uint64_t)c1 * (6 * K0 + 1) + (uint64_t)c5 * (6 * K0 + 5) + 6ull * sw + 6ull * W * bs;
  block_sum3<BLOCK>(cnt, sum, unused, red);
  if (threadIdx.x == 0) {
    if (K0 == 0) {  // 2 and 3 are outside the residue arrays (Section 2.1)
      const uint64_t e2 = (qd.lo <= 2 && 2 < qd.hi), e3 = (qd.lo <= 3 && 3 < qd.hi);
      cnt += e2 + e3;
      sum += 2 * e2 + 3 * e3;
    }
    if (cnt) {
      atomicAdd(a.acc + 2 * q, (unsigned long long)cnt);
      atomicAdd(a.acc + 2 * q + 1, (unsigned long long)sum);
    }
    if (list) a.tile_counts[qd.ltile0 + t] = (uint32_t)cnt;
  }
}

// The persistent sieve kernel: every CTA takes items (in the plan's cost
// order) from the atomic counter until none are left.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, (1024 / BLOCK > 0 ? 1024 / BLOCK : 1)) batch_sieve_kernel(const BatchArena a) {
  constexpr int NWARPS = BLOCK / 32;
  extern __shared__ uint32_t smem[];
  __shared__ uint32_t sh_idx, sh_next, sh_np, sh_allsq;
  __shared__ uint64_t red[3 * NWARPS];
  const char *plan = (const char *)a.plan;
  const BatchHeader *hdr = (const BatchHeader *)plan;
  const uint32_t nitems = hdr->nitems;
  const int npat = (int)hdr->npat;
  const BatchQuery *queries = (const BatchQuery *)(plan + hdr->off_queries);
  const BatchItem *items = (const BatchItem *)(plan + hdr->off_items);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint2 *starts = (uint2 *)(smem + 2 * a.Wmax);

  for (;;) {
    if (threadIdx.x == 0) {
      const bool yield = 2 * blockIdx.x >= gridDim.x &&
                         *(volatile const uint32_t *)&a.state->yield_batch == hdr->batch_id;
      sh_idx = yield ? nitems : atomicAdd(&a.state->next_item, 1u);
    }
    __syncthreads();
    const uint32_t idx = sh_idx;
    if (idx >= nitems) break;
    const BatchItem it = items[idx];
    const BatchQuery &qd = queries[it.q];
    const uint32_t logL = qd.logL, logW = logL - 5, W = 1u << logW, L = 1u << logL;
    const bool merged = (qd.flags & kQueryMerged) != 0;

    if (it.t == kStrip) {
      // large primes over the whole query: one start computation per prime
      // for the query base, then every hit up to the query's end
      const uint64_t Bq = 6 * qd.k_begin;
      const uint64_t span = qd.k_end - qd.k_begin;
      uint32_t *gq = a.slot_bm + qd.slot_base;
      const uint64_t stream = l2_policy_evict_first(), keep = l2_policy_evict_last();
      // the next prime's entries are loaded before the current prime is
      // walked, so that their latency overlaps its atomics
      uint32_t i = it.i0 + threadIdx.x;
      uint32_t Pn = 0;
      uint64_t mn = 0;
      if (i < it.i1) {
        Pn = ld_hint_u32(a.primes + i, stream);
        mn = ld_hint_u64(a.magic + i, stream);
      }
      for (; i < it.i1; i += BLOCK) {
        const uint32_t P = Pn;
        const uint64_t m = mn;
        if (i + BLOCK < it.i1) {
          Pn = ld_hint_u32(a.primes + i + BLOCK, stream);
          mn = ld_hint_u64(a.magic + i + BLOCK, stream);
        }
        uint64_t k1, k5;
        if ((uint64_t)P * P <= Bq && P < 0x80000000u) {  // the inverse-of-6 start (= Table 1's)
          uint32_t i1, i5;
          starts_from_inverse(qd.k_begin, P, m, inverse6_constants(P), i1, i5);
          k1 = i1;
          k5 = i5;
        } else {
          tile_starts(Bq, P, m, k1, k5);
        }
        for (uint64_t k = k1; k < span; k += P) strike_merged(gq, k, 0, logL, logW, keep);
        for (uint64_t k = k5; k < span; k += P) strike_merged(gq, k, 1, logL, logW, keep);
      }
      __syncthreads();
      continue;
    }

    // tile item
    const uint64_t K0 = qd.k_begin + (uint64_t)it.t * L;
    const uint64_t left = qd.k_end - K0;
    TileGeom tg;
    tg.W = W;
    tg.logW = logW;
    tg.len = left < L ? (uint32_t)left : L;
    const uint64_t B = 6 * K0;
    const uint64_t tile_end = B + 6ull * tg.len;
    const uint64_t vend = tile_end < qd.hi ? tile_end : qd.hi;
    uint32_t *s1 = smem, *s5 = smem + W;
    if (warp == 0) {
      // primes this tile needs: P <= isqrt(vend - 1), within the item's range
      const uint64_t s = vend >= 2 ? isqrt_dev(vend - 1) : 0;
      const uint32_t np = warp_count_le(a.primes, it.i1, s);
      const uint32_t npt = np > it.i0 ? np : it.i0;
      // every needed prime is below sqrt(B) (and 2^31): no P^2 clamp in this tile
      const uint64_t Plast = npt ? __ldg(a.primes + npt - 1) : 0;
      if (lane == 0) {
        sh_np = npt;
        sh_allsq = Plast * Plast <= B && Plast < 0x80000000ull;
        sh_next = it.i0;
      }
    }
    const PatternSetDev *ps = a.psets + logW;
    presieve_copy<BLOCK>(s1, s5, tg, K0, ps->d, ps->pd, npat);
    const uint32_t split = qd.i_split < it.i1 ? qd.i_split : it.i1;
    warp_band_starts<BLOCK>(starts, B, tg.len, a.primes, a.magic, a.cinv, it.i0, split);
    __syncthreads();
    strike_primes<BLOCK, true>(s1, s5, B, tg, a.primes, a.magic, a.cinv, starts, it.i0, split, sh_np,
                               sh_allsq != 0, &sh_next, B / 6);  // B / 6 rather than K0: measured faster here
    __syncthreads();
    if (merged) {
      // AND the shared-memory result into the query's bitmap in global memory
      uint32_t *g1 = a.slot_bm + qd.slot_base + (uint64_t)it.t * 2 * W, *g5 = g1 + W;
      const uint64_t keep = l2_policy_evict_last();
      for (uint32_t w = threadIdx.x; w < W; w += BLOCK) {
        const uint32_t x = s1[w], y = s5[w];
        if (x != 0xFFFFFFFFu) red_and_hint(g1 + w, x, keep);
        if (y != 0xFFFFFFFFu) red_and_hint(g5 + w, y, keep);
      }
    } else {
      fixup_tile<BLOCK>(s1, s5, tg, K0, valid_range(qd.lo, qd.hi, B, tg.len), npat);  // ends with a barrier if needed
      emit_tile<BLOCK>(a, qd, it.q, it.t, s1, s5, W, logW, K0, red);
    }
    __syncthreads();  // shared memory and sh_idx are reused by the next item
  }
}

// Merged tiles, after every item of the batch: load the tile from global
// memory, apply the fix-ups, count and emit it.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_finish_kernel(const BatchArena a) {
  constexpr int NWARPS = BLOCK / 32;
  extern __shared__ uint32_t smem[];
  __shared__ uint64_t red[3 * NWARPS];
  const char *plan = (const char *)a.plan;
  const BatchHeader *hdr = (const BatchHeader *)plan;
  const uint32_t nmerged = hdr->nmerged;
  const int npat = (int)hdr->npat;
  const BatchQuery *queries = (const BatchQuery *)(plan + hdr->off_queries);
  const uint2 *mtiles = (const uint2 *)(plan + hdr->off_mtiles);
  for (uint32_t j = blockIdx.x; j < nmerged; j += gridDim.x) {
    const uint2 qt = mtiles[j];
    const BatchQuery &qd = queries[qt.x];
    const uint32_t logL = qd.logL, logW = logL - 5, W = 1u << logW, L = 1u << logL;
    const uint64_t K0 = qd.k_begin + (uint64_t)qt.y * L;
    const uint64_t left = qd.k_end - K0;
    TileGeom tg;
    tg.W = W;
    tg.logW = logW;
    tg.len = left < L ? (uint32_t)left : L;
    uint32_t *s1 = smem, *s5 = smem + W;
    const uint32_t *g1 = a.slot_bm + qd.slot_base + (uint64_t)qt.y * 2 * W, *g5 = g1 + W;
    for (uint32_t w = threadIdx.x; w < W; w += BLOCK) {
      s1[w] = g1[w];
      s5[w] = g5[w];
    }
    __syncthreads();
    fixup_tile<BLOCK>(s1, s5, tg, K0, valid_range(qd.lo, qd.hi, 6 * K0, tg.len), npat);  // ends with a barrier if needed
    emit_tile<BLOCK>(a, qd, qt.x, qt.y, s1, s5, W, logW, K0, red);
    __syncthreads();
  }
}

// List offsets: exclusive scan of the list tiles' counts (one CTA), then the
// CSR offsets of every query (offsets[q] = start of query q's first list
// tile; offsets[nq] = total) and the capacity checks.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_scan_kernel(const BatchArena a) {
  constexpr int NWARPS = BLOCK / 32;
  __shared__ uint64_t warp_tot[NWARPS];
  __shared__ uint64_t carry;
  const char *plan = (const char *)a.plan;
  const BatchHeader *hdr = (const BatchHeader *)plan;
  const uint32_t n = hdr->nltiles, nq = hdr->nq;
  const uint32_t *ltile0 = (const uint32_t *)(plan + hdr->off_ltile0);  // nq + 1 entries
  const BatchQuery *queries = (const BatchQuery *)(plan + hdr->off_queries);
  const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += BLOCK) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t x = i < n ? a.tile_counts[i] : 0;
    uint64_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t y = __shfl_up_sync(kFullMask, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      uint64_t wt = lane < NWARPS ? warp_tot[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(kFullMask, wt, o);
        if (lane >= (uint32_t)o) wt += y;
      }
      if (lane < NWARPS) warp_tot[lane] = wt;
    }
    __syncthreads();
    const uint64_t before = carry + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (i < n) a.tile_off[i] = before + incl - x;
    __syncthreads();
    if (threadIdx.x == BLOCK - 1) carry = before + incl;
    __syncthreads();
  }
  if (threadIdx.x == 0) a.tile_off[n] = carry;
  __syncthreads();
  for (uint32_t q = threadIdx.x; q <= nq; q += BLOCK) {
    const uint64_t o = a.tile_off[ltile0[q]];
    a.offsets[q] = o;
    if (q < nq && hdr->fixed_out && (queries[q].flags & kQueryList)) {
      const uint64_t c = a.tile_off[ltile0[q + 1]] - o;
      if (c > queries[q].out_cap) atomicOr(&a.state->status, 2u);
    }
  }
  if (threadIdx.x == 0 && !hdr->fixed_out && carry > hdr->cap) atomicOr(&a.state->status, 1u);
}

// Write every list tile's primes in value order: to offsets[q] + (tile offset
// within the query) in CSR mode, or to the query's out_base in fixed mode.
// Whether the list compaction stages a tile's bitmap in shared memory (Wmax
// pairs before the emission staging) or reads it from global memory.
constexpr bool kBatchCompactSbuf = false;
// batch tiles are small (few chunks per warp): the shallow staging row keeps
// three CTAs per SM, measured faster than deeper rows
constexpr uint32_t kBatchStageRow = 64;

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) batch_compact_kernel(const BatchArena a) {
  constexpr int NWARPS = BLOCK / 32;
  __shared__ uint32_t warp_cnt[NWARPS * 32];
  extern __shared__ __align__(16) uint2 sbuf[];  // [one tile's bitmap (up to Wmax pairs)] [emission staging]
  uint16_t *stage = (uint16_t *)(sbuf + (kBatchCompactSbuf ? a.Wmax : 0));
  const char *plan = (const char *)a.plan;
  const BatchHeader *hdr = (const BatchHeader *)plan;
  const uint32_t n = hdr->nltiles;
  if (!hdr->fixed_out && a.tile_off[n] > hdr->cap) return;  // reported by the host
  const BatchQuery *queries = (const BatchQuery *)(plan + hdr->off_queries);
  const uint2 *ltiles = (const uint2 *)(plan + hdr->off_ltiles);
  uint64_t *out = hdr->values;
  for (uint32_t lt = blockIdx.x; lt < n; lt += gridDim.x) {
    const uint2 qt = ltiles[lt];
    const BatchQuery &qd = queries[qt.x];
    const uint32_t logL = qd.logL, logW = logL - 5, W = 1u << logW, L = 1u << logL;
    uint64_t off = a.tile_off[lt];
    if (hdr->fixed_out) {
      const uint64_t q0 = a.tile_off[qd.ltile0];
      const uint64_t qn = a.tile_off[qd.ltile0 + qd.ntiles] - q0;
      if (qn > qd.out_cap) continue;  // flagged by the scan
      off = qd.out_base + (off - q0);
    }
    const uint64_t K0 = qd.k_begin + (uint64_t)qt.y * L;
    if (K0 == 0) {  // 2 and 3 first
      const uint32_t e2 = (qd.lo <= 2 && 2 < qd.hi), e3 = (qd.lo <= 3 && 3 < qd.hi);
      if (threadIdx.x == 0) {
        uint64_t o = off;
        if (e2) out[o++] = 2;
        if (e3) out[o++] = 3;
      }
      off += e2 + e3;
    }
    compact_tile<BLOCK, uint64_t, kBatchCompactSbuf, kBatchStageRow>(a.list_bm + qd.bitmap_off + (uint64_t)qt.y * W, logW, K0, off,
                                                     out, warp_cnt, sbuf, stage);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- host: runner

void destroy_batch_runner(BatchRunner *r) {
  if (!r) return;
  if (r->exec) cudaGraphExecDestroy(r->exec);
  if (r->graph) cudaGraphDestroy(r->graph);
  cudaFree(r->d_plan);
  cudaFree(r->d_state);
  cudaFree(r->d_acc);
  cudaFree(r->d_slot_bm);
  cudaFree(r->d_tile_counts);
  cudaFree(r->d_tile_off);
  cudaFree(r->d_offsets);
  cudaFree(r->d_list_bm);
  if (r->h_plan) cudaFreeHost(r->h_plan);
  if (r->h_back) cudaFreeHost(r->h_back);
  delete r;
}

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

uint32_t log2_floor(uint64_t x) {
  uint32_t r = 0;
  while (x >>= 1) r++;
  return r;
}

template <typename T>
int grow_device(T **p, size_t *cap, size_t need, bool *changed) {
  if (need <= *cap && *p) return SIEVE_OK;
  size_t n = std::max<size_t>(need + need / 2, 256);
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  SIEVE_CUDA_TRY(cudaMalloc((void **)p, n * sizeof(T)));
  *cap = n;
  *changed = true;
  return SIEVE_OK;
}

BatchArena arena_of(const BatchRunner &r) {
  BatchArena a;
  a.plan = r.d_plan;
  a.state = r.d_state;
  a.acc = r.d_acc;
  a.slot_bm = r.d_slot_bm;
  a.tile_counts = r.d_tile_counts;
  a.tile_off = r.d_tile_off;
  a.offsets = r.d_offsets;
  a.list_bm = r.d_list_bm;
  a.primes = r.ctx->table.primes;
  a.magic = r.ctx->table.magic;
  a.cinv = r.ctx->table.cinv;
  a.psets = r.ctx->d_psets;
  a.Wmax = r.Wmax;
  a.band_max = r.band_max;
  return a;
}

void *sieve_kernel_fn(int threads) {
  switch (threads) {
    case 256: return (void *)batch_sieve_kernel<256>;
    case 512: return (void *)batch_sieve_kernel<512>;
    default: return (void *)batch_sieve_kernel<1024>;
  }
}

constexpr int kFinishThreads = 256;
constexpr int kCompactThreads = 512;

static size_t batch_compact_smem(uint32_t Wmax) {
  return (kBatchCompactSbuf ? (size_t)Wmax * sizeof(uint2) : 0) +
         compact_stage_bytes(kCompactThreads, kBatchStageRow);
}
constexpr int kScanThreads = 1024;

// Launch shape for the context's current options: threads, largest tile,
// warp-band size and the persistent grid (every resident CTA slot).
int configure(BatchRunner &r) {
  sieve_ctx *ctx = r.ctx;
  const uint32_t Lmax = ctx->opt.batch_tile_bits ? ctx->opt.batch_tile_bits : ctx->opt.tile_bits;
  const int threads = (int)ctx->opt.block_threads;
  const uint32_t i_first = first_struck_prime_index((int)ctx->opt.presieve_groups);
  const uint64_t gmax = Lmax / (32ull * std::max<uint32_t>(1u, ctx->opt.group_hits));
  uint32_t i_split = host_prime_count_le_table(ctx->table, gmax);
  const uint32_t band = i_split > i_first ? i_split - i_first : 0;
  const uint32_t logLmax = log2_floor(Lmax);
  const size_t smem = (size_t)(Lmax / 32) * 2 * sizeof(uint32_t) + (size_t)band * sizeof(uint2);
  if (smem > (size_t)ctx->smem_optin) {
    set_error("batch tile of %u bits needs %zu bytes of shared memory", Lmax, smem);
    return SIEVE_ERR_INVALID;
  }
  const size_t fsmem = (size_t)(Lmax / 32) * 2 * sizeof(uint32_t);
  if (r.exec && threads == r.threads && logLmax == r.logLmax && band == r.band_max &&
      r.table_epoch == ctx->table_epoch)
    return SIEVE_OK;
  void *fn = sieve_kernel_fn(threads);
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->smem_optin));
  SIEVE_CUDA_TRY(cudaFuncSetAttribute((void *)batch_finish_kernel<kFinishThreads>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->smem_optin));
  SIEVE_CUDA_TRY(cudaFuncSetAttribute((void *)batch_compact_kernel<kCompactThreads>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, ctx->smem_optin));
  int per_sm = 0, fper_sm = 0;
  SIEVE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  SIEVE_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &fper_sm, (const void *)batch_finish_kernel<kFinishThreads>, kFinishThreads, fsmem));
  if (per_sm < 1 || fper_sm < 1) {
    set_error("batch kernels do not fit on an SM with %zu bytes of shared memory", smem);
    return SIEVE_ERR_INVALID;
  }
  if (ctx->opt.ctas_per_sm && (int)ctx->opt.ctas_per_sm < per_sm) per_sm = (int)ctx->opt.ctas_per_sm;
  r.threads = threads;
  r.grid = ctx->num_sms * per_sm;
  r.finish_grid = ctx->num_sms * fper_sm;
  r.smem = smem;
  r.finish_smem = fsmem;
  r.logLmax = logLmax;
  r.Wmax = Lmax / 32;
  r.band_max = band;
  // the graph holds the old shape
  if (r.exec) {
    cudaGraphExecDestroy(r.exec);
    r.exec = nullptr;
  }
  if (r.graph) {
    cudaGraphDestroy(r.graph);
    r.graph = nullptr;
  }
  return SIEVE_OK;
}

// The batch as one CUDA graph: plan upload -> init -> sieve -> finish -> scan
// -> compact.  Only the upload size changes between launches (set on the
// executable graph before each launch); every kernel reads its sizes from the
// uploaded plan.
int build_graph(BatchRunner &r) {
  if (r.exec) return SIEVE_OK;
  cudaGraph_t g = nullptr;
  SIEVE_CUDA_TRY(cudaGraphCreate(&g, 0));
  r.graph = g;
  BatchArena a = arena_of(r);
  void *args[] = {&a};
  cudaGraphNode_t n_copy, n_init, n_sieve, n_finish, n_scan, n_compact;
  SIEVE_CUDA_TRY(cudaGraphAddMemcpyNode1D(&n_copy, g, nullptr, 0, r.d_plan, r.h_plan, sizeof(BatchHeader),
                                          cudaMemcpyHostToDevice));
  cudaKernelNodeParams kp;
  memset(&kp, 0, sizeof(kp));
  kp.kernelParams = args;
  kp.func = (void *)batch_init_kernel;
  kp.gridDim = dim3(r.ctx->num_sms * 4);
  kp.blockDim = dim3(256);
  SIEVE_CUDA_TRY(cudaGraphAddKernelNode(&n_init, g, &n_copy, 1, &kp));
  kp.func = sieve_kernel_fn(r.threads);
  kp.gridDim = dim3(r.grid);
  kp.blockDim = dim3(r.threads);
  kp.sharedMemBytes = (unsigned)r.smem;
  SIEVE_CUDA_TRY(cudaGraphAddKernelNode(&n_sieve, g, &n_init, 1, &kp));
  kp.func = (void *)batch_finish_kernel<kFinishThreads>;
  kp.gridDim = dim3(r.finish_grid);
  kp.blockDim = dim3(kFinishThreads);
  kp.sharedMemBytes = (unsigned)r.finish_smem;
  SIEVE_CUDA_TRY(cudaGraphAddKernelNode(&n_finish, g, &n_sieve, 1, &kp));
  kp.func = (void *)batch_scan_kernel<kScanThreads>;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kScanThreads);
  kp.sharedMemBytes = 0;
  SIEVE_CUDA_TRY(cudaGraphAddKernelNode(&n_scan, g, &n_finish, 1, &kp));
  kp.func = (void *)batch_compact_kernel<kCompactThreads>;
  kp.gridDim = dim3(r.ctx->num_sms * 3);
  kp.blockDim = dim3(kCompactThreads);
  kp.sharedMemBytes = (unsigned)batch_compact_smem(r.Wmax);
  SIEVE_CUDA_TRY(cudaGraphAddKernelNode(&n_compact, g, &n_scan, 1, &kp));
  SIEVE_CUDA_TRY(cudaGraphInstantiate(&r.exec, g, 0));
  r.n_copy = n_copy;
  r.table_epoch = r.ctx->table_epoch;
  return SIEVE_OK;
}

}  // namespace

// Kernels per graph launch (for the context's launch counter).
constexpr uint64_t kBatchGraphKernels = 5;

// ---------------------------------------------------------------- host: planner

namespace {

// ln x for x >= 1, to about 1e-5 absolute, for the cost model: x = 2^e m with
// m in [1, 2), and ln m = 2 atanh(t), t = (m - 1) / (m + 1) <= 1/3, summed to
// the t^7 term.  (The planner evaluates it tens of times per work item, in
// the binary searches that size the items; the library log was a large part
// of planning a batch.)
double fast_ln(double x) {
  uint64_t b;
  memcpy(&b, &x, sizeof(b));
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  b = (b & 0x000FFFFFFFFFFFFFull) | 0x3FF0000000000000ull;
  double m;
  memcpy(&m, &b, sizeof(m));
  const double t = (m - 1.0) / (m + 1.0), t2 = t * t;
  return e * 0.6931471805599453 + 2.0 * t * (1.0 + t2 * (1.0 / 3.0 + t2 * (1.0 / 5.0 + t2 * (1.0 / 7.0))));
}

// ln ln x for the strike-count estimate: the class-1 and class-5 multiples of
// the primes in (a, b] among n indices number about 2 n (ln ln b - ln ln a)
// (Mertens' second theorem).
double lnln(double x) { return fast_ln(fast_ln(std::max(x, 23.0))); }

// Relative cost units of the work an item does (one unit ~ one strike in
// shared memory).  An atomic AND in global memory is priced at many strikes:
// the merge bitmaps of a batch rarely stay in L2, so each costs a DRAM
// read-modify-write of a 32-byte sector.
constexpr double kCostItem = 4000.0;   // fixed per item: barriers, set-up
constexpr double kCostPrime = 10.0;    // one Table 1 evaluation
constexpr double kCostWord = 6.0;      // presieve copy + count of one word pair
constexpr double kCostGlobal = 40.0;   // one atomic AND in global memory (L2-resident bitmap);
                                       // 75 measured slower on the batch and serving mixes
constexpr double kL2Bitmap = 48e6;     // a merged query's bitmap above this many bytes
                                       // spills from L2: its atomics cost 4x
constexpr uint32_t kMinChunk = 256;    // fewest primes in a split piece of a tile

struct QueryPlanInfo {
  uint32_t np = 0, i_mid = 0;
  bool strips = false;  // primes [i_mid, np) go to strip items
  double tile_cost = 0.0;
  double gcost = 0.0;   // cost of one global atomic for this query's bitmap
  double total = 0.0;   // all items of the query
};

// Cost of striking primes [a, b) into a tile of L indices per class.
double tile_primes_cost(const uint32_t *P, uint32_t a, uint32_t b, uint32_t L) {
  if (b <= a) return 0.0;
  return kCostPrime * (b - a) + 2.0 * (double)L * (lnln((double)P[b - 1]) - lnln((double)P[a]));
}

// Largest n in [1, cap] with cost(n) <= target (1 if even cost(1) is above);
// cost must grow with n.
template <typename F>
uint32_t largest_within(uint32_t cap, double target, F cost) {
  if (cost(cap) <= target) return cap;
  uint32_t lo = 1, hi = cap;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo + 1) / 2;
    if (cost(mid) <= target)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

}  // namespace

// Plan a batch into r's pinned host buffer.  values / cap describe the list
// output for CSR mode (fixed_out = 0); in fixed mode out_base / out_cap give
// every query its own place.  Returns SIEVE_OK or an error for the first bad
// query.
int batch_plan(BatchRunner &r, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode, size_t nq,
               uint64_t *values, uint64_t cap, int fixed_out, const uint64_t *out_base, const uint64_t *out_cap) {
  sieve_ctx *ctx = r.ctx;
  const DeviceTable &table = ctx->table;
  if (nq >= 0x7FFFFFFFull) {
    set_error("too many queries in one batch");
    return SIEVE_ERR_INVALID;
  }
  const uint32_t logLmax = r.logLmax;
  const uint32_t gh = std::max<uint32_t>(1u, ctx->opt.group_hits);
  const uint32_t chunk = std::max<uint32_t>(1024u, ctx->opt.chunk_primes);
  const uint32_t i_first = first_struck_prime_index((int)ctx->opt.presieve_groups);
  const uint32_t *P = table.host_primes;
  r.q.assign(nq, BatchQuery{});
  r.items.clear();
  r.cost.clear();
  r.mtiles.clear();
  r.ltiles.clear();
  r.ltile0.assign(nq + 1, 0);
  r.slot_words = 0;
  r.list_words = 0;
  r.used_logW = 0;
  std::vector<QueryPlanInfo> info(nq);
  double total_cost = 0.0;
  uint32_t nlt = 0;
  for (size_t i = 0; i < nq; i++) {
    BatchQuery &bq = r.q[i];
    if (lo[i] > hi[i]) {
      set_error("query %zu: lo (%llu) > hi (%llu)", i, (unsigned long long)lo[i], (unsigned long long)hi[i]);
      return SIEVE_ERR_INVALID;
    }
    if (mode[i] > 1) {
      set_error("query %zu: mode must be SIEVE_COUNT or SIEVE_LIST", i);
      return SIEVE_ERR_INVALID;
    }
    if (hi[i] > (1ull << 63)) {
      set_error("query %zu: hi must be <= 2^63", i);
      return SIEVE_ERR_RANGE;
    }
    bq.lo = lo[i];
    bq.hi = hi[i];
    bq.flags = mode[i] == SIEVE_LIST ? kQueryList : 0u;
    bq.ltile0 = nlt;
    r.ltile0[i] = nlt;
    if (fixed_out) {
      bq.out_base = out_base[i];
      bq.out_cap = out_cap[i];
    }
    bq.logL = 10;
    if (lo[i] == hi[i]) continue;  // empty: no tiles
    const uint64_t s = isqrt_u64(hi[i] - 1);
    if (s > table.limit) {
      set_error("query %zu: isqrt(hi - 1) = %llu exceeds the base table limit %llu", i, (unsigned long long)s,
                (unsigned long long)table.limit);
      return SIEVE_ERR_RANGE;
    }
    bq.k_begin = lo[i] / 6;
    bq.k_end = (hi[i] + 4) / 6;
    const uint64_t span = bq.k_end > bq.k_begin ? bq.k_end - bq.k_begin : 0;
    if (span == 0) continue;
    uint32_t logL = 10;
    while (logL < logLmax && (1ull << logL) < span) logL++;
    const uint32_t L = 1u << logL;
    const uint64_t ntiles = (span + L - 1) >> logL;
    if (ntiles > 0x7FFFFFFFull) {
      set_error("query %zu needs too many tiles", i);
      return SIEVE_ERR_INVALID;
    }
    bq.logL = logL;
    bq.ntiles = (uint32_t)ntiles;
    r.used_logW |= 1u << (logL - 5);
    const uint32_t np = host_prime_count_le_table(table, s);
    bq.np = np;
    uint32_t i_split = host_prime_count_le_table(table, L / (32ull * gh));
    if (i_split < i_first) i_split = i_first;
    bq.i_split = i_split;
    // Primes above the tile length hit a tile at most twice.  Strips locate
    // them once per query and clear each hit with a global atomic; tiles
    // locate them once per tile.  A prime p costs ntiles evaluations on the
    // tiles and one evaluation plus about 2 span / p atomics as a strip, so
    // the tiles keep every prime below p* = gcost 2 span / (kCostPrime
    // (ntiles - 1)) (about 8 L), and strips take the primes above it when
    // they cost less in total.
    QueryPlanInfo &qi = info[i];
    qi.gcost = (double)span / 4.0 > kL2Bitmap ? 4.0 * kCostGlobal : kCostGlobal;
    const double pstar =
        ntiles > 1 ? qi.gcost * 2.0 * (double)span / (kCostPrime * (double)(ntiles - 1)) : (double)L;
    const uint64_t p_split = std::max<uint64_t>(L, (uint64_t)std::min(pstar, (double)s));
    uint32_t i_mid = host_prime_count_le_table(table, p_split);
    if (i_mid < i_first) i_mid = i_first;
    qi.np = np;
    qi.i_mid = i_mid;
    const double pm = (double)P[std::min(i_mid, table.nprimes - 1)];
    const double hits = np > i_mid ? 2.0 * (double)span * (lnln((double)P[np - 1]) - lnln(pm)) : 0.0;
    const double large = np > i_mid ? (double)(np - i_mid) : 0.0;
    qi.strips = ntiles >= 2 && span < (1ull << 31) && np > i_mid &&
                kCostPrime * large + qi.gcost * hits < kCostPrime * large * (double)ntiles;
    const uint32_t t_end = qi.strips ? i_mid : std::max(np, i_first);
    qi.tile_cost = kCostItem + kCostWord * (L / 32) + tile_primes_cost(P, i_first, t_end, L);
    total_cost += (double)ntiles * qi.tile_cost;
    if (qi.strips) total_cost += kCostPrime * large + qi.gcost * hits;
    if (bq.flags & kQueryList) {
      bq.bitmap_off = r.list_words;
      r.list_words += ntiles * (uint64_t)(L / 32);
      nlt += (uint32_t)ntiles;
    }
  }
  r.ltile0[nq] = nlt;
  // target cost per item: a few items per CTA slot so that the cost-ordered
  // queue ends evenly
  const double target = std::max(total_cost / ((double)r.grid * 4.0), 2.0e5);

  for (size_t i = 0; i < nq; i++) {
    BatchQuery &bq = r.q[i];
    if (bq.ntiles == 0) continue;
    const QueryPlanInfo &qi = info[i];
    const uint32_t L = 1u << bq.logL, W = L / 32;
    const uint64_t span = bq.k_end - bq.k_begin;
    const uint32_t t_end = qi.strips ? qi.i_mid : std::max(qi.np, i_first);
    // a tile too costly for one item is split by primes into pieces that
    // different CTAs sieve in shared memory and AND into global memory
    const bool split = qi.tile_cost > target && t_end - i_first >= 2 * kMinChunk;
    if (qi.strips || split) {
      bq.flags |= kQueryMerged;
      bq.slot_base = r.slot_words;
      r.slot_words += (uint64_t)bq.ntiles * 2ull * W;
    }
    const double fixed = kCostItem + kCostWord * W;
    for (uint32_t t = 0; t < bq.ntiles; t++) {
      if (!split) {
        r.items.push_back(BatchItem{(uint32_t)i, t, i_first, t_end});
        r.cost.push_back((float)qi.tile_cost);
      } else {
        uint32_t a = i_first;
        while (a < t_end) {
          const uint32_t cap = std::min<uint32_t>(chunk, t_end - a);
          uint32_t n = largest_within(cap, target, [&](uint32_t k) { return fixed + tile_primes_cost(P, a, a + k, L); });
          if (n < kMinChunk) n = std::min<uint32_t>(kMinChunk, t_end - a);
          r.items.push_back(BatchItem{(uint32_t)i, t, a, a + n});
          r.cost.push_back((float)(fixed + tile_primes_cost(P, a, a + n, L)));
          a += n;
        }
      }
      if (bq.flags & kQueryMerged) r.mtiles.push_back(make_uint2((uint32_t)i, t));
      if (bq.flags & kQueryList) r.ltiles.push_back(make_uint2((uint32_t)i, t));
    }
    if (qi.strips) {
      // strips of primes [i_mid, np): at most `chunk` primes and about
      // `target` cost each
      uint32_t a = qi.i_mid;
      while (a < qi.np) {
        const double la = lnln((double)P[a]);
        auto strip_cost = [&](uint32_t n) {
          return kCostItem + kCostPrime * n + qi.gcost * 2.0 * (double)span * (lnln((double)P[a + n - 1]) - la);
        };
        const uint32_t n = largest_within(std::min<uint32_t>(chunk, qi.np - a), target, strip_cost);
        r.items.push_back(BatchItem{(uint32_t)i, kStrip, a, a + n});
        r.cost.push_back((float)strip_cost(n));
        a += n;
      }
    }
  }
  if (r.items.size() > 0xFFFFFFF0ull) {
    set_error("batch needs too many work items");
    return SIEVE_ERR_INVALID;
  }

  // Order: first the merged queries, one query's items after another
  // (largest query first), so that all CTAs strike one query's bitmap in
  // global memory at a time and it stays in L2; then the single-tile items,
  // largest first, so that the queue drains evenly (longest processing time
  // first).  A counting sort on log2 buckets of the cost, stable, so a
  // query's items stay together.
  const size_t ni = r.items.size();
  for (size_t j = 0; j < ni; j++) info[r.items[j].q].total += r.cost[j];
  constexpr int kBuckets = 128;
  size_t bucket_n[2 * kBuckets + 1] = {0};
  std::vector<uint8_t> bk(ni);
  for (size_t j = 0; j < ni; j++) {
    const uint32_t qj = r.items[j].q;
    const bool merged = (r.q[qj].flags & kQueryMerged) != 0;
    const float key = merged ? (float)info[qj].total : r.cost[j];
    int b = (int)(4.0f * std::log2(std::max(key, 1.0f)));
    b = std::min(std::max(b, 0), kBuckets - 1);
    bk[j] = (uint8_t)((merged ? 0 : kBuckets) + kBuckets - 1 - b);
    bucket_n[bk[j] + 1]++;
  }
  for (int b = 0; b < 2 * kBuckets; b++) bucket_n[b + 1] += bucket_n[b];
  r.sorted.resize(ni);
  for (size_t j = 0; j < ni; j++) r.sorted[bucket_n[bk[j]]++] = r.items[j];

  // layout of the plan
  BatchHeader h;
  memset(&h, 0, sizeof(h));
  h.nq = (uint32_t)nq;
  h.nitems = (uint32_t)ni;
  h.nmerged = (uint32_t)r.mtiles.size();
  h.nltiles = nlt;
  h.slot_words = r.slot_words;
  size_t off = align256(sizeof(BatchHeader));
  h.off_queries = off;
  off = align256(off + nq * sizeof(BatchQuery));
  h.off_items = off;
  off = align256(off + ni * sizeof(BatchItem));
  h.off_mtiles = off;
  off = align256(off + r.mtiles.size() * sizeof(uint2));
  h.off_ltiles = off;
  off = align256(off + r.ltiles.size() * sizeof(uint2));
  h.off_ltile0 = off;
  off = align256(off + (nq + 1) * sizeof(uint32_t));
  h.values = values;
  h.cap = cap;
  h.fixed_out = fixed_out ? 1u : 0u;
  h.npat = 1u + ctx->opt.presieve_groups;
  r.batch_id = r.batch_id == 0xFFFFFFFFu ? 1u : r.batch_id + 1;
  h.batch_id = r.batch_id;
  r.plan_bytes = off;
  if (off > r.h_plan_cap) {
    if (r.h_plan) {
      SIEVE_CUDA_TRY(cudaStreamSynchronize(r.stream));  // a graph may still read the old buffer
      cudaFreeHost(r.h_plan);
      r.h_plan = nullptr;
      r.h_plan_cap = 0;
    }
    const size_t n = off + off / 2;
    SIEVE_CUDA_TRY(cudaMallocHost((void **)&r.h_plan, n));
    r.h_plan_cap = n;
    if (r.exec) {  // the graph's copy node points at the old buffer
      cudaGraphExecDestroy(r.exec);
      r.exec = nullptr;
      cudaGraphDestroy(r.graph);
      r.graph = nullptr;
    }
  }
  char *hp = r.h_plan;
  memcpy(hp, &h, sizeof(h));
  if (nq) memcpy(hp + h.off_queries, r.q.data(), nq * sizeof(BatchQuery));
  if (ni) memcpy(hp + h.off_items, r.sorted.data(), ni * sizeof(BatchItem));
  if (!r.mtiles.empty()) memcpy(hp + h.off_mtiles, r.mtiles.data(), r.mtiles.size() * sizeof(uint2));
  if (!r.ltiles.empty()) memcpy(hp + h.off_ltiles, r.ltiles.data(), r.ltiles.size() * sizeof(uint2));
  memcpy(hp + h.off_ltile0, r.ltile0.data(), (nq + 1) * sizeof(uint32_t));
  return SIEVE_OK;
}

// ---------------------------------------------------------------- host: run

// Device buffers for the planned batch (grown as needed; the graph is rebuilt
// when a buffer moves), the pattern sets its tile widths use, and the graph.
int batch_prepare(BatchRunner &r) {
  sieve_ctx *ctx = r.ctx;
  bool changed = false;
  int rc;
  const BatchHeader *h = (const BatchHeader *)r.h_plan;
  if ((rc = grow_device(&r.d_plan, &r.plan_cap, r.plan_bytes, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_acc, &r.acc_cap, 2ull * h->nq + 2, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_offsets, &r.offsets_cap, (size_t)h->nq + 1, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_slot_bm, &r.slot_cap, (size_t)h->slot_words + 4, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_tile_counts, &r.counts_cap, (size_t)h->nltiles + 1, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_tile_off, &r.toff_cap, (size_t)h->nltiles + 1, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_list_bm, &r.list_cap, (size_t)r.list_words + 1, &changed)) != SIEVE_OK) return rc;
  if (!r.d_state) {
    SIEVE_CUDA_TRY(cudaMalloc(&r.d_state, sizeof(BatchState)));
    // yield_batch = 0 (no batch id); complete before any yield request can
    // be written from another stream
    SIEVE_CUDA_TRY(cudaMemsetAsync(r.d_state, 0, sizeof(BatchState), r.stream));
    SIEVE_CUDA_TRY(cudaStreamSynchronize(r.stream));
    changed = true;
  }
  if (!r.h_back) SIEVE_CUDA_TRY(cudaMallocHost((void **)&r.h_back, 4 * sizeof(uint64_t)));
  for (uint32_t lw = 0; lw < 32; lw++)
    if (r.used_logW & (1u << lw))
      if ((rc = ensure_pattern_set_dev(ctx, lw)) != SIEVE_OK) return rc;
  if (!ctx->d_psets && (rc = ensure_pattern_set_dev(ctx, 5)) != SIEVE_OK) return rc;
  if (changed && r.exec) {
    cudaGraphExecDestroy(r.exec);
    r.exec = nullptr;
    cudaGraphDestroy(r.graph);
    r.graph = nullptr;
  }
  return build_graph(r);
}

// Allocate a runner's buffers up front for batches of up to nq queries,
// `items` work items, `slot_words` merge-bitmap words and `list_words` list
// bitmap pairs, so that planning such batches never grows (and so never
// frees, which would synchronise the device) a buffer.
int batch_reserve(BatchRunner &r, size_t nq, size_t items, uint64_t slot_words, uint64_t list_words) {
  bool changed = false;
  int rc;
  const size_t ltiles = (size_t)(list_words / 32) + nq + 1;
  const size_t plan = align256(sizeof(BatchHeader)) + align256(nq * sizeof(BatchQuery)) +
                      align256(items * sizeof(BatchItem)) + 2 * align256(ltiles * sizeof(uint2)) +
                      align256((nq + 1) * sizeof(uint32_t));
  if ((rc = grow_device(&r.d_plan, &r.plan_cap, plan, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_acc, &r.acc_cap, 2 * nq + 2, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_offsets, &r.offsets_cap, nq + 1, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_slot_bm, &r.slot_cap, (size_t)slot_words + 4, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_tile_counts, &r.counts_cap, ltiles, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_tile_off, &r.toff_cap, ltiles, &changed)) != SIEVE_OK) return rc;
  if ((rc = grow_device(&r.d_list_bm, &r.list_cap, (size_t)list_words + 1, &changed)) != SIEVE_OK) return rc;
  if (plan > r.h_plan_cap) {
    if (r.h_plan) cudaFreeHost(r.h_plan);
    r.h_plan = nullptr;
    r.h_plan_cap = 0;
    SIEVE_CUDA_TRY(cudaMallocHost((void **)&r.h_plan, plan));
    r.h_plan_cap = plan;
    changed = true;
  }
  if (changed && r.exec) {
    cudaGraphExecDestroy(r.exec);
    r.exec = nullptr;
    cudaGraphDestroy(r.graph);
    r.graph = nullptr;
  }
  return SIEVE_OK;
}

// Launch the planned batch on r.stream (asynchronous).
int batch_launch(BatchRunner &r) {
  SIEVE_CUDA_TRY(cudaGraphExecMemcpyNodeSetParams1D(r.exec, r.n_copy, r.d_plan, r.h_plan, r.plan_bytes,
                                                    cudaMemcpyHostToDevice));
  SIEVE_CUDA_TRY(cudaGraphLaunch(r.exec, r.stream));
  r.ctx->launches += kBatchGraphKernels;
  return SIEVE_OK;
}

BatchRunner *new_batch_runner(sieve_ctx *ctx, cudaStream_t stream) {
  BatchRunner *r = new (std::nothrow) BatchRunner();
  if (!r) return nullptr;
  r->ctx = ctx;
  r->stream = stream;
  return r;
}

int batch_configure(BatchRunner &r) { return configure(r); }

// Re-run the compaction of the last batch into `values` (capacity cap), after
// the first run found its output buffer too small.
int batch_recompact(BatchRunner &r, uint64_t *values, uint64_t cap) {
  struct {
    uint64_t *v;
    uint64_t c;
  } patch = {values, cap};
  static_assert(offsetof(BatchHeader, cap) == offsetof(BatchHeader, values) + 8, "header layout");
  memcpy(r.h_back + 2, &patch, sizeof(patch));
  SIEVE_CUDA_TRY(cudaMemcpyAsync(r.d_plan + offsetof(BatchHeader, values), r.h_back + 2, sizeof(patch),
                                 cudaMemcpyHostToDevice, r.stream));
  BatchArena a = arena_of(r);
  batch_compact_kernel<kCompactThreads>
      <<<r.ctx->num_sms * 3, kCompactThreads, batch_compact_smem(r.Wmax), r.stream>>>(a);
  r.ctx->launches++;
  SIEVE_CUDA_TRY(cudaGetLastError());
  return SIEVE_OK;
}

}  // namespace sieve

using namespace sieve;

extern "C" int sieve_range_batch(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode,
                                 size_t nq, sieve_count_result *cnt, uint64_t *offsets, uint64_t *values,
                                 size_t cap, size_t *n_values, unsigned flags) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (n_values) *n_values = 0;
  if (nq && (!lo || !hi || !mode || !cnt)) {
    set_error("sieve_range_batch: lo, hi, mode and cnt must not be NULL");
    return SIEVE_ERR_INVALID;
  }
  if (!offsets || (!values && cap)) {
    set_error("sieve_range_batch: offsets (nq + 1 entries) must not be NULL, nor values when cap > 0");
    return SIEVE_ERR_INVALID;
  }
  const bool dev = (flags & SIEVE_OUT_DEVICE) != 0;
  cudaStream_t st = ctx->stream;
  if (nq == 0) {
    const uint64_t z = 0;
    if (dev)
      SIEVE_CUDA_TRY(cudaMemcpyAsync(offsets, &z, sizeof(z), cudaMemcpyHostToDevice, st));
    else
      offsets[0] = 0;
    SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
    return SIEVE_OK;
  }
  if (!ctx->batch) {
    ctx->batch = new_batch_runner(ctx, st);
    if (!ctx->batch) {
      set_error("host allocation failed");
      return SIEVE_ERR_OOM;
    }
  }
  BatchRunner &r = *ctx->batch;
  r.stream = st;
  int rc = configure(r);
  if (rc != SIEVE_OK) return rc;
  uint64_t *target = dev ? values : (uint64_t *)ctx->d_stage;
  uint64_t tcap = dev ? cap : ctx->stage_bytes / sizeof(uint64_t);
  const auto t_plan = std::chrono::steady_clock::now();
  if ((rc = batch_plan(r, lo, hi, mode, nq, target, tcap, 0, nullptr, nullptr)) != SIEVE_OK) return rc;
  if ((rc = batch_prepare(r)) != SIEVE_OK) return rc;
  if (ctx->phase_timing) {
    ctx->ph = sieve_phase_times{};
    ctx->ph.batch_plan_ms =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_plan).count();
    ctx->ph_recorded = 0;
    if (cudaEventRecord(ctx->ph_ev[0], st) == cudaSuccess) ctx->ph_recorded |= 1u;
  }
  if ((rc = batch_launch(r)) != SIEVE_OK) return rc;
  if (ctx->phase_timing && cudaEventRecord(ctx->ph_ev[1], st) == cudaSuccess) ctx->ph_recorded |= 2u;
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  SIEVE_CUDA_TRY(cudaMemcpyAsync(cnt, r.d_acc, nq * sizeof(sieve_count_result), kind, st));
  SIEVE_CUDA_TRY(cudaMemcpyAsync(offsets, r.d_offsets, (nq + 1) * sizeof(uint64_t), kind, st));
  SIEVE_CUDA_TRY(cudaMemcpyAsync(r.h_back + 1, r.d_offsets + nq, sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  const uint64_t total = r.h_back[1];
  if (n_values) *n_values = (size_t)total;
  if (total > cap) {
    set_error("output capacity %zu is below the %llu primes listed", cap, (unsigned long long)total);
    return SIEVE_ERR_CAPACITY;
  }
  if (dev || total == 0) return SIEVE_OK;
  if (total > tcap) {  // host output: the staging buffer was too small; grow it and compact again
    if ((rc = ensure_stage(ctx, (size_t)total * sizeof(uint64_t))) != SIEVE_OK) return rc;
    if ((rc = batch_recompact(r, (uint64_t *)ctx->d_stage, ctx->stage_bytes / sizeof(uint64_t))) != SIEVE_OK)
      return rc;
  }
  SIEVE_CUDA_TRY(cudaMemcpyAsync(values, ctx->d_stage, (size_t)total * sizeof(uint64_t), cudaMemcpyDeviceToHost, st));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(st));
  return SIEVE_OK;
}

// One sieve_range per query: the plain one-range-per-launch way of answering
// a batch, kept as the comparison point of the batched launch.
extern "C" int sieve_range_each(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode,
                                size_t nq, sieve_count_result *cnt, uint64_t *offsets, uint64_t *values,
                                size_t cap, size_t *n_values, unsigned flags) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (n_values) *n_values = 0;
  if ((nq && (!lo || !hi || !mode || !cnt)) || !offsets || (!values && cap)) {
    set_error("sieve_range_each: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  const bool dev = (flags & SIEVE_OUT_DEVICE) != 0;
  std::vector<uint64_t> off(nq + 1, 0);
  uint64_t run = 0;
  bool overflow = false;
  for (size_t i = 0; i < nq; i++) {
    if (mode[i] > 1) {
      set_error("query %zu: mode must be SIEVE_COUNT or SIEVE_LIST", i);
      return SIEVE_ERR_INVALID;
    }
    off[i] = run;
    RangeRequest rq;
    rq.lo = lo[i];
    rq.hi = hi[i];
    rq.total = cnt + i;
    rq.out_on_device = dev;
    size_t n = 0;
    int rc;
    if (mode[i] == SIEVE_LIST && !overflow) {
      rq.list = 1;
      rq.out_bytes = 8;
      rq.out = values ? values + run : nullptr;
      rq.cap = cap > run ? cap - run : 0;
      rc = run_range(ctx, ctx->table, rq, &n);
      if (rc == SIEVE_ERR_CAPACITY) {
        overflow = true;
        rc = SIEVE_OK;
      }
      if (rc != SIEVE_OK) return rc;
      run += n;
    } else {
      rq.async = dev;
      if ((rc = run_range(ctx, ctx->table, rq, nullptr)) != SIEVE_OK) return rc;
      if (mode[i] == SIEVE_LIST) {  // past the capacity: count only, for the size report
        sieve_count_result c;
        if (dev) {
          SIEVE_CUDA_TRY(cudaMemcpyAsync(&c, cnt + i, sizeof(c), cudaMemcpyDeviceToHost, ctx->stream));
          SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
        } else {
          c = cnt[i];
        }
        run += c.count;
      }
    }
  }
  off[nq] = run;
  if (n_values) *n_values = (size_t)run;
  if (dev) {
    SIEVE_CUDA_TRY(cudaMemcpyAsync(offsets, off.data(), (nq + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice,
                                   ctx->stream));
    SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  } else {
    memcpy(offsets, off.data(), (nq + 1) * sizeof(uint64_t));
  }
  if (overflow) {
    set_error("output capacity %zu is below the %llu primes listed", cap, (unsigned long long)run);
    return SIEVE_ERR_CAPACITY;
  }
  return SIEVE_OK;
}
