// batch.cuh -- many [lo, hi) queries sieved by one persistent launch.
//
// A batch is planned on the host into work items, uploaded as one block (the
// "plan"), and run as a fixed sequence of kernels captured in a CUDA graph:
//   init -> sieve (persistent, items taken from an atomic counter in cost
//   order) -> finish (merged tiles) -> scan (list offsets) -> compact.
//
// Work items (Sections 2.2-2.3: independent workers on contiguous chunks;
// Section 3: per-prime start indices):
//   * tile item: one tile of one query, sieved in shared memory as in the
//     single-range kernel, for the base primes [i0, i1).  A query's tile is
//     sized to the query (a power of two >= 1024 indices per class, at most
//     the batch tile size), so narrow queries use small tiles.
//   * strip item: base primes [i0, i1) that exceed the tile length, applied to
//     a whole query at once: each prime's first index comes from one start
//     evaluation for the query, then every later hit (index + P) is cleared
//     with an atomic AND in the query's bitmap in global memory.  This is the
//     work a bucket sieve saves for primes larger than a segment: a prime is
//     located once per query instead of once per tile, and a tile pays only
//     for the hits that land in it.
// Queries with strips are "merged": their tiles live in global memory (all
// ones after init); tile items AND their shared-memory result into it, strips
// strike it directly, and the finish kernel counts / emits each merged tile
// after the sieve kernel has ended (a kernel boundary orders them, so no
// kernel waits on another CTA).
#pragma once

#include <vector>

#include "sieve_internal.cuh"

namespace sieve {

constexpr uint32_t kStrip = 0xFFFFFFFFu;  // BatchItem::t of a strip item

struct BatchQuery {
  uint64_t lo, hi;          // [lo, hi)
  uint64_t k_begin, k_end;  // class indices; tile t covers [k_begin + t L, ...) up to k_end
  uint64_t bitmap_off;      // list mode: uint2 offset of tile 0's bitmap in the list scratch
  uint64_t slot_base;       // merged: u32 offset of tile 0 in the merge bitmaps (2 W words per tile)
  uint64_t out_base;        // fixed-output mode: element offset of this query's list
  uint64_t out_cap;         // fixed-output mode: elements reserved for it
  uint32_t logL, ntiles;    // tile length L = 2^logL indices per class
  uint32_t np;              // primes[0..np) cover isqrt(hi - 1)
  uint32_t i_split;         // primes below this index are struck by whole warps
  uint32_t ltile0;          // list tiles of the queries before this one
  uint32_t flags;           // bit 0: list mode, bit 1: merged
};

constexpr uint32_t kQueryList = 1u, kQueryMerged = 2u;

struct BatchItem {
  uint32_t q, t;    // query; tile within it, or kStrip
  uint32_t i0, i1;  // base-prime indices [i0, i1)
};

// Start of the uploaded plan.  Section offsets are bytes from the plan start.
struct BatchHeader {
  uint32_t nq, nitems, nmerged, nltiles;
  uint64_t slot_words;   // u32 words of merge bitmaps (all ones after init)
  uint64_t off_queries, off_items, off_mtiles, off_ltiles, off_ltile0;
  uint64_t *values;      // list output (device memory)
  uint64_t cap;          // CSR mode: capacity of values
  uint32_t fixed_out;    // 0: CSR (query q at offsets[q]); 1: query q at out_base
  uint32_t npat;         // presieve patterns in use
  uint32_t batch_id;     // distinct for every launch of a runner (see BatchState)
  uint32_t pad_;
};

// Device-written state of one batch.
struct BatchState {
  uint32_t next_item;
  uint32_t status;       // bit 0: CSR capacity exceeded; bit 1: a query exceeded its out_cap
  uint32_t yield_batch;  // when it equals the running batch's id, CTAs in the upper half of
                         // the grid take no further item and exit, making room for another
                         // batch (the lower half finishes the queue).  Written by the host
                         // at any time; never reset by the batch, so an early or late write
                         // for another batch id has no effect.
  uint32_t pad_;
};

// Device buffers of a batch arena (kernel parameters; fixed for a graph).
struct BatchArena {
  const void *plan;
  BatchState *state;
  unsigned long long *acc;  // 2 per query: count, checksum
  uint32_t *slot_bm;        // merge bitmaps
  uint32_t *tile_counts;    // per list tile
  uint64_t *tile_off;       // per list tile + 1
  uint64_t *offsets;        // per query + 1
  uint2 *list_bm;           // list tiles' bitmaps
  const uint32_t *primes;
  const uint64_t *magic;
  const uint2 *cinv;
  const PatternSetDev *psets;  // indexed by log2(W)
  uint32_t Wmax;               // words per class of the largest tile
  uint32_t band_max;           // warp-band start slots in shared memory
};

// Host side of one batch arena: its device buffers, pinned plan, CUDA graph
// and planning scratch (batch.cu).  A runner launches on its own stream; a
// plan may be rebuilt only once the runner's previous launch has completed.
struct BatchRunner {
  sieve_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  // launch shape, fixed for one graph
  int threads = 0, grid = 0, finish_grid = 0;
  size_t smem = 0, finish_smem = 0;
  uint32_t logLmax = 0, Wmax = 0, band_max = 0;
  // device capacities (elements of each buffer)
  size_t plan_cap = 0, acc_cap = 0, offsets_cap = 0, slot_cap = 0, counts_cap = 0, toff_cap = 0, list_cap = 0;
  char *d_plan = nullptr;
  BatchState *d_state = nullptr;
  unsigned long long *d_acc = nullptr;
  uint32_t *d_slot_bm = nullptr, *d_tile_counts = nullptr;
  uint64_t *d_tile_off = nullptr, *d_offsets = nullptr;
  uint2 *d_list_bm = nullptr;
  // pinned host plan and read-back words
  char *h_plan = nullptr;
  size_t h_plan_cap = 0;
  uint64_t *h_back = nullptr;  // [0] status, [1] list total
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t n_copy = nullptr;
  // planning scratch
  std::vector<BatchQuery> q;
  std::vector<BatchItem> items, sorted;
  std::vector<float> cost;
  std::vector<uint2> mtiles, ltiles;
  std::vector<uint32_t> ltile0;
  uint64_t slot_words = 0, list_words = 0;
  size_t plan_bytes = 0;
  uint32_t used_logW = 0;  // bit mask of tile widths in the plan
  uint32_t batch_id = 0;   // id of the last planned batch (first is 1)
  uint32_t table_epoch = 0;  // base-table epoch the graph's kernel arguments point into
};

// Runner operations (batch.cu).
BatchRunner *new_batch_runner(sieve_ctx *ctx, cudaStream_t stream);
int batch_configure(BatchRunner &r);
int batch_plan(BatchRunner &r, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode, size_t nq,
               uint64_t *values, uint64_t cap, int fixed_out, const uint64_t *out_base, const uint64_t *out_cap);
int batch_prepare(BatchRunner &r);
int batch_reserve(BatchRunner &r, size_t nq, size_t items, uint64_t slot_words, uint64_t list_words);
int batch_launch(BatchRunner &r);

}  // namespace sieve
