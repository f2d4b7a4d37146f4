// sieve_internal.cuh -- context layout and the arithmetic shared by every kernel.
//
// Notation follows the paper: a segment ("tile") of the 6k+1 / 6k+5 residue
// bitmaps (Section 2.1) holds `len` indices per class; index i of class r
// (r in {1, 5}) stands for the value B + 6 i + r, where B = 6 K0 is the
// segment's base value.  A base prime P strikes indices id_r, id_r + P, ...
// (Section 3: adding P to the index adds 6P to the value).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>
#include <vector>

#include "sieve.h"

namespace sieve {

constexpr uint32_t kFullMask = 0xFFFFFFFFu;

// Presieve: the multiples of the smallest base primes are removed by copying
// periodic bit patterns into a tile instead of striking them one by one.  In
// class-r index space a prime p coprime to 6 repeats with period p, so a group
// of primes repeats with the product of its members.  Pattern 0 is the wheel
// {5, 7, 11, 13, 17, 19}; patterns 1..kMaxPresieveGroups are groups of three
// consecutive primes from 23 on.  A context presieves with the wheel and the
// first `presieve_groups` groups; the strike loop starts after the last
// presieved prime.
constexpr int kMaxPresieveGroups = 8;
constexpr int kNumPatterns = 1 + kMaxPresieveGroups;
constexpr uint32_t kWheelPeriod = 5u * 7u * 11u * 13u * 17u * 19u;  // 1616615
// the primes of each pattern (0-padded)
constexpr uint32_t kPatternPrimes[kNumPatterns][6] = {
    {5, 7, 11, 13, 17, 19}, {23, 29, 31, 0, 0, 0},    {37, 41, 43, 0, 0, 0},
    {47, 53, 59, 0, 0, 0},  {61, 67, 71, 0, 0, 0},    {73, 79, 83, 0, 0, 0},
    {89, 97, 101, 0, 0, 0}, {103, 107, 109, 0, 0, 0}, {113, 127, 131, 0, 0, 0}};
constexpr uint32_t pattern_period(int g) {
  return g == 0 ? kWheelPeriod : kPatternPrimes[g][0] * kPatternPrimes[g][1] * kPatternPrimes[g][2];
}
// index (in the table 2, 3, 5, ...) of the first prime struck after presieving
// with the wheel and `groups` groups: 8 primes up to 19, then 3 per group
__host__ __device__ constexpr uint32_t first_struck_prime_index(int groups) { return 8u + 3u * (uint32_t)groups; }

// Per-pattern layout in the pattern buffer: class 1 at off1, class 5 at off5.
struct PatternDesc {
  uint32_t period;
  uint32_t off1, off5;
  uint32_t pad_;
  uint64_t magic;  // reciprocal64(period), for K0 mod period
};

// A set of presieve patterns for one tile width, as the batch kernels see it.
struct PatternSetDev {
  const uint32_t *d;
  PatternDesc pd[kNumPatterns];
};

// ---------------------------------------------------------------- arithmetic

__host__ __device__ __forceinline__ uint64_t mulhi64(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
  return __umul64hi(a, b);
#else
  return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}

// Division by an invariant divisor d (Granlund & Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994): with the precomputed
// reciprocal m = floor((2^64 - 1) / d), q' = floor(n m / 2^64) satisfies
// q - 1 <= q' <= q for every n < 2^63 (the deficit n (1 + e) / (d 2^64), with
// e < d the rounding of m, stays below 1/2), so one correction step gives q.
__host__ __device__ __forceinline__ uint64_t div_invariant(uint64_t n, uint32_t d, uint64_t m) {
  uint64_t q = mulhi64(n, m);
  uint64_t r = n - q * (uint64_t)d;
  if (r >= d) q++;
  return q;
}

__host__ __device__ __forceinline__ uint64_t reciprocal64(uint32_t d) { return ~0ull / d; }

// floor(a / 6) for a signed a (so that a - 6 floor(a / 6) is in [0, 6)).
__host__ __device__ __forceinline__ int64_t floor_div6(int64_t a) {
  int64_t q = a / 6;
  if (a - q * 6 < 0) q--;
  return q;
}

// Section 3, Table 1, with the P^2 start of Section 2.4.
//
// For a segment with base value B (B % 6 == 0) and start value M >= B, and a
// prime P >= 5 with reciprocal `m`:
//   M'  = max(M, P^2)                     (start no earlier than P^2)
//   Q   = greatest multiple of P below M' = floor((M' - 1) / P) * P
//   q   = Q mod 6,  p = P mod 6 (1 or 5),  R = floor(P / 6)
//   I   = floor((Q - B) / 6)              (the index "near" Q; may be negative)
//   id_1 = I + (Table 1 increment for class 1), id_5 likewise.
// The result indexes the first class-1 / class-5 multiple of P above Q, which
// is the first one >= M'.  Q - B lies in [-P, segment span), signed 64-bit.
// Table 1 as coefficients: id_r = I + a_r * R' + b_r, with R' = R when p = 1
// and R' = R + 1 when p = 5:
//   p = 1: id_1: q = 0 -> R,      q >= 1 -> (7 - q) R + 1
//          id_5: q <= 4 -> (5 - q) R,     q = 5 -> 6 R + 1
//   p = 5: id_1: q = 0 -> 5 R' - 1, q = 1 -> 6 R' - 1, q >= 2 -> (q - 1) R'
//          id_5: (q + 1) R' - 1
struct StartIndex {
  int64_t id1, id5;
};

__host__ __device__ __forceinline__ StartIndex table1_start(uint64_t B, uint64_t M, uint32_t P,
                                                            uint64_t m) {
  uint64_t P2 = (uint64_t)P * P;
  uint64_t Mp = M > P2 ? M : P2;
  uint64_t Q = div_invariant(Mp - 1, P, m) * P;
  int64_t d = (int64_t)(Q - B);
  int64_t I = floor_div6(d);
  int32_t q = (int32_t)(d - 6 * I);
  int32_t R = (int32_t)(P / 6u);
  int32_t a1, b1, a5, b5, Rp;
  if (P % 6u == 1u) {
    Rp = R;
    a1 = q == 0 ? 1 : 7 - q;
    b1 = q == 0 ? 0 : 1;
    a5 = q == 5 ? 6 : 5 - q;
    b5 = q == 5 ? 1 : 0;
  } else {
    Rp = R + 1;
    a1 = q == 0 ? 5 : (q == 1 ? 6 : q - 1);
    b1 = q <= 1 ? -1 : 0;
    a5 = q + 1;
    b5 = -1;
  }
  StartIndex s;
  s.id1 = I + (int64_t)a1 * Rp + b1;
  s.id5 = I + (int64_t)a5 * Rp + b5;
  return s;
}

// u = 1 + ((B - 1) mod P), in [1, P]: B - u is the greatest multiple of P
// below B (the Q of Table 1 for a segment starting at M = B), and the first
// multiple at or above B is B + (P - u).  One 64-bit remainder by the
// reciprocal m of P.
__host__ __device__ __forceinline__ uint32_t dist_below(uint64_t B, uint32_t P, uint64_t m) {
  const uint64_t n = B - 1;
  const uint64_t qq = mulhi64(n, m);
  uint32_t r = (uint32_t)(n - qq * (uint64_t)P);
  if (r >= P) r -= P;
  return r + 1;
}

// Table 1 start indices for a tile with base B, start value M = B, and a
// prime P with P^2 <= B and P < 2^31, from u = dist_below(B, P, m): the index
// near Q = B - u is I = floor(-u / 6) = -ceil(u / 6) and q = Q mod 6 =
// (-u) mod 6; everything is 32-bit.  The sum I + a R' + b is formed modulo 2^32
// (unsigned, so that the wrap is defined); the start itself is in [0, 2^32)
// for P < 2^31, so the result is exact.  Same result as table1_start(B, B, P, m).
__host__ __device__ __forceinline__ void table1_from_dist(uint32_t u, uint32_t P, uint32_t &id1, uint32_t &id5) {
  const uint32_t cu = (u + 5) / 6;
  const uint32_t q = 6 * cu - u;
  const uint32_t R = P / 6u;
  uint32_t a1, b1, a5, b5, Rp;
  if (P % 6u == 1u) {
    Rp = R;
    a1 = q == 0 ? 1 : 7 - q;
    b1 = q == 0 ? 0 : 1;
    a5 = q == 5 ? 6 : 5 - q;
    b5 = q == 5 ? 1 : 0;
  } else {
    Rp = R + 1;
    a1 = q == 0 ? 5 : (q == 1 ? 6 : q - 1);
    b1 = q <= 1 ? 0xFFFFFFFFu : 0;  // -1
    a5 = q + 1;
    b5 = 0xFFFFFFFFu;               // -1
  }
  id1 = a1 * Rp + b1 - cu;
  id5 = a5 * Rp + b5 - cu;
}

__host__ __device__ __forceinline__ void table1_start_tile(uint64_t B, uint32_t P, uint64_t m, uint32_t &id1,
                                                           uint32_t &id5) {
  table1_from_dist(dist_below(B, P, m), P, id1, id5);
}

// Start indices of prime P in the tile with base B (M = B), as uint64 (every
// start is >= 0): the 32-bit path when P^2 <= B and P < 2^31, else the
// general one.  The kernels and the host entry sieve_table1_start use this.
__host__ __device__ __forceinline__ void tile_starts(uint64_t B, uint32_t P, uint64_t m, uint64_t &k1,
                                                     uint64_t &k5) {
  const uint64_t P2 = (uint64_t)P * P;
  if (P2 <= B && P < 0x80000000u) {
    uint32_t i1, i5;
    table1_start_tile(B, P, m, i1, i5);
    k1 = i1;
    k5 = i5;
  } else {
    const StartIndex st = table1_start(B, B, P, m);
    k1 = (uint64_t)st.id1;
    k5 = (uint64_t)st.id5;
  }
}

// Start indices of P in a tile with base B whose values end below B + span6,
// or false when P has no multiple in [B, B + span6) at all: then neither class
// is hit and the Table 1 step is skipped (the common case for primes larger
// than a narrow tile).
__host__ __device__ __forceinline__ bool tile_starts_within(uint64_t B, uint32_t P, uint64_t m, uint32_t span6,
                                                            uint64_t &k1, uint64_t &k5) {
  const uint64_t P2 = (uint64_t)P * P;
  if (P2 <= B && P < 0x80000000u) {
    const uint32_t u = dist_below(B, P, m);
    if (P - u >= span6) return false;
    uint32_t i1, i5;
    table1_from_dist(u, P, i1, i5);
    k1 = i1;
    k5 = i5;
    return true;
  }
  const StartIndex st = table1_start(B, B, P, m);
  k1 = (uint64_t)st.id1;
  k5 = (uint64_t)st.id5;
  return true;
}

// The same start indices from the inverse of 6.  Class r's index k holds
// value 6 (K0 + k) + r, which P divides iff K0 + k = -r / 6 (mod P); so with
// c_r = (-r / 6) mod P the first such k >= 0 is (c_r - K0 mod P) mod P.  The
// base table keeps (c_1, c_5) per prime for the tiles' one-lane band (a load
// is cheaper there than the arithmetic below, measured); the strips, which
// stream the table from DRAM, compute them.  This
// equals the Table 1 start whenever P^2 <= 6 K0 (no clamp; the start lies
// below P), and costs one invariant-division remainder and a few 32-bit
// operations instead of the table's case split.  The constants have a closed
// form in R = floor(P / 6): 6^{-1} mod P is (P + 1) / 6 = R + 1 for P = 6R + 5
// and (5 P + 1) / 6 = 5R + 1 for P = 6R + 1, so
//   P = 6R + 1:  c_1 = R,       c_5 = 5R
//   P = 6R + 5:  c_1 = 5R + 4,  c_5 = R
// (P >= 5, P % 6 in {1, 5}).
__host__ __device__ __forceinline__ uint2 inverse6_constants(uint32_t P) {
  const uint32_t R = P / 6u;
  return P - 6u * R == 1u ? make_uint2(R, 5u * R) : make_uint2(5u * R + 4u, R);
}

// k1 / k5 = (c - K0 mod P) mod P for P < 2^31 (m = reciprocal64(P)).
__host__ __device__ __forceinline__ void starts_from_inverse(uint64_t K0, uint32_t P, uint64_t m, uint2 c,
                                                             uint32_t &k1, uint32_t &k5) {
  const uint64_t q = mulhi64(K0, m);  // floor(K0 / P) or one less
  uint32_t r = (uint32_t)K0 - (uint32_t)q * P;  // exact: K0 - q P < 2 P < 2^32
  if (r >= P) r -= P;
  k1 = c.x >= r ? c.x - r : c.x - r + P;
  k5 = c.y >= r ? c.y - r : c.y - r + P;
}

// ---------------------------------------------------------------- context

struct DeviceTable {
  const uint32_t *primes = nullptr;       // device: 2, 3, 5, 7, ... (all primes <= limit)
  const uint64_t *magic = nullptr;        // device: reciprocal64(primes[i])
  const uint2 *cinv = nullptr;            // device: inverse6_constants(primes[i])
  const uint32_t *host_primes = nullptr;  // host copy of primes
  uint32_t nprimes = 0;
  uint64_t limit = 0;
  // host: count_idx[j] = number of table primes below j << kCountIndexShift,
  // for j < count_idx_n (optional: without it counts search the whole table)
  const uint32_t *count_idx = nullptr;
  uint64_t count_idx_n = 0;
};

// Bucket width of the host prime-count index: a count searches one bucket of
// about 2^12 / ln x primes instead of the whole table (a batch plan makes
// three counts per query).
constexpr uint32_t kCountIndexShift = 12;

struct BatchRunner;  // batch.cu

// Number of table primes <= s (host binary search).
uint32_t host_prime_count_le_table(const DeviceTable &t, uint64_t s);

}  // namespace sieve

struct sieve_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int smem_optin = 0;          // max dynamic shared memory per block
  uint64_t max_hi = 0;
  sieve::DeviceTable table;    // views into the buffers below
  uint32_t *d_primes = nullptr;
  uint64_t *d_magic = nullptr;
  uint2 *d_cinv = nullptr;
  std::vector<uint32_t> h_primes;  // host copy of the base table
  std::vector<uint32_t> h_count_idx;  // its prime-count index (DeviceTable::count_idx)
  // presieve patterns in the sliced layout, one set per tile width W = 2^logW
  struct SlicedSet {
    uint32_t *d = nullptr;
    sieve::PatternDesc pd[sieve::kNumPatterns];
  } sliced[32];
  sieve_options opt{};
  std::atomic<uint64_t> launches{0};  // read by other threads while a server runs
  uint32_t table_epoch = 0;           // bumped whenever the base table moves
  // device copy of the pattern sets, indexed by log2(W); entry i is valid
  // when bit i of psets_ready is set
  sieve::PatternSetDev *d_psets = nullptr;
  uint32_t psets_ready = 0;
  // batch runner of the synchronous batch call (batch.cu)
  sieve::BatchRunner *batch = nullptr;
  // small device scratch: accumulators and status words
  unsigned long long *d_acc = nullptr;
  size_t acc_words = 0;
  // growable device scratch for list mode (bitmaps, tile counts, offsets)
  void *d_scratch = nullptr;
  size_t scratch_bytes = 0;
  // growable device staging for list output bound for host memory
  void *d_stage = nullptr;
  size_t stage_bytes = 0;
  // resident CTAs per SM of the range kernels, by (threads 256/512/1024,
  // list mode, log2 of the tile length); 0 = not asked yet (range.cu)
  int occ_cache[3][2][32] = {};
  // bucket sieve buffers of single-range calls (entries, counts, overflow
  // flags), kept across calls and grown on demand (range.cu)
  void *d_bucket = nullptr;
  size_t bucket_bytes = 0;
  // device address of the fixed scratch array of sieve_range_list_noalloc,
  // looked up by sieve_create with this context's device current (noalloc.cu)
  void *noalloc_scratch = nullptr;
  // pinned host staging
  unsigned long long *h_acc = nullptr;
  // phase timing of single-range calls (sieve_set_phase_timing): events
  // around the tile kernel (0, 1), after the scan (2; it starts at 1), and
  // around the compaction (3, 4)
  bool phase_timing = false;
  cudaEvent_t ph_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  uint32_t ph_recorded = 0;  // bit i: ph_ev[i] recorded by the last call
  sieve_phase_times ph{};
};

namespace sieve {

// error reporting (thread-local message)
void set_error(const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define SIEVE_CUDA_TRY(expr)                              \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return sieve::cuda_fail(_e, #expr); \
  } while (0)

// scratch management (api.cu); contents are not preserved when they grow
int ensure_scratch(sieve_ctx *ctx, size_t bytes);
int ensure_stage(sieve_ctx *ctx, size_t bytes);

// exact integer square root (host)
uint64_t isqrt_u64(uint64_t n);

// cudaFuncAttributeMaxDynamicSharedMemorySize for the range kernels (range.cu)
int range_set_smem_attributes(int bytes);

// The presieve patterns in the sliced layout for tiles of W = 2^logW words per
// class, built on first use (api.cu).
int sliced_patterns(sieve_ctx *ctx, uint32_t logW, const uint32_t **ptr, PatternDesc *pd);
// Make sure the device table entry for log2(W) = logW is filled (api.cu).
int ensure_pattern_set_dev(sieve_ctx *ctx, uint32_t logW);

// Grow the base table to every prime <= new_limit (at most the square of
// its current limit; api.cu).
int extend_base_table(sieve_ctx *ctx, uint64_t new_limit);

// Looks up the device address of the fixed no-allocation scratch array on
// the current device into ctx->noalloc_scratch (noalloc.cu).  Called by
// sieve_create, so that the array's module is loaded while the context is
// being made (which allocates anyway), not by a later call that must not.
int noalloc_setup(sieve_ctx *ctx);

// batch runner lifetime (batch.cu)
void destroy_batch_runner(BatchRunner *r);

// Range driver used by the public calls and by the base-table builder
// (range.cu).  Output kinds for list mode: 4 (uint32) or 8 (uint64) bytes.
struct RangeRequest {
  uint64_t lo = 0, hi = 0;
  int list = 0;              // 0: count only; 1: also write the list
  int out_bytes = 8;         // list element size
  void *out = nullptr;       // list output (device or host per out_on_device)
  size_t cap = 0;
  int out_on_device = 0;
  uint64_t seg_width = 0;    // 0: no per-segment counts
  uint64_t *bins = nullptr;  // per-segment counts (device or host)
  size_t nbins = 0;
  sieve_count_result *total = nullptr;  // may be null
  int async = 0;             // count mode with device outputs: enqueue only
};

int run_range(sieve_ctx *ctx, const DeviceTable &table, const RangeRequest &req, size_t *n_out);

// Whether run_range would send the large primes of a count of [lo, hi) through
// the bucket sieve (range.cu); sieve_range then keeps the range on the tile
// path instead of routing it to the batch path's strips (the buckets measured
// faster on every far range tried).
bool range_prefers_buckets(sieve_ctx *ctx, uint64_t lo, uint64_t hi);

// Bytes of a range's two class bitmaps up to which they stay in L2: below it
// the batch path's strips (atomic ANDs into the bitmap) beat the bucket sieve
// for a far range, above it the bucket sieve wins (measured both ways).
constexpr uint64_t kStripBitmapL2 = 48000000;

// Whether the batch path's strips beat the bucket sieve on a far range:
// measured on one GB300 (counts, widths 1e8..1e9 and 1e10, lo 1e12..1e18),
// they do when the range's bitmap fits in L2, the range is at least 3e8 wide
// and its base primes reach 1e8 (lo above about 1e16): a single pass of
// locations over tens of millions of primes and L2-resident atomic ANDs cost
// less than the bucket entries' round trip.  Below that the bucket sieve is
// faster (e.g. [1e15, 1e15 + 1e8): 0.13 against 0.30 ms) or equal (api.cu).
bool strips_beat_buckets(uint64_t lo, uint64_t hi);

}  // namespace sieve
