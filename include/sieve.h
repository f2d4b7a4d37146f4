/*
 * sieve.h -- C ABI of the GB300 segmented prime sieve (libsieve_gb300.so).
 *
 * The library finds the primes of a range with the incremental segmented
 * Sieve of Eratosthenes of "Memory Efficient Multithreaded Incremental
 * Segmented Sieve Algorithm" (Ning & Kaeli):
 *   - problem statement: all primes from 2 through n (Section 1.1, Figure 1);
 *   - only candidates 6k+1 and 6k+5 are stored, one bit each, in two residue
 *     bitmaps per segment (Section 2.1, Figure 2; the paper's A_one / A_five);
 *   - the range is cut into contiguous segments, each owned by one worker
 *     (Sections 2.2 and 2.3) -- here one CTA per segment, bitmaps in shared
 *     memory;
 *   - a base prime P starts sieving at P^2 (Section 2.4), and its first index
 *     in each residue class of a segment comes from the Table 1 operation
 *     (Section 3), after which the index advances by P (6P in value);
 *   - the segments' survivors are counted or written out in increasing order
 *     (Section 4, Figure 4: "return all k such that mod1[k] or mod5[k]").
 *
 * Conventions shared by every call:
 *   - Every call returns a sieve_status.  On failure sieve_last_error() gives a
 *     message (thread-local, valid until the thread's next call).
 *   - Ranges are half-open [lo, hi) unless a call says "inclusive"; n-style
 *     calls are inclusive (primes p with 2 <= p <= n).  lo > hi is
 *     SIEVE_ERR_INVALID; lo == hi is SIEVE_OK with nothing found.
 *   - hi - 1 must not exceed the context's max_hi - 1 (the square of its base
 *     table's limit covers it), else SIEVE_ERR_RANGE.  max_hi <= 2^63.
 *   - Counts are uint64.  A checksum is the sum of the primes modulo 2^64.
 *   - Lists are strictly increasing.
 *   - The caller owns every buffer it passes; the library never frees or
 *     keeps caller memory beyond the call.  The library owns everything it
 *     allocates in a context (base table, wheel pattern, scratch) and frees it
 *     in sieve_destroy.
 *   - flags: SIEVE_OUT_DEVICE says that the call's output pointers are device
 *     memory on the context's device; otherwise they are host memory.  With
 *     SIEVE_OUT_DEVICE | SIEVE_ASYNC a count-mode call only enqueues its work
 *     on the context's stream and returns; every other call returns after its
 *     results are complete.
 *   - A context is not thread-safe: one host thread at a time per context.
 *   - Device kernels contain no unbounded waits; device-side failures are
 *     reported through a status word read back by the host.
 */
#ifndef SIEVE_GB300_H
#define SIEVE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sieve_ctx sieve_ctx;
typedef struct sieve_server sieve_server;

typedef enum {
  SIEVE_OK = 0,
  SIEVE_PENDING = 1,          /* server: request not finished yet            */
  SIEVE_ERR_INVALID = -1,     /* bad argument                                  */
  SIEVE_ERR_RANGE = -2,       /* range beyond the context's base table         */
  SIEVE_ERR_CAPACITY = -3,    /* output buffer too small; needed size reported */
  SIEVE_ERR_OOM = -4,         /* device or host allocation failed              */
  SIEVE_ERR_CUDA = -5,        /* a CUDA runtime call failed                    */
  SIEVE_ERR_TIMEOUT = -6,     /* a bounded wait ran out                        */
  SIEVE_ERR_BUSY = -7,        /* server: admission refused (backpressure)      */
  SIEVE_ERR_NOT_FOUND = -8    /* server: unknown or already collected request  */
} sieve_status;

typedef enum { SIEVE_COUNT = 0, SIEVE_LIST = 1 } sieve_mode;

#define SIEVE_OUT_DEVICE 1u
#define SIEVE_ASYNC 2u

typedef struct {
  uint64_t count;    /* number of primes found                 */
  uint64_t checksum; /* sum of the primes found, modulo 2^64   */
} sieve_count_result;

/* Tunables of the segment kernels (the autotuners fill them; see
 * sieve_autotune_range / sieve_autotune_batch).  Section 5 measures how the
 * per-thread scratch array size changes the run time; tile_bits is that knob
 * here. */
typedef struct {
  uint32_t tile_bits;      /* L: candidates per residue class per segment (multiple of 1024,
                              2 * L / 8 bytes of shared memory per CTA)                      */
  uint32_t block_threads;  /* threads per CTA: 256, 512 or 1024                              */
  uint32_t ctas_per_sm;    /* resident CTAs per SM the launch aims for (0: as many as fit)   */
  uint32_t group_hits;     /* a prime is struck by a group of lanes when it has at least this
                              many hits per lane in a segment; below that, one lane per prime */
  uint32_t presieve_groups;  /* 0..8: besides the wheel {5..19}, how many groups of three
                              primes (23, 29, 31), (37, 41, 43), ... up to 131 are removed by
                              copying periodic patterns instead of striking                  */
  uint32_t batch_tile_bits;  /* batch calls: largest tile (a query narrower than it gets a
                              smaller power-of-two tile, at least 1024); 0 = tile_bits       */
  uint32_t chunk_primes;   /* batch calls (>= 1024): a query whose base primes above the tile
                              length, times its tiles, reach this number is "merged": those
                              primes are applied by strip items of at most this many primes,
                              each striking the query's bitmap in global memory             */
  uint32_t bucket_threshold; /* single ranges: base primes above bucket_threshold x tile_bits go
                              through the bucket sieve (located once per wave of tiles, their hits
                              sorted into per-tile buckets that each tile drains) when they are
                              many and each hits a tile rarely; where the primes above it hit
                              too often, the planner raises the threshold in steps of a quarter
                              (it is the lowest one); with buckets the presieve copies at most 4
                              groups; 0 = off (every prime is located in every tile); at most 64 */
  uint32_t bucket_wave;    /* bucket sieve: tiles per CTA in one wave (1..16)                  */
  uint32_t bucket_scatter; /* bucket sieve: 1 = direct scatter (each hit stored at once), 2 =
                              sorted scatter (a round's hits sorted by tile in shared memory,
                              written in runs), 0 = direct while a wave's entries fit in L2,
                              else sorted with waves of at least 4 tiles per CTA              */
  uint32_t list_single_pass; /* single-range lists into device memory: 1 = one pass (each tile
                              compacted from shared memory at an offset found by look-back over
                              the tiles before it), 0 = two passes (bitmaps to global memory,
                              scan, compaction; the default, measured faster); host-bound
                              lists always take two passes                                    */
  uint32_t cluster_ctas;   /* single ranges: 0 = off; 2, 4, 8 or 16 = cluster segments (Sections
                              2.2-2.3 with the chunk spread over a thread-block cluster): C CTAs
                              sieve C consecutive tiles together, the base primes above
                              cluster_threshold x tile_bits are located once per segment and
                              struck into the member CTAs' shared memory through distributed
                              shared memory.  Replaces the bucket sieve and the far-range
                              strips route for the call; single-pass lists and ranges whose
                              base primes reach 2^31 keep their usual route.  Measured slower
                              than the bucket sieve on a GB300 (remote shared-memory ANDs run
                              at a small fraction of the local rate); 16 needs a device that
                              allows clusters beyond the portable size of 8                   */
  uint32_t cluster_threshold; /* cluster segments: base primes above cluster_threshold x tile_bits
                              are located once per segment (0: every one-lane prime); at most
                              1024                                                           */
} sieve_options;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` whose calls run on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  Builds the
 * device-resident base table of every prime <= isqrt(max_hi - 1) (the
 * Sieve Data Store of Section 4: primes up to the square root only) and the
 * wheel presieve pattern.  The table is built incrementally (Section 2.4):
 * primes up to its fourth root on the host, the rest by this library's own
 * GPU sieve.  max_hi in [2, 2^63].
 * Errors: INVALID (max_hi out of range, ctx NULL), CUDA, OOM. */
int sieve_create(sieve_ctx **ctx, uint64_t max_hi, int device, void *cuda_stream);

/* Free everything the context owns.  NULL is ignored. */
void sieve_destroy(sieve_ctx *ctx);

/* Stream the context's calls are ordered on from now on. */
int sieve_set_stream(sieve_ctx *ctx, void *cuda_stream);

int sieve_get_options(const sieve_ctx *ctx, sieve_options *opt);
/* Validates every field; INVALID leaves the options unchanged. */
int sieve_set_options(sieve_ctx *ctx, const sieve_options *opt);

/* Base table facts: its limit (every prime <= limit is held), the number of
 * primes in it, and the device address of the uint32 table (owned by ctx). */
int sieve_base_table(const sieve_ctx *ctx, uint64_t *limit, uint64_t *nprimes,
                     const uint32_t **device_primes);

/* Number of kernels this context has launched so far (every launch of the
 * library's own kernels is counted). */
uint64_t sieve_launch_count(const sieve_ctx *ctx);

const char *sieve_last_error(void);

/* ------------------------------------------------------------- range calls */

/* Count of primes p with 2 <= p <= n, and their sum mod 2^64 (Section 1.1). */
int sieve_count(sieve_ctx *ctx, uint64_t n, sieve_count_result *out);

/* Primes p with 2 <= p <= n, increasing, written to out[0..cap).  *n_out gets
 * the number of primes; if it exceeds cap the call returns CAPACITY, writes
 * nothing past out[cap - 1] and leaves out's contents unspecified. */
int sieve_primes(sieve_ctx *ctx, uint64_t n, uint64_t *out, size_t cap, size_t *n_out,
                 unsigned flags);
/* Same with uint32 output (n < 2^32, else INVALID). */
int sieve_primes_u32(sieve_ctx *ctx, uint64_t n, uint32_t *out, size_t cap, size_t *n_out,
                     unsigned flags);

/* Primes in [lo, hi).  mode SIEVE_COUNT fills *cnt; mode SIEVE_LIST also
 * writes the primes to out[0..cap) as uint64 with the CAPACITY rule above.
 * cnt may be NULL in list mode.  In count mode with SIEVE_OUT_DEVICE, cnt is a
 * device pointer to one sieve_count_result.  A range far up -- one whose base
 * primes above the segment length would cost more to locate in every segment
 * than to locate once and strike in a bitmap in global memory -- is run
 * through the batch machinery as a one-query batch (see sieve_range_batch);
 * the result is the same (except that SIEVE_ASYNC ranges always take the
 * segment path). */
int sieve_range(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int mode, sieve_count_result *cnt,
                uint64_t *out, size_t cap, size_t *n_out, unsigned flags);

/* The plain GPU sieve of [lo, hi), the comparison point for the segmented
 * path (Section 1.1 / Figure 1 done directly, one range per call): one bit per
 * odd number of the range in a bitmap in global memory, every odd multiple
 * m >= max(p^2, lo) of every odd base prime p cleared with a global atomic
 * AND (a prime's multiples spread over as many CTAs as they need), then a
 * popcount pass, or a count / scan / write pass for the list.  No residue
 * classes, presieve, shared-memory segments or Table 1.  Same arguments,
 * outputs and errors as sieve_range (the list is uint64), plus OOM when the
 * bitmap (one byte per 16 numbers, e.g. 62.5 GB for [2, 1e12]) does not fit
 * on the device; it allocates and frees the bitmap in every call. */
int sieve_range_naive(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int mode, sieve_count_result *cnt,
                      uint64_t *out, size_t cap, size_t *n_out, unsigned flags);

/* Count, checksum and per-segment counts of the primes in [lo, hi).
 * Segment s is the value interval [s*seg_width, (s+1)*seg_width); counts[i]
 * holds segment floor(lo / seg_width) + i, so ncounts must equal
 * floor((hi - 1) / seg_width) - floor(lo / seg_width) + 1 (0 when lo == hi).
 * seg_width >= 6144.  total may be NULL.  With SIEVE_OUT_DEVICE both counts
 * and total are device pointers. */
int sieve_segment_counts(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t seg_width,
                         uint64_t *counts, size_t ncounts, sieve_count_result *total,
                         unsigned flags);

/* The first k primes greater than `after`, increasing, into out[0..k) (host
 * memory, or device memory with SIEVE_OUT_DEVICE); *n_out = k on success.
 * Incremental in the paper's sense (Sections 2.4 and 4): no upper bound is
 * fixed in advance -- the call sieves forward in windows and, when a window
 * reaches past the square of the base table's limit, grows the table with
 * the sieve itself (the new primes come from sieving the table's extension
 * with the current table).  A chain of calls, each starting after the last
 * prime of the previous one, streams the primes without end (up to 2^63).
 * Growing the table moves it: device pointers from sieve_base_table become
 * stale.  Errors: INVALID, RANGE (past 2^63), OOM, CUDA. */
int sieve_next(sieve_ctx *ctx, uint64_t after, size_t k, uint64_t *out, size_t *n_out, unsigned flags);

/* ------------------------------------------------------------- long runs */

/* The paper's first future-work item (Section 6) is to write results out in
 * store segments instead of keeping them in memory; these two calls do that
 * for counts and for lists, and survive interruption.  Their state files are
 * small binary records (8 magic bytes, little-endian uint64 words, a 64-bit
 * FNV-1a hash of the preceding bytes), written to path + ".tmp" and renamed
 * over the old record after every chunk, so a crash leaves the old or the new
 * record, never a torn one.
 *
 * sieve_count_checkpointed: count, checksum and per-segment counts of
 * [lo, hi) (segments as sieve_segment_counts; seg_width 0 = no segments and
 * ncounts 0), sieved in chunks [lo + k chunk_width, lo + (k + 1) chunk_width).
 * After every chunk the running state (next position, count, checksum, bins)
 * goes to state_path.  A call that finds a state for the same (lo, hi,
 * seg_width, chunk_width) resumes after its last finished chunk; a state of
 * another job, or a damaged one, is INVALID.  max_chunks > 0 stops after that
 * many chunks of this call and returns SIEVE_PENDING with the partial totals
 * (call again to continue); 0 runs to the end.  When the range is done the
 * call returns SIEVE_OK with *total and counts[] (host memory) complete, and
 * a later call with the same state returns them without sieving.  *next (may
 * be NULL) gets the start of the first chunk not yet done. */
int sieve_count_checkpointed(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t seg_width, uint64_t chunk_width,
                             const char *state_path, uint64_t *counts, size_t ncounts,
                             sieve_count_result *total, uint64_t max_chunks, uint64_t *next);

/* The primes of [lo, hi), increasing, as little-endian uint64 in the binary
 * file `path`, written one store segment at a time: a window of the range
 * whose prime count is surely <= segment_primes (0 = 125,000,000, i.e. 1 GB
 * of output per segment) is sieved into device memory, copied to pinned host
 * memory and appended, then path + ".state" records the next position and
 * the primes written.  resume != 0 continues from that state (the file is
 * cut back to the primes the state records, dropping what an interrupted
 * segment left); resume == 0 starts a new file.  max_segments > 0 stops after
 * that many segments of this call with SIEVE_PENDING.  *n_written (may be
 * NULL) = primes in the file.  Uses segment_primes x 8 bytes of device memory
 * and as much pinned host memory, allocated and freed by the call.  Errors:
 * INVALID (bad argument, file error, state of another job), RANGE, OOM, CUDA. */
int sieve_primes_to_file(sieve_ctx *ctx, uint64_t lo, uint64_t hi, const char *path, size_t segment_primes,
                         int resume, uint64_t max_segments, uint64_t *n_written);

/* ------------------------------------------------------------- batches */

/* Many independent ranges in one call: query i is [lo[i], hi[i]) in mode
 * mode[i] (SIEVE_COUNT or SIEVE_LIST).  Each query is the problem of Section
 * 1.1 on its own range, sieved as in Sections 2-4; what the batch adds is the
 * scheduling.  The queries are planned on the host into work items -- one
 * per tile, sized to the query (a power of two of at least 1024 and at most
 * sieve_options.batch_tile_bits indices per class), plus, for queries with
 * many base primes above the tile length, "strips" that locate those primes
 * once per query (Table 1) and clear their hits in a global bitmap with
 * atomic ANDs -- and run by ONE persistent kernel launch that takes the items
 * from an atomic counter: first the items of those "merged" queries, one
 * query after another (so that its bitmap stays in L2), then the rest in
 * decreasing estimated cost.  The launch and its set-up / finish / scan /
 * compaction kernels are replayed as one CUDA graph.
 *
 * Inputs lo, hi, mode: HOST arrays of nq entries (the plan is built on the
 * host).  Outputs, host or device memory per SIEVE_OUT_DEVICE:
 *   cnt[nq]        count and checksum of every query (both modes);
 *   offsets[nq+1]  list-mode primes of query i are values[offsets[i] ..
 *                  offsets[i+1]) (count queries get an empty run);
 *   values[cap]    the listed primes, uint64, each query's run increasing.
 * *n_values (may be NULL) gets offsets[nq].  If it exceeds cap the call
 * returns CAPACITY after filling cnt and offsets, writes nothing to values,
 * and *n_values tells the size needed.  Per-query errors (lo > hi, mode not
 * 0/1, hi beyond the base table) reject the whole batch (INVALID / RANGE,
 * with the query index in the message).  Synchronous: returns after every
 * output is complete.  The context keeps the batch buffers for the next call. */
int sieve_range_batch(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode, size_t nq,
                      sieve_count_result *cnt, uint64_t *offsets, uint64_t *values, size_t cap,
                      size_t *n_values, unsigned flags);

/* The same contract answered the plain way: one segment-path range sieve
 * (its own kernel launches and synchronisation, as sieve_range without the
 * batch route) per query, in order.  It is the comparison point for
 * sieve_range_batch.  On CAPACITY, *n_values is exact
 * (the queries past the capacity are counted but not listed). */
int sieve_range_each(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode, size_t nq,
                     sieve_count_result *cnt, uint64_t *offsets, uint64_t *values, size_t cap,
                     size_t *n_values, unsigned flags);

/* ------------------------------------------------------------- autotuning */

/* Pick tunables by timing them, as Section 5 does for its per-thread array
 * size.  Each candidate runs once untimed, then `reps` times under CUDA events
 * on the context's stream; the one with the smallest median time becomes the
 * context's options (returned in *best, time in *best_ms; either may be
 * NULL).  Every candidate's results must equal the first candidate's, else
 * the call fails with SIEVE_ERR_CUDA and the options are left unchanged.
 *   sieve_autotune_batch: batch_tile_bits {2^15 .. 2^19} x block_threads
 *     {512, 1024} x chunk_primes {2^13, 2^15, 2^17} on the given batch (host
 *     arrays, as sieve_range_batch), then presieve_groups {4 .. 7} with the
 *     winner's other settings; allocates and frees its own device outputs.
 *   sieve_autotune_range: tile_bits {2^18, 2^19} x block_threads {512, 1024}
 *     x ctas_per_sm {0, 1, 2} (512 threads only) x group_hits {3, 4, 5, 6, 8}
 *     x presieve_groups {5, 6, 7, 8} on the count of [lo, hi) (a sample of the
 *     ranges to come; every candidate sieves it reps + 1 times); then, when
 *     the range's large primes can use the bucket sieve, bucket_threshold
 *     {0, 2, 4, 8, 16} x bucket_wave {1, 4} x bucket_scatter {1, 2} with the
 *     winner's other settings.  The context's own options stay when they are
 *     among the candidates and within 1% of the fastest (run-to-run noise). */
int sieve_autotune_batch(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode, size_t nq,
                         int reps, sieve_options *best, double *best_ms);
int sieve_autotune_range(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int reps, sieve_options *best,
                         double *best_ms);

/* A cache of tuned options in a small JSON file, keyed by (device name, SM
 * count, workload name), so that a tuning run is paid once per device and
 * workload class.  The file holds {"sieve_tune_cache": 1, "entries": [...]}
 * with one entry per line; the workload name is any caller-chosen label of at
 * most 200 characters without quotes, backslashes or control characters.
 *   sieve_tune_cache_store: writes the context's current options (with `ms`,
 *     the tuned time, for information) under this device and workload,
 *     replacing an entry with the same key and keeping the others; the file
 *     is written to path + ".tmp" and renamed over path.
 *   sieve_tune_cache_load: if the file has an entry for this device and
 *     workload, validates it and makes it the context's options (*found = 1,
 *     *ms = its time; ms may be NULL); else leaves the options unchanged with
 *     *found = 0 (a missing file is not an error).
 * Errors: INVALID (NULL argument, bad name, unwritable file, invalid entry),
 * CUDA. */
int sieve_tune_cache_store(sieve_ctx *ctx, const char *path, const char *workload, double ms);
int sieve_tune_cache_load(sieve_ctx *ctx, const char *path, const char *workload, int *found, double *ms);

/* ------------------------------------------------------------- serving */

/* A request loop with continuous batching on top of sieve_range_batch's
 * machinery.  Clients submit [lo, hi) queries from any thread; a server
 * thread forms batches from the admitted requests and runs each as one
 * batched launch on one of two streams, so that a batch formed while another
 * is on the GPU overlaps it (the paper's per-chunk workers, Sections 2.2-2.3,
 * fed from a queue instead of a fixed split).  Results stay on the device
 * until collected.
 *
 * Admission is by device memory: a list-mode request reserves, at submit, room
 * for the largest possible answer (min(2 ceil(w/6) + 2, 2 w / ln w + 64)
 * primes for width w; the second is the Montgomery-Vaughan bound with slack)
 * in a device pool of pool_bytes, and returns it when collected.  A full pool
 * or queue makes submit return SIEVE_ERR_BUSY (nothing is queued; retry
 * later).  While a server runs on a context, make no other call on that
 * context. */
typedef struct {
  size_t pool_bytes;           /* device pool for list results awaiting collection        */
  size_t max_batch;            /* requests per batch (0: 4096)                             */
  size_t max_queue;            /* admitted requests waiting for a batch (0: 65536)         */
  size_t batch_scratch_bytes;  /* scratch a batch may plan for; a request above it runs
                                  alone (0: 1 GiB)                                         */
} sieve_server_config;

typedef struct {
  uint64_t completed;           /* requests answered since start or the last reset        */
  uint64_t rejected;            /* submits refused with SIEVE_ERR_BUSY                    */
  uint64_t batches;             /* batches launched                                       */
  uint64_t overlapped_batches;  /* batches launched while the other stream was busy       */
  uint64_t queued;              /* requests admitted and waiting now                      */
  uint64_t pool_used_bytes;     /* pool reserved now                                      */
  double mean_batch;            /* requests per batch                                     */
  double p50_us, p99_us, mean_us, max_us;  /* submit-to-result latency of completed requests */
} sieve_server_stats;

/* Start a server on ctx (config NULL: defaults with no pool, i.e. count mode
 * only).  Errors: INVALID, OOM, CUDA. */
int sieve_server_start(sieve_ctx *ctx, const sieve_server_config *config, sieve_server **srv);
/* Admit one query; *req_id identifies it.  INVALID / RANGE for a bad query,
 * CAPACITY if its list could never fit the pool, BUSY for backpressure. */
int sieve_server_submit(sieve_server *srv, uint64_t lo, uint64_t hi, int mode, uint64_t *req_id);
/* SIEVE_PENDING while the request is queued or on the GPU.  When done: fills
 * *cnt (may be NULL) and *n_out (may be NULL), copies a list-mode answer to
 * out[0..n) (host memory, or device memory with SIEVE_OUT_DEVICE), releases
 * the request and returns SIEVE_OK.  A too-small cap returns CAPACITY with
 * *n_out set and keeps the request for another poll.  NOT_FOUND for an unknown
 * or already collected id. */
int sieve_server_poll(sieve_server *srv, uint64_t req_id, sieve_count_result *cnt, uint64_t *out, size_t cap,
                      size_t *n_out, unsigned flags);
/* Id of a request that finished since the last call (in completion order),
 * waiting up to timeout_us microseconds; SIEVE_PENDING if none. */
int sieve_server_next_done(sieve_server *srv, uint64_t *req_id, int timeout_us);
/* Counters and latency percentiles; reset != 0 clears them afterwards. */
int sieve_server_get_stats(sieve_server *srv, sieve_server_stats *st, int reset);
/* Finish every admitted request, then stop the thread and free the server
 * (uncollected results are dropped).  NULL is ignored. */
void sieve_server_stop(sieve_server *srv);

/* ------------------------------------------------------------- no allocation */

/* Size of the fixed device scratch array used by sieve_range_list_noalloc. */
#define SIEVE_NOALLOC_SCRATCH_BYTES (16u << 20)

/* The paper has no counterpart to this call; it exists for callers that
 * cannot allocate device memory when they need primes -- a process whose
 * device memory belongs to another allocator, a latency-critical thread that
 * must not pay for cudaMalloc / cudaFree (cudaFree synchronizes the device),
 * a fixed memory budget.
 *
 * Same result as sieve_range(ctx, lo, hi, SIEVE_LIST, cnt, out, cap, n_out,
 * SIEVE_OUT_DEVICE): the primes in [lo, hi), increasing, as uint64 in the
 * caller's DEVICE buffer out[0..cap), *n_out = their number, *cnt (host, may
 * be NULL) = count and checksum.  It allocates nothing: no cudaMalloc,
 * cudaFree or allocating library routine.  It uses the context's base table
 * and accumulators and, as scratch for per-tile bitmaps, counts and offsets,
 * one file-scope device array of SIEVE_NOALLOC_SCRATCH_BYTES that every GPU
 * loading the library holds until exit.  The array's device address is looked
 * up (cudaGetSymbolAddress, with the context's device current) by sieve_create,
 * which is also when the array is made under lazy module loading; the entry
 * point itself does no set-up.  The bitmaps take one bit per candidate, about
 * one byte per 24 numbers: with the default tile length (2^19 candidates per
 * class) a call covers any range of at most 399,507,452 numbers; a wider
 * range returns SIEVE_ERR_INVALID with a message giving the limit for the
 * context's tile length.  It does not presieve (the presieve patterns are
 * allocated on demand by the other calls), so it is slower than sieve_range.
 *
 * All calls share the one array and it keeps the previous call's contents
 * (each call writes every entry it reads).  Calls that overlap on the GPU (on
 * different streams, contexts or threads) race and give wrong results.
 * Errors: INVALID, RANGE, CAPACITY (nothing written when the list does not
 * fit), CUDA. */
int sieve_range_list_noalloc(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out, size_t cap,
                             size_t *n_out, sieve_count_result *cnt);

/* ------------------------------------------------------------- measurement */

/* The paper has no counterpart to this call; it measures the device resource
 * that bounds the strike loops, for roofline reporting: the throughput of
 * 32-bit shared-memory atomic AND, in lane operations per SM per clock, with
 * one CTA of 1024 threads per SM issuing 4096 atomics per thread into 128 KB
 * of shared memory -- conflict-free (lane l always on bank l) and at
 * pseudo-random words.  Times the slowest SM with clock64, so the result does
 * not depend on the clock.  Runs on the legacy default stream of `device`
 * and synchronises it.  Errors: INVALID, CUDA, OOM. */
int sieve_measure_smem_atomics(int device, double *conflict_free, double *random_banks);

/* ------------------------------------------------------------- phase timing */

/* Device time of the phases of the last call on this context that reached
 * the tile kernel (sieve_count, sieve_primes, sieve_primes_u32, sieve_range,
 * sieve_segment_counts) or a batch graph (sieve_range_batch), measured with
 * CUDA events on the context's stream while phase timing is enabled (it is
 * off by default; the events cost a few microseconds per call), and a batch
 * call's host planning time.  The paper has no counterpart: this backs the
 * roofline figures of the tile kernel, the list compaction and the batch. */
typedef struct {
  double sieve_ms;    /* the tile kernel: strikes, count, bitmap write-out in list mode
                         (sieve_range_batch: the batch's whole graph, upload to compaction) */
  double scan_ms;     /* list mode: the scan of per-tile counts (0 otherwise) */
  double compact_ms;  /* list mode: the compaction kernel (0 otherwise) */
  uint64_t tiles;     /* tiles the tile kernel sieved */
  uint64_t tile_len;  /* indices per residue class per tile */
  uint64_t listed;    /* list mode: primes the compaction wrote */
  uint64_t bucket_waves; /* waves of the bucket sieve (0: not used) */
  uint64_t cluster_ctas; /* CTAs per cluster of the cluster segments (0: not used) */
  double batch_plan_ms;  /* sieve_range_batch: host time of planning the batch (work items,
                            their cost order, the plan buffer) and preparing its buffers */
} sieve_phase_times;

/* enable != 0 turns phase timing on (creating the events), 0 turns it off.
 * Errors: INVALID (NULL ctx), CUDA. */
int sieve_set_phase_timing(sieve_ctx *ctx, int enable);
/* Waits for the last call's recorded events and fills *out; phases the call
 * did not run read 0.  INVALID if ctx or out is NULL or timing is off. */
int sieve_get_phase_times(sieve_ctx *ctx, sieve_phase_times *out);

/* ------------------------------------------------------------- table 1 */

/* Host evaluation of the start-index routine the kernels run (Section 3,
 * Table 1, with the P^2 start of Section 2.4).  For a segment whose index 0
 * stands for value B (B % 6 == 0; index i of class r stands for B + 6 i + r),
 * a start value M >= B and a prime P >= 5: *id1 / *id5 receive the smallest
 * index i with B + 6 i + 1 (resp. + 5) a multiple of P that is >= max(M, P^2).
 * INVALID if B % 6 != 0, M < B, P < 5 or P % 6 not in {1, 5}. */
int sieve_table1_start(uint64_t B, uint64_t M, uint32_t P, int64_t *id1, int64_t *id5);

/* Host evaluation of the other start-index routine the kernels run: the
 * per-tile starts of Section 3 for a tile whose index 0 stands for value B
 * (M = B), from a per-prime inverse of 6 instead of Table 1's case split.
 * Index k of class r stands for 6 (B / 6 + k) + r, which P divides iff
 * B / 6 + k = -r / 6 (mod P), so the first such k is
 * (c_r - (B / 6) mod P) mod P with c_r = (-r / 6) mod P (in closed form:
 * with R = floor(P / 6), (c_1, c_5) = (R, 5R) for P = 6R + 1 and (5R + 4, R)
 * for P = 6R + 5).  The tiles' one-lane strike band and the batch strips use
 * it whenever P^2 <= B (then it equals Table 1's start).
 * Requires B % 6 == 0, 5 <= P < 2^31, P % 6 in {1, 5} and P^2 <= B, else
 * INVALID. */
int sieve_inverse6_start(uint64_t B, uint32_t P, uint32_t *id1, uint32_t *id5);

#ifdef __cplusplus
}
#endif

#endif /* SIEVE_GB300_H */
