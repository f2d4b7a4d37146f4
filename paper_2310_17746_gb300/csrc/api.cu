// api.cu -- context lifetime, the device-resident base table, the wheel
// pattern, and the public range calls of sieve.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "sieve_internal.cuh"

namespace sieve {

// ---------------------------------------------------------------- errors

static thread_local char g_err[512];

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? SIEVE_ERR_OOM : SIEVE_ERR_CUDA;
}

// ---------------------------------------------------------------- helpers

uint64_t isqrt_u64(uint64_t n) {
  // the double square root is within a few units of the integer root (its
  // rounding matters only near 2^53 and above); exact 128-bit products settle it
  uint64_t x = (uint64_t)std::sqrt((double)n);
  if (x > 0xFFFFFFFFull) x = 0xFFFFFFFFull;
  while (x > 0 && (unsigned __int128)x * x > n) x--;
  while ((unsigned __int128)(x + 1) * (x + 1) <= n) x++;
  return x;
}

uint32_t host_prime_count_le_table(const DeviceTable &t, uint64_t s) {
  const uint32_t *b = t.host_primes, *e = t.host_primes + t.nprimes;
  if (s >= 0xFFFFFFFFull) return t.nprimes;
  const uint64_t j = s >> kCountIndexShift;
  if (t.count_idx && j + 1 < t.count_idx_n) {  // only the bucket holding s: the primes below it are <= s,
    e = t.host_primes + t.count_idx[j + 1];    // the primes above it > s
    b = t.host_primes + t.count_idx[j];
  }
  return (uint32_t)(std::upper_bound(b, e, (uint32_t)s) - t.host_primes);
}

// Build the context table's prime-count index over values up to its limit.
static void build_count_index(sieve_ctx *c) {
  const uint64_t n = (c->table.limit >> kCountIndexShift) + 2;
  c->h_count_idx.assign(n, 0);
  const size_t np = c->h_primes.size();
  size_t i = 0;
  for (uint64_t j = 0; j < n; j++) {
    const uint64_t v = j << kCountIndexShift;
    while (i < np && c->h_primes[i] < v) i++;
    c->h_count_idx[j] = (uint32_t)i;
  }
  c->table.count_idx = c->h_count_idx.data();
  c->table.count_idx_n = n;
}

int ensure_scratch(sieve_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->scratch_bytes) return SIEVE_OK;
  if (ctx->d_scratch) {
    SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_scratch);
    ctx->d_scratch = nullptr;
    ctx->scratch_bytes = 0;
  }
  size_t grow = bytes + bytes / 4;
  SIEVE_CUDA_TRY(cudaMalloc(&ctx->d_scratch, grow));
  ctx->scratch_bytes = grow;
  return SIEVE_OK;
}

int ensure_stage(sieve_ctx *ctx, size_t bytes) {
  if (bytes <= ctx->stage_bytes) return SIEVE_OK;
  if (ctx->d_stage) {
    SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_stage);
    ctx->d_stage = nullptr;
    ctx->stage_bytes = 0;
  }
  SIEVE_CUDA_TRY(cudaMalloc(&ctx->d_stage, bytes));
  ctx->stage_bytes = bytes;
  return SIEVE_OK;
}

// Presieve pattern g in the sliced layout for tiles of W words per class: word
// j holds, at bit b, whether 6 x + r (x = (j + b W) mod period) has no factor
// among the pattern's primes.  Words run to period + W so that a tile's W
// words starting at any phase below the period are contiguous.
struct SlicedGenArgs {
  uint32_t period, W, words, off1, off5;
  uint32_t primes[6];  // 0 = unused
};

__global__ void sliced_pattern_kernel(uint32_t *pat, const SlicedGenArgs a) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.words) return;
  uint32_t w1 = 0, w5 = 0;
  for (uint32_t b = 0; b < 32; b++) {
    const uint32_t x = (uint32_t)(((uint64_t)j + (uint64_t)b * a.W) % a.period);
    const uint64_t v1 = 6ull * x + 1, v5 = 6ull * x + 5;
    bool c1 = true, c5 = true;
#pragma unroll
    for (int q = 0; q < 6; q++) {
      if (a.primes[q] == 0) continue;
      c1 = c1 && (v1 % a.primes[q] != 0);
      c5 = c5 && (v5 % a.primes[q] != 0);
    }
    w1 |= (uint32_t)c1 << b;
    w5 |= (uint32_t)c5 << b;
  }
  pat[a.off1 + j] = w1;
  pat[a.off5 + j] = w5;
}

// Per-prime constants of the base table: the invariant-division reciprocal
// and the inverse-of-6 start constants.
__global__ void reciprocal_kernel(const uint32_t *__restrict__ primes, uint64_t *__restrict__ magic,
                                  uint2 *__restrict__ cinv, uint32_t n) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    magic[i] = reciprocal64(primes[i]);
    cinv[i] = inverse6_constants(primes[i]);
  }
}

// Host Eratosthenes for the first, small part of the base table.
static std::vector<uint32_t> host_small_primes(uint32_t n) {
  std::vector<uint8_t> a(n + 1, 1);
  std::vector<uint32_t> out;
  a[0] = 0;
  if (n >= 1) a[1] = 0;
  for (uint64_t i = 2; i * i <= n; i++)
    if (a[i])
      for (uint64_t j = i * i; j <= n; j += i) a[j] = 0;
  for (uint32_t i = 2; i <= n; i++)
    if (a[i]) out.push_back(i);
  return out;
}

// Upper bound on pi(x) for x >= 17 (Rosser & Schoenfeld 1962: pi(x) <
// 1.25506 x / ln x for x > 1), with slack.
static uint64_t pi_upper(uint64_t x) {
  if (x < 100) return 30;
  double lx = __builtin_log((double)x);
  return (uint64_t)(1.25506 * (double)x / lx) + 64;
}

int sliced_patterns(sieve_ctx *ctx, uint32_t logW, const uint32_t **ptr, PatternDesc *pd) {
  if (logW >= 32) {
    set_error("tile width out of range");
    return SIEVE_ERR_INVALID;
  }
  auto &ss = ctx->sliced[logW];
  if (!ss.d) {
    const uint32_t W = 1u << logW;
    uint64_t total = 0;
    PatternDesc d[kNumPatterns];
    for (int g = 0; g < kNumPatterns; g++) {
      const uint32_t words = pattern_period(g) + W + 32;
      d[g].period = pattern_period(g);
      d[g].off1 = (uint32_t)total;
      d[g].off5 = (uint32_t)(total + words);
      d[g].pad_ = 0;
      d[g].magic = reciprocal64(pattern_period(g));
      total += 2ull * words;
    }
    uint32_t *buf = nullptr;
    SIEVE_CUDA_TRY(cudaMalloc(&buf, total * sizeof(uint32_t)));
    for (int g = 0; g < kNumPatterns; g++) {
      SlicedGenArgs a;
      a.period = d[g].period;
      a.W = W;
      a.words = d[g].period + W + 32;
      a.off1 = d[g].off1;
      a.off5 = d[g].off5;
      for (int q = 0; q < 6; q++) a.primes[q] = kPatternPrimes[g][q];
      sliced_pattern_kernel<<<(a.words + 255) / 256, 256, 0, ctx->stream>>>(buf, a);
      ctx->launches++;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) {
        cudaFree(buf);
        return cuda_fail(e, "sliced_pattern_kernel");
      }
    }
    ss.d = buf;
    for (int g = 0; g < kNumPatterns; g++) ss.pd[g] = d[g];
  }
  *ptr = ss.d;
  for (int g = 0; g < kNumPatterns; g++) pd[g] = ss.pd[g];
  return SIEVE_OK;
}

int ensure_pattern_set_dev(sieve_ctx *ctx, uint32_t logW) {
  if (logW >= 32) {
    set_error("tile width out of range");
    return SIEVE_ERR_INVALID;
  }
  if (ctx->psets_ready & (1u << logW)) return SIEVE_OK;
  if (!ctx->d_psets) SIEVE_CUDA_TRY(cudaMalloc(&ctx->d_psets, 32 * sizeof(PatternSetDev)));
  PatternSetDev ps;
  int rc = sliced_patterns(ctx, logW, &ps.d, ps.pd);
  if (rc != SIEVE_OK) return rc;
  // synchronous copy: ps lives on this stack frame
  SIEVE_CUDA_TRY(cudaMemcpyAsync(ctx->d_psets + logW, &ps, sizeof(ps), cudaMemcpyHostToDevice, ctx->stream));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
  ctx->psets_ready |= 1u << logW;
  return SIEVE_OK;
}

}  // namespace sieve

using namespace sieve;

// ---------------------------------------------------------------- context

static void free_ctx(sieve_ctx *c) {
  if (!c) return;
  destroy_batch_runner(c->batch);
  cudaFree(c->d_psets);
  cudaFree(c->d_primes);
  cudaFree(c->d_magic);
  cudaFree(c->d_cinv);
  for (auto &ss : c->sliced) cudaFree(ss.d);
  cudaFree(c->d_acc);
  cudaFree(c->d_scratch);
  cudaFree(c->d_stage);
  cudaFree(c->d_bucket);
  if (c->h_acc) cudaFreeHost(c->h_acc);
  for (cudaEvent_t &e : c->ph_ev)
    if (e) cudaEventDestroy(e);
  delete c;
}

static sieve_options default_options() {
  sieve_options o;
  memset(&o, 0, sizeof(o));
  o.tile_bits = 1u << 19;
  o.block_threads = 1024;
  o.ctas_per_sm = 0;
  o.group_hits = 5;       // measured best with presieve_groups 7 at [2, 1e12] (181.4 ms; 4: 182.1, 8: 184.1)
  o.presieve_groups = 7;  // patterns to 109
  o.batch_tile_bits = 1u << 18;
  o.chunk_primes = 1u << 15;
  o.bucket_threshold = 4;  // primes above 4 L through the bucket sieve, where it pays (measured best of 1..16)
  o.bucket_wave = 1;
  o.bucket_scatter = 0;    // direct or sorted scatter by the size of a wave's buckets
  o.list_single_pass = 0;  // one pass measured slower: 8.25 vs 6.84 ms for the uint64 list of [1e12, 1e12+2e10)
  o.cluster_ctas = 0;      // cluster segments off: slower than the bucket sieve ([1e16, +1e10): 19.9 vs 8.5 ms)
  o.cluster_threshold = 4;  // measured best of 4 / 16 / 64 with 8 and 16 CTAs per cluster
  return o;
}

static int validate_options(const sieve_ctx *c, const sieve_options &o) {
  if (o.tile_bits < 1024 || (o.tile_bits & (o.tile_bits - 1)) || o.tile_bits > (1u << 20)) {
    set_error("tile_bits must be a power of two in [1024, 2^19]");
    return SIEVE_ERR_INVALID;
  }
  if ((int)(o.tile_bits / 4) > c->smem_optin) {
    set_error("tile_bits %u needs %u bytes of shared memory; the device allows %d", o.tile_bits,
              o.tile_bits / 4, c->smem_optin);
    return SIEVE_ERR_INVALID;
  }
  if (o.block_threads != 256 && o.block_threads != 512 && o.block_threads != 1024) {
    set_error("block_threads must be 256, 512 or 1024");
    return SIEVE_ERR_INVALID;
  }
  if (o.ctas_per_sm > 32) {
    set_error("ctas_per_sm must be <= 32");
    return SIEVE_ERR_INVALID;
  }
  if (o.group_hits == 0 || o.group_hits > 1024) {
    set_error("group_hits must be in [1, 1024]");
    return SIEVE_ERR_INVALID;
  }
  if (o.batch_tile_bits && (o.batch_tile_bits < 1024 || (o.batch_tile_bits & (o.batch_tile_bits - 1)) ||
                            o.batch_tile_bits > (1u << 19) || (int)(o.batch_tile_bits / 4) > c->smem_optin)) {
    set_error("batch_tile_bits must be 0 or a power of two in [1024, 2^19] that fits in shared memory");
    return SIEVE_ERR_INVALID;
  }
  if (o.chunk_primes < 1024) {
    set_error("chunk_primes must be >= 1024");
    return SIEVE_ERR_INVALID;
  }
  if (o.bucket_threshold > 64) {
    set_error("bucket_threshold must be in [0, 64]");
    return SIEVE_ERR_INVALID;
  }
  if (o.list_single_pass > 1) {
    set_error("list_single_pass must be 0 or 1");
    return SIEVE_ERR_INVALID;
  }
  if (o.bucket_scatter > 2) {
    set_error("bucket_scatter must be 0 (automatic), 1 (direct) or 2 (sorted)");
    return SIEVE_ERR_INVALID;
  }
  if (o.bucket_wave < 1 || o.bucket_wave > 16) {
    set_error("bucket_wave must be in [1, 16]");
    return SIEVE_ERR_INVALID;
  }
  if (o.cluster_ctas != 0 && o.cluster_ctas != 2 && o.cluster_ctas != 4 && o.cluster_ctas != 8 &&
      o.cluster_ctas != 16) {
    set_error("cluster_ctas must be 0 (off), 2, 4, 8 or 16");
    return SIEVE_ERR_INVALID;
  }
  if (o.cluster_threshold > 1024) {
    set_error("cluster_threshold must be in [0, 1024]");
    return SIEVE_ERR_INVALID;
  }
  if (o.presieve_groups > (uint32_t)kMaxPresieveGroups) {
    set_error("presieve_groups must be in [0, %d]", kMaxPresieveGroups);
    return SIEVE_ERR_INVALID;
  }
  return SIEVE_OK;
}

static int build_base_table(sieve_ctx *c, uint64_t limit) {
  // Section 2.4 / Section 4: the sieving primes are only those up to the
  // square root; they are themselves found incrementally.  Primes <= sqrt(limit)
  // come from a host sieve, the rest from this library's GPU sieve using them.
  const uint32_t small_n = (uint32_t)isqrt_u64(limit) + 1;
  std::vector<uint32_t> small = host_small_primes(small_n);
  const uint64_t cap = pi_upper(limit);
  SIEVE_CUDA_TRY(cudaMalloc(&c->d_primes, cap * sizeof(uint32_t)));
  SIEVE_CUDA_TRY(cudaMalloc(&c->d_magic, cap * sizeof(uint64_t)));
  SIEVE_CUDA_TRY(cudaMalloc(&c->d_cinv, cap * sizeof(uint2)));
  SIEVE_CUDA_TRY(cudaMemcpyAsync(c->d_primes, small.data(), small.size() * sizeof(uint32_t),
                                 cudaMemcpyHostToDevice, c->stream));
  const uint32_t ns = (uint32_t)small.size();
  reciprocal_kernel<<<(ns + 255) / 256, 256, 0, c->stream>>>(c->d_primes, c->d_magic, c->d_cinv, ns);
  c->launches++;
  SIEVE_CUDA_TRY(cudaGetLastError());

  DeviceTable t0;
  t0.primes = c->d_primes;
  t0.magic = c->d_magic;
  t0.cinv = c->d_cinv;
  t0.host_primes = small.data();
  t0.nprimes = ns;
  t0.limit = small_n;
  uint64_t total = ns;
  if (limit > small_n) {
    RangeRequest rq;
    rq.lo = (uint64_t)small_n + 1;
    rq.hi = limit + 1;
    rq.list = 1;
    rq.out_bytes = 4;
    rq.out = c->d_primes + ns;
    rq.cap = cap - ns;
    rq.out_on_device = 1;
    size_t n = 0;
    int rc = run_range(c, t0, rq, &n);
    if (rc != SIEVE_OK) return rc;
    total += n;
    if (n) {
      reciprocal_kernel<<<(uint32_t)((n + 255) / 256), 256, 0, c->stream>>>(c->d_primes + ns, c->d_magic + ns,
                                                                           c->d_cinv + ns, (uint32_t)n);
      c->launches++;
      SIEVE_CUDA_TRY(cudaGetLastError());
    }
  }
  c->h_primes.resize(total);
  SIEVE_CUDA_TRY(cudaMemcpyAsync(c->h_primes.data(), c->d_primes, total * sizeof(uint32_t),
                                 cudaMemcpyDeviceToHost, c->stream));
  SIEVE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  c->table.primes = c->d_primes;
  c->table.magic = c->d_magic;
  c->table.cinv = c->d_cinv;
  c->table.host_primes = c->h_primes.data();
  c->table.nprimes = (uint32_t)total;
  c->table.limit = limit;
  build_count_index(c);
  return SIEVE_OK;
}

namespace sieve {

// Grow the base table to every prime <= new_limit (Section 2.4: the sieving
// primes are found incrementally -- the current table, complete up to L,
// sieves (L, new_limit] as long as new_limit <= L^2).  The table moves to new
// device arrays; kernels launched earlier have completed (the stream is
// synchronised first) and batch runners notice the new table epoch.
int extend_base_table(sieve_ctx *c, uint64_t new_limit) {
  const uint64_t L = c->table.limit;
  if (new_limit <= L) return SIEVE_OK;
  if (new_limit > L * L) new_limit = L * L;
  if (new_limit > 0xFFFFFFFFull) new_limit = 0xFFFFFFFFull;
  const uint64_t cap = pi_upper(new_limit);
  uint32_t *np_ = nullptr;
  uint64_t *nm = nullptr;
  uint2 *nc = nullptr;
  SIEVE_CUDA_TRY(cudaStreamSynchronize(c->stream));
  SIEVE_CUDA_TRY(cudaMalloc(&np_, cap * sizeof(uint32_t)));
  cudaError_t e = cudaMalloc(&nm, cap * sizeof(uint64_t));
  if (e == cudaSuccess) e = cudaMalloc(&nc, cap * sizeof(uint2));
  if (e != cudaSuccess) {
    cudaFree(np_);
    cudaFree(nm);
    return cuda_fail(e, "cudaMalloc (base table)");
  }
  const uint32_t n0 = c->table.nprimes;
  int rc = SIEVE_OK;
  size_t n = 0;
  do {
    if ((e = cudaMemcpyAsync(np_, c->d_primes, n0 * sizeof(uint32_t), cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(nm, c->d_magic, n0 * sizeof(uint64_t), cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(nc, c->d_cinv, n0 * sizeof(uint2), cudaMemcpyDeviceToDevice, c->stream)) !=
            cudaSuccess) {
      rc = cuda_fail(e, "cudaMemcpyAsync (base table)");
      break;
    }
    RangeRequest rq;
    rq.lo = L + 1;
    rq.hi = new_limit + 1;
    rq.list = 1;
    rq.out_bytes = 4;
    rq.out = np_ + n0;
    rq.cap = cap - n0;
    rq.out_on_device = 1;
    if ((rc = run_range(c, c->table, rq, &n)) != SIEVE_OK) break;
    if (n) {
      reciprocal_kernel<<<(uint32_t)((n + 255) / 256), 256, 0, c->stream>>>(np_ + n0, nm + n0, nc + n0,
                                                                           (uint32_t)n);
      c->launches++;
      if ((e = cudaGetLastError()) != cudaSuccess) {
        rc = cuda_fail(e, "reciprocal_kernel");
        break;
      }
    }
    c->h_primes.resize(n0 + n);
    if ((e = cudaMemcpyAsync(c->h_primes.data() + n0, np_ + n0, n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess ||
        (e = cudaStreamSynchronize(c->stream)) != cudaSuccess) {
      rc = cuda_fail(e, "base table read-back");
      break;
    }
  } while (0);
  if (rc != SIEVE_OK) {
    c->h_primes.resize(n0);
    c->table.host_primes = c->h_primes.data();  // the resize above may have moved the host copy
    cudaFree(np_);
    cudaFree(nm);
    cudaFree(nc);
    return rc;
  }
  cudaFree(c->d_primes);
  cudaFree(c->d_magic);
  cudaFree(c->d_cinv);
  c->d_primes = np_;
  c->d_magic = nm;
  c->d_cinv = nc;
  c->table.primes = np_;
  c->table.magic = nm;
  c->table.cinv = nc;
  c->table.host_primes = c->h_primes.data();
  c->table.nprimes = (uint32_t)(n0 + n);
  c->table.limit = new_limit;
  build_count_index(c);
  c->max_hi = new_limit >= 0xB504F333ull ? (1ull << 63) : (new_limit + 1) * (new_limit + 1);
  c->table_epoch++;
  return SIEVE_OK;
}

}  // namespace sieve

extern "C" int sieve_create(sieve_ctx **ctx, uint64_t max_hi, int device, void *cuda_stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  *ctx = nullptr;
  if (max_hi < 2 || max_hi > (1ull << 63)) {
    set_error("max_hi must be in [2, 2^63]");
    return SIEVE_ERR_INVALID;
  }
  sieve_ctx *c = new (std::nothrow) sieve_ctx();
  if (!c) {
    set_error("host allocation failed");
    return SIEVE_ERR_OOM;
  }
  int rc = SIEVE_OK;
  do {
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "cudaSetDevice");
      break;
    }
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->max_hi = max_hi;
    if ((e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess ||
        (e = cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device)) !=
            cudaSuccess) {
      rc = cuda_fail(e, "cudaDeviceGetAttribute");
      break;
    }
    // keep room for the kernels' static shared memory
    c->smem_optin -= 2048;
    if ((rc = range_set_smem_attributes(c->smem_optin)) != SIEVE_OK) break;
    c->opt = default_options();
    while (c->opt.tile_bits / 4 > (uint32_t)c->smem_optin) c->opt.tile_bits /= 2;
    c->acc_words = 16;
    if ((e = cudaMalloc(&c->d_acc, c->acc_words * sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMallocHost(&c->h_acc, c->acc_words * sizeof(unsigned long long))) != cudaSuccess) {
      rc = cuda_fail(e, "context allocation");
      break;
    }
    // the no-allocation entry point's scratch address, with the device current
    if ((rc = noalloc_setup(c)) != SIEVE_OK) break;
    const uint64_t limit = std::max<uint64_t>(isqrt_u64(max_hi - 1), 1u << 16);
    rc = build_base_table(c, limit);
  } while (0);
  if (rc != SIEVE_OK) {
    free_ctx(c);
    return rc;
  }
  *ctx = c;
  return SIEVE_OK;
}

extern "C" void sieve_destroy(sieve_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  free_ctx(ctx);
}

extern "C" int sieve_set_stream(sieve_ctx *ctx, void *cuda_stream) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  ctx->stream = (cudaStream_t)cuda_stream;
  return SIEVE_OK;
}

extern "C" int sieve_get_options(const sieve_ctx *ctx, sieve_options *opt) {
  if (!ctx || !opt) {
    set_error("NULL argument");
    return SIEVE_ERR_INVALID;
  }
  *opt = ctx->opt;
  return SIEVE_OK;
}

extern "C" int sieve_set_options(sieve_ctx *ctx, const sieve_options *opt) {
  if (!ctx || !opt) {
    set_error("NULL argument");
    return SIEVE_ERR_INVALID;
  }
  int rc = validate_options(ctx, *opt);
  if (rc != SIEVE_OK) return rc;
  ctx->opt = *opt;
  return SIEVE_OK;
}

extern "C" int sieve_base_table(const sieve_ctx *ctx, uint64_t *limit, uint64_t *nprimes,
                                const uint32_t **device_primes) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  if (limit) *limit = ctx->table.limit;
  if (nprimes) *nprimes = ctx->table.nprimes;
  if (device_primes) *device_primes = ctx->table.primes;
  return SIEVE_OK;
}

extern "C" uint64_t sieve_launch_count(const sieve_ctx *ctx) { return ctx ? ctx->launches.load() : 0; }

extern "C" int sieve_set_phase_timing(sieve_ctx *ctx, int enable) {
  if (!ctx) {
    set_error("sieve_set_phase_timing: NULL context");
    return SIEVE_ERR_INVALID;
  }
  if (enable) {
    SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
    for (cudaEvent_t &e : ctx->ph_ev)
      if (!e) SIEVE_CUDA_TRY(cudaEventCreate(&e));
  }
  ctx->phase_timing = enable != 0;
  ctx->ph_recorded = 0;
  ctx->ph = sieve_phase_times{};
  return SIEVE_OK;
}

extern "C" int sieve_get_phase_times(sieve_ctx *ctx, sieve_phase_times *out) {
  if (!ctx || !out || !ctx->phase_timing) {
    set_error("sieve_get_phase_times: NULL argument or phase timing off");
    return SIEVE_ERR_INVALID;
  }
  sieve_phase_times t = ctx->ph;
  const uint32_t r = ctx->ph_recorded;
  const int from[3] = {0, 1, 3}, to[3] = {1, 2, 4};
  double *dst[3] = {&t.sieve_ms, &t.scan_ms, &t.compact_ms};
  for (int i = 0; i < 3; i++) {
    if ((r & (1u << from[i])) == 0 || (r & (1u << to[i])) == 0) continue;
    float ms = 0.0f;
    SIEVE_CUDA_TRY(cudaEventSynchronize(ctx->ph_ev[to[i]]));
    SIEVE_CUDA_TRY(cudaEventElapsedTime(&ms, ctx->ph_ev[from[i]], ctx->ph_ev[to[i]]));
    *dst[i] = ms;
  }
  *out = t;
  return SIEVE_OK;
}

extern "C" const char *sieve_last_error(void) { return g_err; }

// ---------------------------------------------------------------- range calls

static int enter(sieve_ctx *ctx) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  g_err[0] = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return SIEVE_OK;
}

extern "C" int sieve_count(sieve_ctx *ctx, uint64_t n, sieve_count_result *out) {
  int rc = enter(ctx);
  if (rc != SIEVE_OK) return rc;
  if (!out) {
    set_error("out is NULL");
    return SIEVE_ERR_INVALID;
  }
  if (n >= (1ull << 63)) {
    set_error("n must be < 2^63");
    return SIEVE_ERR_RANGE;
  }
  RangeRequest rq;
  rq.lo = 0;
  rq.hi = n + 1;
  rq.total = out;
  return run_range(ctx, ctx->table, rq, nullptr);
}

static int primes_common(sieve_ctx *ctx, uint64_t n, void *out, size_t cap, size_t *n_out, unsigned flags,
                         int bytes) {
  int rc = enter(ctx);
  if (rc != SIEVE_OK) return rc;
  if (!n_out || (!out && cap)) {
    set_error("NULL argument");
    return SIEVE_ERR_INVALID;
  }
  if (bytes == 4 && n > 0xFFFFFFFFull) {
    set_error("uint32 output needs n < 2^32");
    return SIEVE_ERR_INVALID;
  }
  if (n >= (1ull << 63)) {
    set_error("n must be < 2^63");
    return SIEVE_ERR_RANGE;
  }
  RangeRequest rq;
  rq.lo = 0;
  rq.hi = n + 1;
  rq.list = 1;
  rq.out_bytes = bytes;
  rq.out = out;
  rq.cap = cap;
  rq.out_on_device = (flags & SIEVE_OUT_DEVICE) != 0;
  return run_range(ctx, ctx->table, rq, n_out);
}

extern "C" int sieve_primes(sieve_ctx *ctx, uint64_t n, uint64_t *out, size_t cap, size_t *n_out,
                            unsigned flags) {
  return primes_common(ctx, n, out, cap, n_out, flags, 8);
}

extern "C" int sieve_primes_u32(sieve_ctx *ctx, uint64_t n, uint32_t *out, size_t cap, size_t *n_out,
                                unsigned flags) {
  return primes_common(ctx, n, out, cap, n_out, flags, 4);
}

// Whether [lo, hi) is better sieved with strips (batch path) than tile by
// tile: the rule of the batch planner -- locating the primes above the tile
// length once per tile costs more than locating them once and clearing their
// hits with global atomics (priced 4x higher when the range's bitmap would
// not fit half of L2).
namespace sieve {
bool strips_beat_buckets(uint64_t lo, uint64_t hi) {
  if (hi <= lo) return false;
  const uint64_t span = (hi + 4) / 6 - lo / 6;
  return span / 4 <= kStripBitmapL2 && hi - lo >= 300000000ull && isqrt_u64(hi - 1) >= 100000000ull;
}
}  // namespace sieve

static bool strips_pay_off(const sieve_ctx *ctx, uint64_t lo, uint64_t hi) {
  if (hi <= lo || hi > (1ull << 63)) return false;
  const uint64_t s = isqrt_u64(hi - 1);
  if (s > ctx->table.limit) return false;  // run_range reports RANGE
  const uint64_t L = ctx->opt.batch_tile_bits ? ctx->opt.batch_tile_bits : ctx->opt.tile_bits;
  const uint64_t span = (hi + 4) / 6 - lo / 6;
  const uint64_t ntiles = (span + L - 1) / L;
  if (ntiles < 2 || span >= (1ull << 31)) return false;
  const uint32_t np = host_prime_count_le_table(ctx->table, s);
  const uint32_t imid = host_prime_count_le_table(ctx->table, L);
  if (np <= imid + 1) return false;
  const uint32_t *P = ctx->table.host_primes;
  const double large = (double)(np - imid);
  const double hits = 2.0 * (double)span *
                      (std::log(std::log((double)P[np - 1])) - std::log(std::log((double)P[imid])));
  const double gcost = (double)span / 4.0 > 48e6 ? 160.0 : 40.0;
  return 10.0 * large + gcost * hits < 10.0 * large * (double)ntiles;
}

extern "C" int sieve_range(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int mode, sieve_count_result *cnt,
                           uint64_t *out, size_t cap, size_t *n_out, unsigned flags) {
  int rc = enter(ctx);
  if (rc != SIEVE_OK) return rc;
  if (mode != SIEVE_COUNT && mode != SIEVE_LIST) {
    set_error("mode must be SIEVE_COUNT or SIEVE_LIST");
    return SIEVE_ERR_INVALID;
  }
  if (mode == SIEVE_COUNT && !cnt) {
    set_error("cnt is NULL in count mode");
    return SIEVE_ERR_INVALID;
  }
  if (mode == SIEVE_LIST && (!n_out || (!out && cap))) {
    set_error("list mode needs n_out and an output buffer");
    return SIEVE_ERR_INVALID;
  }
  RangeRequest rq;
  rq.lo = lo;
  rq.hi = hi;
  rq.list = mode == SIEVE_LIST;
  rq.out_bytes = 8;
  rq.out = out;
  rq.cap = cap;
  rq.out_on_device = (flags & SIEVE_OUT_DEVICE) != 0;
  rq.total = cnt;
  rq.async = mode == SIEVE_COUNT && (flags & SIEVE_OUT_DEVICE) && (flags & SIEVE_ASYNC);
  // far ranges: the batch path's strips when they pay off and beat the bucket
  // sieve ([1e18, +1e9): 1.2 ms against 2.1 ms), else the bucket sieve where it
  // applies ([1e16, +1e10): 8.6 ms against 22.8 ms through strips)
  // (cluster segments, when asked for, replace both)
  if (!rq.async && ctx->opt.cluster_ctas == 0 && strips_pay_off(ctx, lo, hi) &&
      (strips_beat_buckets(lo, hi) || !range_prefers_buckets(ctx, lo, hi))) {
    // a range far up: run it as a one-query batch, whose planner locates the
    // primes above the tile length once for the whole range (strips) instead
    // of once per tile
    const uint8_t m8 = (uint8_t)mode;
    sieve_count_result local{0, 0};
    uint64_t h_off[2] = {0, 0};
    const bool dev = rq.out_on_device;
    sieve_count_result *c = cnt ? cnt : (dev ? (sieve_count_result *)(ctx->d_acc + 4) : &local);
    uint64_t *offs = dev ? (uint64_t *)(ctx->d_acc + 2) : h_off;
    size_t n = 0;
    rc = sieve_range_batch(ctx, &lo, &hi, &m8, 1, c, offs, mode == SIEVE_LIST ? out : nullptr,
                           mode == SIEVE_LIST ? cap : 0, &n, flags & SIEVE_OUT_DEVICE);
    if (n_out) *n_out = mode == SIEVE_LIST ? n : 0;
    return rc;
  }
  return run_range(ctx, ctx->table, rq, n_out);
}

extern "C" int sieve_segment_counts(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t seg_width,
                                    uint64_t *counts, size_t ncounts, sieve_count_result *total,
                                    unsigned flags) {
  int rc = enter(ctx);
  if (rc != SIEVE_OK) return rc;
  if (seg_width == 0 || (!counts && ncounts)) {
    set_error("seg_width must be > 0 and counts non-NULL");
    return SIEVE_ERR_INVALID;
  }
  RangeRequest rq;
  rq.lo = lo;
  rq.hi = hi;
  rq.seg_width = seg_width;
  rq.bins = counts;
  rq.nbins = ncounts;
  rq.total = total;
  rq.out_on_device = (flags & SIEVE_OUT_DEVICE) != 0;
  rq.async = (flags & SIEVE_OUT_DEVICE) && (flags & SIEVE_ASYNC);
  return run_range(ctx, ctx->table, rq, nullptr);
}

// ---------------------------------------------------------------- table 1 (host)

extern "C" int sieve_inverse6_start(uint64_t B, uint32_t P, uint32_t *id1, uint32_t *id5) {
  if (!id1 || !id5 || B % 6 != 0 || P < 5 || (P % 6 != 1 && P % 6 != 5) || P >= 0x80000000u ||
      (uint64_t)P * P > B || B >= (1ull << 63)) {
    set_error("sieve_inverse6_start: invalid argument");
    return SIEVE_ERR_INVALID;
  }
  starts_from_inverse(B / 6, P, reciprocal64(P), inverse6_constants(P), *id1, *id5);
  return SIEVE_OK;
}

extern "C" int sieve_table1_start(uint64_t B, uint64_t M, uint32_t P, int64_t *id1, int64_t *id5) {
  if (!id1 || !id5 || B % 6 != 0 || M < B || P < 5 || (P % 6 != 1 && P % 6 != 5) ||
      M >= (1ull << 63) || B >= (1ull << 63)) {
    set_error("sieve_table1_start: invalid argument");
    return SIEVE_ERR_INVALID;
  }
  const uint64_t P2 = (uint64_t)P * P;
  const uint64_t Mp = M > P2 ? M : P2;
  if (Mp - B >= (1ull << 62)) {
    set_error("sieve_table1_start: max(M, P^2) - B too large");
    return SIEVE_ERR_INVALID;
  }
  if (M == B) {  // the tile case the kernels evaluate
    uint64_t k1, k5;
    tile_starts(B, P, reciprocal64(P), k1, k5);
    *id1 = (int64_t)k1;
    *id5 = (int64_t)k5;
    return SIEVE_OK;
  }
  StartIndex s = table1_start(B, M, P, reciprocal64(P));
  *id1 = s.id1;
  *id5 = s.id5;
  return SIEVE_OK;
}
