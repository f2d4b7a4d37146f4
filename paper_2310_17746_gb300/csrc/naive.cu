// naive.cu -- the plain GPU sieve: the comparison point for the segmented one.
//
// Section 1.1 / Figure 1 done the direct way on a GPU, one range per call:
// one bit per odd number of [lo, hi) in a bitmap in global memory (no residue
// classes, no presieve, no shared-memory segments, no Table 1), every odd
// multiple m >= max(p^2, lo) of every odd base prime p <= isqrt(hi - 1)
// cleared with a global atomic AND, then a popcount pass (count and sum) or a
// count / scan / write pass (the sorted list).  The work of a prime is split
// over as many CTAs as its multiples need, so that small primes do not
// serialise on one thread; otherwise nothing is arranged for locality.
#include <algorithm>
#include <vector>

#include "sieve_internal.cuh"

namespace sieve {
namespace {

constexpr int kNaiveBlock = 256;
constexpr uint32_t kNaiveStrikesPerThread = 64;
constexpr uint64_t kNaiveStrikesPerBlock = (uint64_t)kNaiveBlock * kNaiveStrikesPerThread;
constexpr uint32_t kNaiveWordsPerThread = 8;  // list pass: each thread owns 8 consecutive words
constexpr uint32_t kNaiveWordsPerBlock = kNaiveBlock * kNaiveWordsPerThread;
const uint64_t kTwo = 2;  // source of the list's first element when 2 is in range

struct NaiveRange {
  uint64_t lo, hi;
  uint64_t olo;    // first odd value >= lo: bit i stands for olo + 2 i
  uint64_t nbits;  // odd values in [lo, hi)
  uint64_t nwords;
};

// First odd multiple of p that is >= max(p^2, lo), for odd p.
__host__ __device__ __forceinline__ uint64_t naive_first_odd_multiple(uint64_t p, uint64_t lo) {
  uint64_t m = (lo + p - 1) / p * p;
  if (m < p * p) m = p * p;
  if ((m & 1) == 0) m += p;
  return m;
}

// Odd multiples of p from its first one below hi.
__host__ __device__ __forceinline__ uint64_t naive_multiples(uint64_t p, uint64_t lo, uint64_t hi) {
  const uint64_t m0 = naive_first_odd_multiple(p, lo);
  return m0 < hi ? (hi - 1 - m0) / (2 * p) + 1 : 0;
}

// Block b strikes for prime primes[i0 + k], k the largest index with
// first_block[k] <= b; its threads take consecutive multiples.
__global__ void __launch_bounds__(kNaiveBlock) naive_strike_kernel(uint32_t *__restrict__ bits, const NaiveRange r,
                                                                    const uint32_t *__restrict__ primes,
                                                                    const uint32_t *__restrict__ first_block,
                                                                    uint32_t i0, uint32_t nk) {
  const uint32_t b = blockIdx.x;
  uint32_t lo = 0, hi = nk;  // first_block[lo] <= b < first_block[hi] (first_block[nk] = grid)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (first_block[mid] <= b) lo = mid;
    else hi = mid;
  }
  const uint64_t p = primes[i0 + lo];
  const uint64_t m0 = naive_first_odd_multiple(p, r.lo);
  const uint64_t n = naive_multiples(p, r.lo, r.hi);
  const uint64_t j0 = (uint64_t)(b - first_block[lo]) * kNaiveStrikesPerBlock;
  for (uint32_t s = 0; s < kNaiveStrikesPerThread; s++) {
    const uint64_t j = j0 + (uint64_t)s * kNaiveBlock + threadIdx.x;
    if (j >= n) break;
    const uint64_t bit = (m0 + 2 * p * j - r.olo) >> 1;
    atomicAnd(bits + (bit >> 5), ~(1u << (bit & 31)));
  }
}

// Word w with the bits past the range and the value 1 cleared.
__device__ __forceinline__ uint32_t naive_word(const uint32_t *__restrict__ bits, const NaiveRange &r, uint64_t w) {
  uint32_t x = bits[w];
  if (w == r.nwords - 1 && (r.nbits & 31)) x &= (1u << (r.nbits & 31)) - 1;
  if (w == 0 && r.olo == 1) x &= ~1u;
  return x;
}

__global__ void __launch_bounds__(kNaiveBlock) naive_count_kernel(const uint32_t *__restrict__ bits,
                                                                   const NaiveRange r,
                                                                   unsigned long long *acc) {
  __shared__ unsigned long long red[2][kNaiveBlock / 32];
  unsigned long long c = 0, s = 0;
  for (uint64_t w = blockIdx.x * (uint64_t)kNaiveBlock + threadIdx.x; w < r.nwords;
       w += (uint64_t)gridDim.x * kNaiveBlock) {
    uint32_t x = naive_word(bits, r, w);
    const uint32_t pc = __popc(x);
    c += pc;
    s += (unsigned long long)pc * (r.olo + 64 * w);
    while (x) {  // + 2 b for every set bit b
      s += 2u * (uint32_t)(__ffs(x) - 1);
      x &= x - 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c += __shfl_down_sync(kFullMask, c, o);
    s += __shfl_down_sync(kFullMask, s, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = c;
    red[1][threadIdx.x >> 5] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kNaiveBlock / 32; i++) {
      c += red[0][i];
      s += red[1][i];
    }
    atomicAdd(acc, c);
    atomicAdd(acc + 1, s);
  }
}

// List pass 1: survivors per block of kNaiveWordsPerBlock words.
__global__ void __launch_bounds__(kNaiveBlock) naive_block_counts_kernel(const uint32_t *__restrict__ bits,
                                                                          const NaiveRange r,
                                                                          uint32_t *__restrict__ counts) {
  __shared__ uint32_t red[kNaiveBlock / 32];
  uint32_t c = 0;
  const uint64_t w0 = (uint64_t)blockIdx.x * kNaiveWordsPerBlock + (uint64_t)threadIdx.x * kNaiveWordsPerThread;
  for (uint32_t i = 0; i < kNaiveWordsPerThread; i++)
    if (w0 + i < r.nwords) c += __popc(naive_word(bits, r, w0 + i));
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(kFullMask, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < kNaiveBlock / 32; i++) c += red[i];
    counts[blockIdx.x] = c;
  }
}

// List pass 2: exclusive prefix of the block counts (one CTA, sequential
// chunks of kNaiveBlock); offsets[n] = total.
__global__ void __launch_bounds__(kNaiveBlock) naive_scan_kernel(const uint32_t *__restrict__ counts,
                                                                  uint64_t *__restrict__ offsets, uint32_t n,
                                                                  uint64_t first) {
  __shared__ uint64_t buf[kNaiveBlock];
  __shared__ uint64_t carry;
  if (threadIdx.x == 0) carry = first;
  __syncthreads();
  for (uint32_t base = 0; base < n; base += kNaiveBlock) {
    const uint32_t i = base + threadIdx.x;
    const uint64_t x = i < n ? counts[i] : 0;
    buf[threadIdx.x] = x;
    __syncthreads();
    for (int d = 1; d < kNaiveBlock; d <<= 1) {  // inclusive Hillis-Steele scan
      const uint64_t y = threadIdx.x >= (uint32_t)d ? buf[threadIdx.x - d] : 0;
      __syncthreads();
      buf[threadIdx.x] += y;
      __syncthreads();
    }
    if (i < n) offsets[i] = carry + buf[threadIdx.x] - x;
    __syncthreads();
    if (threadIdx.x == kNaiveBlock - 1) carry += buf[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n] = carry;
}

// List pass 3: each thread writes the survivors of its words, in order, at
// its block's offset plus the prefix of the threads before it.
__global__ void __launch_bounds__(kNaiveBlock) naive_write_kernel(const uint32_t *__restrict__ bits,
                                                                   const NaiveRange r,
                                                                   const uint64_t *__restrict__ offsets,
                                                                   uint64_t *__restrict__ out) {
  __shared__ uint32_t pre[kNaiveBlock];
  const uint64_t w0 = (uint64_t)blockIdx.x * kNaiveWordsPerBlock + (uint64_t)threadIdx.x * kNaiveWordsPerThread;
  uint32_t c = 0;
  for (uint32_t i = 0; i < kNaiveWordsPerThread; i++)
    if (w0 + i < r.nwords) c += __popc(naive_word(bits, r, w0 + i));
  pre[threadIdx.x] = c;
  __syncthreads();
  for (int d = 1; d < kNaiveBlock; d <<= 1) {
    const uint32_t y = threadIdx.x >= (uint32_t)d ? pre[threadIdx.x - d] : 0;
    __syncthreads();
    pre[threadIdx.x] += y;
    __syncthreads();
  }
  uint64_t o = offsets[blockIdx.x] + pre[threadIdx.x] - c;
  for (uint32_t i = 0; i < kNaiveWordsPerThread; i++) {
    const uint64_t w = w0 + i;
    if (w >= r.nwords) break;
    uint32_t x = naive_word(bits, r, w);
    while (x) {
      const uint32_t b = __ffs(x) - 1;
      out[o++] = r.olo + 2 * (32 * w + b);
      x &= x - 1;
    }
  }
}

}  // namespace
}  // namespace sieve

using namespace sieve;

extern "C" int sieve_range_naive(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int mode, sieve_count_result *cnt,
                                 uint64_t *out, size_t cap, size_t *n_out, unsigned flags) {
  if (!ctx) {
    set_error("ctx is NULL");
    return SIEVE_ERR_INVALID;
  }
  if (mode != SIEVE_COUNT && mode != SIEVE_LIST) {
    set_error("mode must be SIEVE_COUNT or SIEVE_LIST");
    return SIEVE_ERR_INVALID;
  }
  if ((mode == SIEVE_COUNT && !cnt) || (mode == SIEVE_LIST && (!n_out || (!out && cap)))) {
    set_error("sieve_range_naive: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  if (n_out) *n_out = 0;
  if (lo > hi) {
    set_error("lo (%llu) > hi (%llu)", (unsigned long long)lo, (unsigned long long)hi);
    return SIEVE_ERR_INVALID;
  }
  if (hi > (1ull << 63)) {
    set_error("hi must be <= 2^63");
    return SIEVE_ERR_RANGE;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  const bool dev_out = (flags & SIEVE_OUT_DEVICE) != 0;
  cudaStream_t st = ctx->stream;
  const uint64_t s = hi >= 2 ? isqrt_u64(hi - 1) : 0;
  if (s > ctx->table.limit) {
    set_error("isqrt(hi - 1) = %llu exceeds the base table limit %llu", (unsigned long long)s,
              (unsigned long long)ctx->table.limit);
    return SIEVE_ERR_RANGE;
  }
  NaiveRange r;
  r.lo = lo;
  r.hi = hi;
  r.olo = lo | 1;
  r.nbits = hi > r.olo ? (hi - r.olo + 1) / 2 : 0;
  r.nwords = (r.nbits + 31) / 32;
  const uint64_t two = lo <= 2 && 2 < hi;  // the one even prime, outside the bitmap

  // blocks per odd base prime (table index 1 is 3)
  const uint32_t np = host_prime_count_le_table(ctx->table, s);
  const uint32_t i0 = 1;
  const uint32_t nk = np > i0 ? np - i0 : 0;
  std::vector<uint32_t> first(nk + 1, 0);
  uint64_t blocks = 0;
  for (uint32_t k = 0; k < nk; k++) {
    first[k] = (uint32_t)blocks;
    const uint64_t n = naive_multiples(ctx->table.host_primes[i0 + k], lo, hi);
    blocks += std::max<uint64_t>(1, (n + kNaiveStrikesPerBlock - 1) / kNaiveStrikesPerBlock);
    if (blocks > 0x7FFFFFFFull) {
      set_error("sieve_range_naive: range too wide for one strike launch");
      return SIEVE_ERR_INVALID;
    }
  }
  first[nk] = (uint32_t)blocks;
  const uint64_t nlist_blocks = (r.nwords + kNaiveWordsPerBlock - 1) / kNaiveWordsPerBlock;
  if (nlist_blocks > 0x7FFFFFFFull) {
    set_error("sieve_range_naive: range too wide");
    return SIEVE_ERR_INVALID;
  }

  uint32_t *bits = nullptr, *d_first = nullptr, *counts = nullptr;
  uint64_t *offsets = nullptr;
  int rc = SIEVE_OK;
  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err, const char *what) {
    rc = cuda_fail(err, what);
  };
  do {
    if (r.nwords && (e = cudaMalloc(&bits, r.nwords * sizeof(uint32_t))) != cudaSuccess) {
      fail(e, "cudaMalloc (naive bitmap)");
      break;
    }
    if ((e = cudaMalloc(&d_first, (nk + 1) * sizeof(uint32_t))) != cudaSuccess) {
      fail(e, "cudaMalloc (naive block map)");
      break;
    }
    if ((e = cudaMemcpyAsync(d_first, first.data(), (nk + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, st)) !=
        cudaSuccess) {
      fail(e, "cudaMemcpyAsync");
      break;
    }
    if (r.nwords && (e = cudaMemsetAsync(bits, 0xFF, r.nwords * sizeof(uint32_t), st)) != cudaSuccess) {
      fail(e, "cudaMemsetAsync");
      break;
    }
    if (r.nwords && nk) {
      naive_strike_kernel<<<(uint32_t)blocks, kNaiveBlock, 0, st>>>(bits, r, ctx->table.primes, d_first, i0, nk);
      ctx->launches++;
      if ((e = cudaGetLastError()) != cudaSuccess) {
        fail(e, "naive_strike_kernel");
        break;
      }
    }
    unsigned long long *acc = ctx->d_acc;
    if ((e = cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), st)) != cudaSuccess) {
      fail(e, "cudaMemsetAsync");
      break;
    }
    if (r.nwords) {
      const uint32_t grid = (uint32_t)std::min<uint64_t>((r.nwords + kNaiveBlock - 1) / kNaiveBlock,
                                                         (uint64_t)ctx->num_sms * 8);
      naive_count_kernel<<<grid, kNaiveBlock, 0, st>>>(bits, r, acc);
      ctx->launches++;
      if ((e = cudaGetLastError()) != cudaSuccess) {
        fail(e, "naive_count_kernel");
        break;
      }
    }
    if ((e = cudaMemcpyAsync(ctx->h_acc, acc, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess) {
      fail(e, "naive result read-back");
      break;
    }
    sieve_count_result res{ctx->h_acc[0] + two, ctx->h_acc[1] + 2 * two};
    if (cnt) {
      if (dev_out) {  // as sieve_range: with SIEVE_OUT_DEVICE, cnt is device memory
        if ((e = cudaMemcpy(cnt, &res, sizeof(res), cudaMemcpyHostToDevice)) != cudaSuccess) {
          fail(e, "cudaMemcpy");
          break;
        }
      } else {
        *cnt = res;
      }
    }
    if (mode == SIEVE_COUNT) break;
    *n_out = (size_t)res.count;
    if (res.count > cap) {
      set_error("output capacity %zu is below the %llu primes found", cap, (unsigned long long)res.count);
      rc = SIEVE_ERR_CAPACITY;
      break;
    }
    if (res.count == 0) break;
    uint64_t *dst = out;
    if (!dev_out) {
      if ((rc = ensure_stage(ctx, (size_t)res.count * sizeof(uint64_t))) != SIEVE_OK) break;
      dst = (uint64_t *)ctx->d_stage;
    }
    if (two && (e = cudaMemcpyAsync(dst, &kTwo, sizeof(uint64_t), cudaMemcpyHostToDevice, st)) != cudaSuccess) {
      fail(e, "cudaMemcpyAsync");
      break;
    }
    if (r.nwords) {
      if ((e = cudaMalloc(&counts, nlist_blocks * sizeof(uint32_t))) != cudaSuccess ||
          (e = cudaMalloc(&offsets, (nlist_blocks + 1) * sizeof(uint64_t))) != cudaSuccess) {
        fail(e, "cudaMalloc (naive list)");
        break;
      }
      naive_block_counts_kernel<<<(uint32_t)nlist_blocks, kNaiveBlock, 0, st>>>(bits, r, counts);
      naive_scan_kernel<<<1, kNaiveBlock, 0, st>>>(counts, offsets, (uint32_t)nlist_blocks, two);
      naive_write_kernel<<<(uint32_t)nlist_blocks, kNaiveBlock, 0, st>>>(bits, r, offsets, dst);
      ctx->launches += 3;
      if ((e = cudaGetLastError()) != cudaSuccess) {
        fail(e, "naive list kernels");
        break;
      }
    }
    if (!dev_out &&
        (e = cudaMemcpyAsync(out, dst, (size_t)res.count * sizeof(uint64_t), cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess) {
      fail(e, "cudaMemcpyAsync");
      break;
    }
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) {
      fail(e, "cudaStreamSynchronize");
      break;
    }
  } while (0);
  cudaStreamSynchronize(st);
  cudaFree(bits);
  cudaFree(d_first);
  cudaFree(counts);
  cudaFree(offsets);
  return rc;
}
