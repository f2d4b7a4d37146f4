// incremental.cu -- the primes after a cursor, with no bound fixed in advance.
//
// The paper's sieve is incremental (Sections 2.4 and 4): the sieving primes
// are themselves produced by the sieve, so the range can keep growing past
// any N fixed at the start; only primes up to the square root of the current
// end are ever needed.  sieve_next walks forward from a cursor in windows,
// lists each window with the range sieve, and grows the context's base table
// whenever a window reaches beyond the square of its limit.
#include <algorithm>
#include <cmath>

#include "sieve_internal.cuh"

using namespace sieve;

extern "C" int sieve_next(sieve_ctx *ctx, uint64_t after, size_t k, uint64_t *out, size_t *n_out,
                          unsigned flags) {
  if (!ctx || !n_out || (!out && k)) {
    set_error("sieve_next: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  *n_out = 0;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (k == 0) return SIEVE_OK;
  const bool dev = (flags & SIEVE_OUT_DEVICE) != 0;
  const uint64_t kMaxHi = 1ull << 63;
  size_t found = 0;
  uint64_t lo = after + 1;  // primes > after
  while (found < k) {
    if (lo >= kMaxHi) {
      set_error("sieve_next: the primes after %llu run past 2^63", (unsigned long long)after);
      return SIEVE_ERR_RANGE;
    }
    // window: about 0.9 of the wanted primes at the local density 1 / ln x
    // (so that it rarely holds more than are wanted), at least 2^16 numbers
    const double gap = std::log((double)std::max<uint64_t>(lo, 16));
    const uint64_t width = (uint64_t)(0.9 * gap * (double)(k - found)) + 65536;
    const uint64_t hi = lo + std::min<uint64_t>(width, kMaxHi - lo);
    // grow the base table while isqrt(hi - 1) is beyond it (each step at most squares it)
    while (isqrt_u64(hi - 1) > ctx->table.limit) {
      const uint64_t need = isqrt_u64(hi - 1);
      // a little ahead of need, so that a walk forward does not grow it every call
      const uint64_t target = std::min<uint64_t>(need + need / 4 + 1024, 0xFFFFFFFFull);
      const uint64_t before = ctx->table.limit;
      int rc = extend_base_table(ctx, target);
      if (rc != SIEVE_OK) return rc;
      if (ctx->table.limit == before) {
        set_error("sieve_next: the base table cannot grow past %llu", (unsigned long long)before);
        return SIEVE_ERR_RANGE;
      }
    }
    RangeRequest rq;
    rq.lo = lo;
    rq.hi = hi;
    rq.list = 1;
    rq.out_bytes = 8;
    rq.out = out + found;
    rq.cap = k - found;
    rq.out_on_device = dev;
    size_t n = 0;
    int rc = run_range(ctx, ctx->table, rq, &n);
    if (rc == SIEVE_ERR_CAPACITY) {
      // the window holds n > wanted primes: list it on the device and keep
      // the wanted prefix (the primes after `after` are the window's first ones)
      const size_t want = k - found;
      if ((rc = ensure_stage(ctx, n * sizeof(uint64_t))) != SIEVE_OK) return rc;
      uint64_t *stage = (uint64_t *)ctx->d_stage;
      rq.out = stage;
      rq.cap = n;
      rq.out_on_device = 1;
      size_t n2 = 0;
      if ((rc = run_range(ctx, ctx->table, rq, &n2)) != SIEVE_OK) return rc;
      SIEVE_CUDA_TRY(cudaMemcpyAsync(out + found, stage, want * sizeof(uint64_t),
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
      SIEVE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
      found += want;
      break;
    }
    if (rc != SIEVE_OK) return rc;
    found += n;
    lo = hi;
  }
  *n_out = found;
  return SIEVE_OK;
}
