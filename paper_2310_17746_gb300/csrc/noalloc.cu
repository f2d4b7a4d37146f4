// noalloc.cu -- the one entry point that allocates no memory.
//
// Some callers cannot allocate device memory at the moment they need primes:
// a process whose device memory is entirely owned by another allocator (a
// framework's caching pool that must not see raw cudaMalloc / cudaFree), a
// latency-critical thread where cudaFree's implicit device synchronization or
// an allocation's unpredictable cost is not acceptable, or a host under a
// strict memory budget fixed at start-up.  For them,
// sieve_range_list_noalloc lists the primes of a range into the caller's
// device buffer using only memory that already exists: the context's base
// table and accumulators (made when the context was created) and a fixed
// scratch array that lives in this library's device image.
#include "sieve_internal.cuh"

// Per-tile counts, offsets and bitmaps of one call.  Every GPU that loads the
// library holds this array until the process exits.  All calls on a device
// share it and it keeps the previous call's contents; each call writes every
// entry it later reads (tile counts and bitmaps by the tile kernel, offsets by
// the scan), so nothing needs clearing.
static __device__ __align__(256) unsigned char g_noalloc_scratch[SIEVE_NOALLOC_SCRATCH_BYTES];

namespace sieve {

int run_range_list_into(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out, size_t cap, size_t *n_out,
                        sieve_count_result *cnt, void *scratch, size_t scratch_bytes);

// In host code the array's name is only a host-side stand-in, not a device
// address: a kernel given it would fault or use the wrong memory.  Its device
// address on the context's device is looked up here, with that device
// current, when the context is created.  Under lazy module loading this first
// lookup is what loads the module and so makes the array: it happens inside
// sieve_create, which allocates anyway, and never inside the entry point.
int noalloc_setup(sieve_ctx *ctx) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  ctx->noalloc_scratch = p;
  return SIEVE_OK;
}

}  // namespace sieve

extern "C" int sieve_range_list_noalloc(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t *out, size_t cap,
                                        size_t *n_out, sieve_count_result *cnt) {
  if (!ctx || !n_out || (!out && cap)) {
    sieve::set_error("sieve_range_list_noalloc: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  if (!ctx->noalloc_scratch) {
    sieve::set_error("sieve_range_list_noalloc: the context has no scratch address (sieve_create failed?)");
    return SIEVE_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return sieve::cuda_fail(e, "cudaSetDevice");
  return sieve::run_range_list_into(ctx, lo, hi, out, cap, n_out, cnt, ctx->noalloc_scratch,
                                    SIEVE_NOALLOC_SCRATCH_BYTES);
}
