// autotune.cu -- pick the segment-kernel tunables by timing them.
//
// Section 5 of the paper measures how the per-thread array size changes the
// run time and keeps the best; these calls do the same for the GPU knobs:
// tile length (the array size here), threads per CTA, the warp/lane split for
// striking, the presieve depth and, for batches, the strip size.  Each
// candidate is run once untimed and `reps` times under CUDA events on the
// context's stream; the median decides.  Every candidate's results are
// compared with the first candidate's, so a tunable can never change an
// answer silently.
#include <algorithm>
#include <cstring>
#include <vector>

#include "sieve_internal.cuh"

using namespace sieve;

namespace {

struct EventPair {
  cudaEvent_t a = nullptr, b = nullptr;
  ~EventPair() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

double median(std::vector<double> v) {
  std::sort(v.begin(), v.end());
  return v.empty() ? 0.0 : v[v.size() / 2];
}

}  // namespace

extern "C" int sieve_autotune_batch(sieve_ctx *ctx, const uint64_t *lo, const uint64_t *hi, const uint8_t *mode,
                                    size_t nq, int reps, sieve_options *best, double *best_ms) {
  if (!ctx || !lo || !hi || !mode || nq == 0 || reps < 1) {
    set_error("sieve_autotune_batch: NULL argument, empty batch or reps < 1");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  const sieve_options orig = ctx->opt;
  sieve_count_result *d_cnt = nullptr;
  uint64_t *d_off = nullptr, *d_val = nullptr;
  EventPair ev;
  int rc = SIEVE_OK;
  std::vector<sieve_count_result> ref(nq), got(nq);
  sieve_options best_opt = orig;
  double best_t = 1e300;
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&d_cnt, nq * sizeof(sieve_count_result))) != cudaSuccess ||
        (e = cudaMalloc(&d_off, (nq + 1) * sizeof(uint64_t))) != cudaSuccess ||
        (e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess) {
      rc = cuda_fail(e, "autotune allocation");
      break;
    }
    // size the list output once
    size_t need = 0;
    rc = sieve_range_batch(ctx, lo, hi, mode, nq, d_cnt, d_off, nullptr, 0, &need, SIEVE_OUT_DEVICE);
    if (rc != SIEVE_OK && rc != SIEVE_ERR_CAPACITY) break;
    rc = SIEVE_OK;
    if ((e = cudaMalloc(&d_val, std::max<size_t>(need, 1) * sizeof(uint64_t))) != cudaSuccess) {
      rc = cuda_fail(e, "autotune allocation");
      break;
    }
    const uint32_t tiles[] = {1u << 15, 1u << 16, 1u << 17, 1u << 18, 1u << 19};
    const uint32_t threads[] = {512, 1024};
    const uint32_t chunks[] = {1u << 13, 1u << 15, 1u << 17};
    std::vector<sieve_options> cand;
    for (uint32_t tb : tiles)
      for (uint32_t th : threads)
        for (uint32_t ch : chunks) {
          sieve_options o = orig;
          o.batch_tile_bits = tb;
          o.block_threads = th;
          o.chunk_primes = ch;
          cand.push_back(o);
        }
    bool have_ref = false;
    for (const sieve_options &o : cand) {
      const uint32_t tb = o.batch_tile_bits, th = o.block_threads, ch = o.chunk_primes;
      if (sieve_set_options(ctx, &o) != SIEVE_OK) continue;  // does not fit this device
      std::vector<double> ts;
      size_t n = 0;
      for (int r = 0; r <= reps && rc == SIEVE_OK; r++) {
        if ((e = cudaEventRecord(ev.a, ctx->stream)) != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
        if (rc == SIEVE_OK)
          rc = sieve_range_batch(ctx, lo, hi, mode, nq, d_cnt, d_off, d_val, need, &n, SIEVE_OUT_DEVICE);
        if (rc == SIEVE_OK && (e = cudaEventRecord(ev.b, ctx->stream)) != cudaSuccess)
          rc = cuda_fail(e, "cudaEventRecord");
        if (rc == SIEVE_OK && (e = cudaEventSynchronize(ev.b)) != cudaSuccess)
          rc = cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        if (rc == SIEVE_OK) cudaEventElapsedTime(&ms, ev.a, ev.b);
        if (r > 0) ts.push_back(ms);
      }
      if (rc != SIEVE_OK) break;
      if ((e = cudaMemcpy(got.data(), d_cnt, nq * sizeof(sieve_count_result), cudaMemcpyDeviceToHost)) !=
          cudaSuccess) {
        rc = cuda_fail(e, "cudaMemcpy");
        break;
      }
      if (!have_ref) {
        ref = got;
        have_ref = true;
      } else if (memcmp(ref.data(), got.data(), nq * sizeof(sieve_count_result)) != 0) {
        set_error("autotune: batch_tile_bits %u, block_threads %u, chunk_primes %u changed a result", tb, th,
                  ch);
        rc = SIEVE_ERR_CUDA;
        break;
      }
      const double t = median(ts);
      if (t < best_t) {
        best_t = t;
        best_opt = o;
      }
    }
  } while (0);
  cudaFree(d_cnt);
  cudaFree(d_off);
  cudaFree(d_val);
  ctx->opt = rc == SIEVE_OK ? best_opt : orig;
  if (rc != SIEVE_OK) return rc;
  if (best) *best = best_opt;
  if (best_ms) *best_ms = best_t;
  return SIEVE_OK;
}

extern "C" int sieve_autotune_range(sieve_ctx *ctx, uint64_t lo, uint64_t hi, int reps, sieve_options *best,
                                    double *best_ms) {
  if (!ctx || reps < 1 || lo >= hi) {
    set_error("sieve_autotune_range: NULL context, empty range or reps < 1");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  const sieve_options orig = ctx->opt;
  sieve_count_result *d_tot = nullptr;
  EventPair ev;
  int rc = SIEVE_OK;
  sieve_options best_opt = orig;
  double best_t = 1e300;
  sieve_count_result ref{0, 0}, got{0, 0};
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&d_tot, sizeof(sieve_count_result))) != cudaSuccess ||
        (e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess) {
      rc = cuda_fail(e, "autotune allocation");
      break;
    }
    const uint32_t tiles[] = {1u << 17, 1u << 18, 1u << 19};
    const uint32_t threads[] = {512, 1024};
    const uint32_t ghs[] = {2, 4, 8};
    const uint32_t groups[] = {1, 2, 3, 4};
    std::vector<sieve_options> cand;
    for (uint32_t tb : tiles)
      for (uint32_t th : threads)
        for (uint32_t gh : ghs)
          for (uint32_t g : groups) {
            sieve_options o = orig;
            o.tile_bits = tb;
            o.block_threads = th;
            o.group_hits = gh;
            o.presieve_groups = g;
            cand.push_back(o);
          }
    bool have_ref = false;
    for (const sieve_options &o : cand) {
      const uint32_t tb = o.tile_bits, th = o.block_threads, gh = o.group_hits, g = o.presieve_groups;
      if (sieve_set_options(ctx, &o) != SIEVE_OK) continue;
      std::vector<double> ts;
      for (int r = 0; r <= reps && rc == SIEVE_OK; r++) {
        if ((e = cudaEventRecord(ev.a, ctx->stream)) != cudaSuccess) rc = cuda_fail(e, "cudaEventRecord");
        if (rc == SIEVE_OK)
          rc = sieve_range(ctx, lo, hi, SIEVE_COUNT, d_tot, nullptr, 0, nullptr, SIEVE_OUT_DEVICE | SIEVE_ASYNC);
        if (rc == SIEVE_OK && (e = cudaEventRecord(ev.b, ctx->stream)) != cudaSuccess)
          rc = cuda_fail(e, "cudaEventRecord");
        if (rc == SIEVE_OK && (e = cudaEventSynchronize(ev.b)) != cudaSuccess)
          rc = cuda_fail(e, "cudaEventSynchronize");
        float ms = 0.f;
        if (rc == SIEVE_OK) cudaEventElapsedTime(&ms, ev.a, ev.b);
        if (r > 0) ts.push_back(ms);
      }
      if (rc != SIEVE_OK) break;
      if ((e = cudaMemcpy(&got, d_tot, sizeof(got), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = cuda_fail(e, "cudaMemcpy");
        break;
      }
      if (!have_ref) {
        ref = got;
        have_ref = true;
      } else if (ref.count != got.count || ref.checksum != got.checksum) {
        set_error("autotune: tile_bits %u, block_threads %u, group_hits %u, presieve_groups %u changed the "
                  "result",
                  tb, th, gh, g);
        rc = SIEVE_ERR_CUDA;
        break;
      }
      const double t = median(ts);
      if (t < best_t) {
        best_t = t;
        best_opt = o;
      }
    }
  } while (0);
  cudaFree(d_tot);
  ctx->opt = rc == SIEVE_OK ? best_opt : orig;
  if (rc != SIEVE_OK) return rc;
  if (best) *best = best_opt;
  if (best_ms) *best_ms = best_t;
  return SIEVE_OK;
}
