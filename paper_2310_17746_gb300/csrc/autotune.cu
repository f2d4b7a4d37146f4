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
#include <cstdio>
#include <cstring>
#include <string>
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
    bool have_ref = false;
    // times each candidate (reps runs after an untimed one) and keeps the
    // fastest; every candidate's counts must equal the first one's
    auto try_all = [&](const std::vector<sieve_options> &cand) {
      for (const sieve_options &o : cand) {
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
        if (rc != SIEVE_OK) return;
        if ((e = cudaMemcpy(got.data(), d_cnt, nq * sizeof(sieve_count_result), cudaMemcpyDeviceToHost)) !=
            cudaSuccess) {
          rc = cuda_fail(e, "cudaMemcpy");
          return;
        }
        if (!have_ref) {
          ref = got;
          have_ref = true;
        } else if (memcmp(ref.data(), got.data(), nq * sizeof(sieve_count_result)) != 0) {
          set_error("autotune: batch_tile_bits %u, block_threads %u, chunk_primes %u, presieve_groups %u "
                    "changed a result",
                    o.batch_tile_bits, o.block_threads, o.chunk_primes, o.presieve_groups);
          rc = SIEVE_ERR_CUDA;
          return;
        }
        const double t = median(ts);
        if (t < best_t) {
          best_t = t;
          best_opt = o;
        }
      }
    };
    // stage 1: tile length, block size and strip size
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
    try_all(cand);
    if (rc != SIEVE_OK) break;
    // stage 2: presieve groups around the winner (fewer pattern reads leave
    // L2 to the strips' table streams: 4096 queries, seed 0, 13.98 ms with 7
    // groups, 13.75 with 5)
    cand.clear();
    for (uint32_t pg = 4; pg <= 7; pg++)
      if (pg != best_opt.presieve_groups) {
        sieve_options o = best_opt;
        o.presieve_groups = pg;
        cand.push_back(o);
      }
    try_all(cand);
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
  bool have_ref = false;
  double orig_t = 1e300;  // time of the context's own options, when among the candidates
  // times each candidate (reps runs after an untimed one) and keeps the
  // fastest; every candidate's result must equal the first one's
  auto try_all = [&](const std::vector<sieve_options> &cand) {
    cudaError_t e;
    for (const sieve_options &o : cand) {
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
      if (rc != SIEVE_OK) return;
      if ((e = cudaMemcpy(&got, d_tot, sizeof(got), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = cuda_fail(e, "cudaMemcpy");
        return;
      }
      if (!have_ref) {
        ref = got;
        have_ref = true;
      } else if (ref.count != got.count || ref.checksum != got.checksum) {
        set_error("autotune: tile_bits %u, block_threads %u, ctas_per_sm %u, group_hits %u, presieve_groups %u, "
                  "bucket_threshold %u, bucket_wave %u, bucket_scatter %u changed the result",
                  o.tile_bits, o.block_threads, o.ctas_per_sm, o.group_hits, o.presieve_groups,
                  o.bucket_threshold, o.bucket_wave, o.bucket_scatter);
        rc = SIEVE_ERR_CUDA;
        return;
      }
      const double t = median(ts);
      if (memcmp(&o, &orig, sizeof(o)) == 0) orig_t = t;
      if (t < best_t) {
        best_t = t;
        best_opt = o;
      }
    }
  };
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&d_tot, sizeof(sieve_count_result))) != cudaSuccess ||
        (e = cudaEventCreate(&ev.a)) != cudaSuccess || (e = cudaEventCreate(&ev.b)) != cudaSuccess) {
      rc = cuda_fail(e, "autotune allocation");
      break;
    }
    // stage 1: tile length (Section 5's array size), threads per CTA, CTAs per
    // SM, the warp/lane split and the presieve depth
    const uint32_t tiles[] = {1u << 18, 1u << 19};
    const uint32_t threads[] = {512, 1024};
    const uint32_t ctas[] = {0, 1, 2};
    const uint32_t ghs[] = {3, 4, 5, 6, 8};
    const uint32_t groups[] = {5, 6, 7, 8};
    std::vector<sieve_options> cand;
    for (uint32_t tb : tiles)
      for (uint32_t th : threads)
        for (uint32_t cs : ctas) {
          if (cs && th == 1024) continue;  // a 1024-thread CTA fits once per SM anyway
          for (uint32_t gh : ghs)
            for (uint32_t g : groups) {
              sieve_options o = orig;
              o.tile_bits = tb;
              o.block_threads = th;
              o.ctas_per_sm = cs;
              o.group_hits = gh;
              o.presieve_groups = g;
              cand.push_back(o);
            }
        }
    try_all(cand);
    if (rc != SIEVE_OK) break;
    // stage 2, for ranges whose large primes can go through the bucket sieve:
    // the large-prime threshold (off, or 2..16 tile lengths), the wave size
    // and the scatter kind, with the stage-1 winner's other settings
    sieve_options probe = best_opt;
    probe.bucket_threshold = 2;
    probe.bucket_scatter = 0;
    ctx->opt = probe;
    const bool buckets = range_prefers_buckets(ctx, lo, hi);
    if (buckets) {
      std::vector<sieve_options> bc;
      sieve_options off = best_opt;
      off.bucket_threshold = 0;
      bc.push_back(off);
      for (uint32_t thr : {2u, 4u, 8u, 16u})
        for (uint32_t wv : {1u, 4u})
          for (uint32_t sc : {1u, 2u}) {
            sieve_options o = best_opt;
            o.bucket_threshold = thr;
            o.bucket_wave = wv;
            o.bucket_scatter = sc;
            bc.push_back(o);
          }
      try_all(bc);
    }
    // keep the context's options when they are within 1% of the fastest
    // candidate: such a gap is within run-to-run noise
    if (orig_t <= 1.01 * best_t) {
      best_opt = orig;
      best_t = orig_t;
    }
  } while (0);
  cudaFree(d_tot);
  ctx->opt = rc == SIEVE_OK ? best_opt : orig;
  if (rc != SIEVE_OK) return rc;
  if (best) *best = best_opt;
  if (best_ms) *best_ms = best_t;
  return SIEVE_OK;
}

// ---------------------------------------------------------------- tuning cache
//
// The tuned options persist in a small JSON file keyed by (device name, SM
// count, workload name), one entry per line:
//   {"sieve_tune_cache": 1, "entries": [
//   {"device": "...", "sms": 152, "workload": "...", "tile_bits": ..., ..., "ms": ...},
//   ...
//   ]}
// Storing replaces the entry with the same key and keeps the others.

namespace {

bool cache_name_ok(const char *s) {
  if (!s || !*s || strlen(s) > 200) return false;
  for (const char *c = s; *c; c++)
    if (*c == '"' || *c == '\\' || (unsigned char)*c < 0x20) return false;
  return true;
}

// The string value of "key": "..." in a one-line entry.
bool entry_str(const std::string &line, const char *key, std::string *out) {
  const std::string k = std::string("\"") + key + "\": \"";
  const size_t a = line.find(k);
  if (a == std::string::npos) return false;
  const size_t b = line.find('"', a + k.size());
  if (b == std::string::npos) return false;
  *out = line.substr(a + k.size(), b - a - k.size());
  return true;
}

bool entry_num(const std::string &line, const char *key, double *out) {
  const std::string k = std::string("\"") + key + "\": ";
  const size_t a = line.find(k);
  if (a == std::string::npos) return false;
  return sscanf(line.c_str() + a + k.size(), "%lf", out) == 1;
}

struct CacheEntry {
  std::string line, device, workload;
  int sms = 0;
};

int device_key(const sieve_ctx *ctx, std::string *name) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceProperties");
  *name = prop.name;
  for (char &c : *name)
    if (c == '"' || c == '\\' || (unsigned char)c < 0x20) c = '_';
  return SIEVE_OK;
}

std::vector<CacheEntry> read_cache(const char *path) {
  std::vector<CacheEntry> v;
  FILE *f = fopen(path, "r");
  if (!f) return v;
  char buf[2048];
  while (fgets(buf, sizeof(buf), f)) {
    std::string line(buf);
    while (!line.empty() && (line.back() == '\n' || line.back() == '\r' || line.back() == ',')) line.pop_back();
    if (line.rfind("{\"device\": ", 0) != 0) continue;
    CacheEntry en;
    double sms = 0;
    if (!entry_str(line, "device", &en.device) || !entry_str(line, "workload", &en.workload) ||
        !entry_num(line, "sms", &sms))
      continue;
    en.sms = (int)sms;
    en.line = line;
    v.push_back(en);
  }
  fclose(f);
  return v;
}

}  // namespace

extern "C" int sieve_tune_cache_store(sieve_ctx *ctx, const char *path, const char *workload, double ms) {
  if (!ctx || !path || !cache_name_ok(workload)) {
    set_error("sieve_tune_cache_store: NULL argument, or a workload name that is empty, longer than 200 "
              "characters or holds a quote, backslash or control character");
    return SIEVE_ERR_INVALID;
  }
  std::string dev;
  int rc = device_key(ctx, &dev);
  if (rc != SIEVE_OK) return rc;
  std::vector<CacheEntry> v = read_cache(path);
  const sieve_options &o = ctx->opt;
  char line[1024];
  snprintf(line, sizeof(line),
           "{\"device\": \"%s\", \"sms\": %d, \"workload\": \"%s\", \"tile_bits\": %u, \"block_threads\": %u, "
           "\"ctas_per_sm\": %u, \"group_hits\": %u, \"presieve_groups\": %u, \"batch_tile_bits\": %u, "
           "\"chunk_primes\": %u, \"bucket_threshold\": %u, \"bucket_wave\": %u, \"bucket_scatter\": %u, "
           "\"list_single_pass\": %u, \"cluster_ctas\": %u, \"cluster_threshold\": %u, \"ms\": %.6f}",
           dev.c_str(), ctx->num_sms, workload, o.tile_bits, o.block_threads, o.ctas_per_sm, o.group_hits,
           o.presieve_groups, o.batch_tile_bits, o.chunk_primes, o.bucket_threshold, o.bucket_wave,
           o.bucket_scatter, o.list_single_pass, o.cluster_ctas, o.cluster_threshold, ms);
  CacheEntry mine;
  mine.line = line;
  mine.device = dev;
  mine.workload = workload;
  mine.sms = ctx->num_sms;
  bool replaced = false;
  for (CacheEntry &e : v)
    if (e.device == dev && e.sms == ctx->num_sms && e.workload == workload) {
      e = mine;
      replaced = true;
    }
  if (!replaced) v.push_back(mine);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = fopen(tmp.c_str(), "w");
  if (!f) {
    set_error("sieve_tune_cache_store: cannot write %s", tmp.c_str());
    return SIEVE_ERR_INVALID;
  }
  fprintf(f, "{\"sieve_tune_cache\": 1, \"entries\": [\n");
  for (size_t i = 0; i < v.size(); i++) fprintf(f, "%s%s\n", v[i].line.c_str(), i + 1 < v.size() ? "," : "");
  fprintf(f, "]}\n");
  const bool ok = fclose(f) == 0 && rename(tmp.c_str(), path) == 0;
  if (!ok) {
    set_error("sieve_tune_cache_store: cannot replace %s", path);
    return SIEVE_ERR_INVALID;
  }
  return SIEVE_OK;
}

extern "C" int sieve_tune_cache_load(sieve_ctx *ctx, const char *path, const char *workload, int *found,
                                     double *ms) {
  if (!ctx || !path || !found || !cache_name_ok(workload)) {
    set_error("sieve_tune_cache_load: NULL argument or bad workload name");
    return SIEVE_ERR_INVALID;
  }
  *found = 0;
  std::string dev;
  int rc = device_key(ctx, &dev);
  if (rc != SIEVE_OK) return rc;
  for (const CacheEntry &e : read_cache(path)) {
    if (e.device != dev || e.sms != ctx->num_sms || e.workload != workload) continue;
    const char *keys[7] = {"tile_bits", "block_threads", "ctas_per_sm", "group_hits", "presieve_groups",
                           "batch_tile_bits", "chunk_primes"};
    double v[7];
    for (int i = 0; i < 7; i++)
      if (!entry_num(e.line, keys[i], &v[i]) || v[i] < 0 || v[i] > 4294967295.0) {
        set_error("sieve_tune_cache_load: entry for %s has no valid %s", workload, keys[i]);
        return SIEVE_ERR_INVALID;
      }
    sieve_options o = ctx->opt;
    o.tile_bits = (uint32_t)v[0];
    o.block_threads = (uint32_t)v[1];
    o.ctas_per_sm = (uint32_t)v[2];
    o.group_hits = (uint32_t)v[3];
    o.presieve_groups = (uint32_t)v[4];
    o.batch_tile_bits = (uint32_t)v[5];
    o.chunk_primes = (uint32_t)v[6];
    double bt = 0, bw = 0;  // entries written before the bucket sieve existed lack these
    if (entry_num(e.line, "bucket_threshold", &bt) && bt >= 0 && bt <= 64) o.bucket_threshold = (uint32_t)bt;
    if (entry_num(e.line, "bucket_wave", &bw) && bw >= 1 && bw <= 16) o.bucket_wave = (uint32_t)bw;
    double bs = 0;
    if (entry_num(e.line, "bucket_scatter", &bs) && bs >= 0 && bs <= 2) o.bucket_scatter = (uint32_t)bs;
    double sp = 0, cc = 0, ct = 0;  // nor these, before the one-pass list and cluster segments
    if (entry_num(e.line, "list_single_pass", &sp) && sp >= 0 && sp <= 1) o.list_single_pass = (uint32_t)sp;
    if (entry_num(e.line, "cluster_ctas", &cc) && cc >= 0 && cc <= 16) o.cluster_ctas = (uint32_t)cc;
    if (entry_num(e.line, "cluster_threshold", &ct) && ct >= 0 && ct <= 1024) o.cluster_threshold = (uint32_t)ct;
    rc = sieve_set_options(ctx, &o);  // validates every field
    if (rc != SIEVE_OK) return rc;
    double t = 0;
    if (ms) *ms = entry_num(e.line, "ms", &t) ? t : 0.0;
    *found = 1;
    return SIEVE_OK;
  }
  return SIEVE_OK;
}
