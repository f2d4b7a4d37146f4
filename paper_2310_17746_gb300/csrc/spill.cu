// spill.cu -- long runs that survive interruption, and lists larger than
// device memory (the paper's first future-work item, Section 6: results
// written out in store segments instead of kept in memory).
//
//   * sieve_count_checkpointed: a count (with per-segment counts) of [lo, hi)
//     in chunks; after every chunk the running totals go to a state file, and
//     a later call resumes after the last finished chunk.
//   * sieve_primes_to_file: the primes of [lo, hi) appended to a binary file
//     one store segment (at most segment_primes primes) at a time, with a
//     state file that lets an interrupted run continue where it stopped.
//
// Both state files are small binary records, written to path + ".tmp" and
// renamed over the old one, so that a crash leaves either the old or the new
// record, never a torn one; a 64-bit FNV-1a hash of the record's bytes guards
// against a damaged file.
#include <sys/types.h>
#include <unistd.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sieve_internal.cuh"

namespace sieve {
namespace {

// FNV-1a, 64-bit (Fowler, Noll, Vo): offset basis 14695981039346656037,
// prime 1099511628211.
uint64_t fnv1a64(const void *data, size_t n) {
  const unsigned char *p = (const unsigned char *)data;
  uint64_t h = 14695981039346656037ull;
  for (size_t i = 0; i < n; i++) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

// A record is 8 magic bytes, n little-endian uint64 words, then the hash of
// everything before it.  (Host byte order: every machine this library builds
// for is little-endian.)
bool write_record(const std::string &path, const char magic[8], const std::vector<uint64_t> &words) {
  std::vector<unsigned char> buf(8 + 8 * words.size());
  memcpy(buf.data(), magic, 8);
  if (!words.empty()) memcpy(buf.data() + 8, words.data(), 8 * words.size());
  const uint64_t h = fnv1a64(buf.data(), buf.size());
  const std::string tmp = path + ".tmp";
  FILE *f = fopen(tmp.c_str(), "wb");
  if (!f) return false;
  bool ok = fwrite(buf.data(), 1, buf.size(), f) == buf.size() && fwrite(&h, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  return ok && rename(tmp.c_str(), path.c_str()) == 0;
}

// 1: read (words filled), 0: no such file, -1: damaged or not this kind.
int read_record(const std::string &path, const char magic[8], std::vector<uint64_t> *words) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return 0;
  std::vector<unsigned char> buf;
  unsigned char tmp[4096];
  size_t n;
  while ((n = fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + n);
  fclose(f);
  if (buf.size() < 16 || buf.size() % 8 != 0 || memcmp(buf.data(), magic, 8) != 0) return -1;
  uint64_t h;
  memcpy(&h, buf.data() + buf.size() - 8, 8);
  if (fnv1a64(buf.data(), buf.size() - 8) != h) return -1;
  words->resize((buf.size() - 16) / 8);
  if (!words->empty()) memcpy(words->data(), buf.data() + 8, buf.size() - 16);
  return 1;
}

const char kCountMagic[8] = {'S', 'I', 'E', 'V', 'E', 'C', 'K', '1'};
const char kSpillMagic[8] = {'S', 'I', 'E', 'V', 'E', 'S', 'P', '1'};

// Largest width w whose prime count is surely <= cap wherever the window
// starts: the count of integers prime to 6 (2 ceil(w / 6) + 2, with 2 and 3)
// and the Montgomery-Vaughan bound pi(x + w) - pi(x) <= 2 w / ln w (for
// w > 1), with slack, both bound it; take the larger w allowed by either.
uint64_t width_for_primes(uint64_t cap) {
  auto bound = [](uint64_t w) -> double {
    const double a = 2.0 * std::ceil((double)w / 6.0) + 2.0;
    const double b = w > 1 ? 2.0 * (double)w / std::log((double)w) + 64.0 : a;
    return std::min(a, b);
  };
  uint64_t lo = 1, hi = (uint64_t)1 << 62;
  while (hi - lo > 1) {
    const uint64_t mid = lo + (hi - lo) / 2;
    (bound(mid) <= (double)cap ? lo : hi) = mid;
  }
  return lo;
}

}  // namespace
}  // namespace sieve

using namespace sieve;

extern "C" int sieve_count_checkpointed(sieve_ctx *ctx, uint64_t lo, uint64_t hi, uint64_t seg_width,
                                        uint64_t chunk_width, const char *state_path, uint64_t *counts,
                                        size_t ncounts, sieve_count_result *total, uint64_t max_chunks,
                                        uint64_t *next) {
  if (!ctx || !state_path || !total || chunk_width == 0 || (ncounts && !counts) || lo > hi) {
    set_error("sieve_count_checkpointed: NULL argument, chunk_width 0 or lo > hi");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t nb = (seg_width && hi > lo) ? (size_t)((hi - 1) / seg_width - lo / seg_width + 1) : 0;
  if (ncounts != nb || (seg_width && seg_width < 6144)) {
    set_error("sieve_count_checkpointed: ncounts must be %zu (seg_width 0 or >= 6144)", nb);
    return SIEVE_ERR_INVALID;
  }
  // state: lo, hi, seg_width, chunk_width, next, count, checksum, nbins, bins...
  std::vector<uint64_t> st;
  const std::string path(state_path);
  const int got = read_record(path, kCountMagic, &st);
  if (got < 0) {
    set_error("sieve_count_checkpointed: %s is damaged or not a count state", state_path);
    return SIEVE_ERR_INVALID;
  }
  if (got == 1) {
    if (st.size() != 8 + nb || st[0] != lo || st[1] != hi || st[2] != seg_width || st[3] != chunk_width ||
        st[7] != nb || st[4] < lo || st[4] > hi) {
      set_error("sieve_count_checkpointed: %s belongs to another job", state_path);
      return SIEVE_ERR_INVALID;
    }
  } else {
    st.assign(8 + nb, 0);
    st[0] = lo;
    st[1] = hi;
    st[2] = seg_width;
    st[3] = chunk_width;
    st[4] = lo;
    st[7] = nb;
  }
  std::vector<uint64_t> chunk_bins;
  uint64_t done = 0;
  int rc = SIEVE_OK;
  while (st[4] < hi && (max_chunks == 0 || done < max_chunks)) {
    const uint64_t a = st[4];
    const uint64_t b = hi - a > chunk_width ? a + chunk_width : hi;
    RangeRequest rq;
    rq.lo = a;
    rq.hi = b;
    sieve_count_result r{0, 0};
    rq.total = &r;
    if (seg_width) {
      chunk_bins.assign((size_t)((b - 1) / seg_width - a / seg_width + 1), 0);
      rq.seg_width = seg_width;
      rq.bins = chunk_bins.data();
      rq.nbins = chunk_bins.size();
    }
    if ((rc = run_range(ctx, ctx->table, rq, nullptr)) != SIEVE_OK) return rc;
    st[5] += r.count;
    st[6] += r.checksum;  // mod 2^64
    const size_t first = seg_width ? (size_t)(a / seg_width - lo / seg_width) : 0;
    for (size_t i = 0; i < chunk_bins.size(); i++) st[8 + first + i] += chunk_bins[i];
    st[4] = b;
    if (!write_record(path, kCountMagic, st)) {
      set_error("sieve_count_checkpointed: cannot write %s", state_path);
      return SIEVE_ERR_INVALID;
    }
    done++;
  }
  if (next) *next = st[4];
  total->count = st[5];
  total->checksum = st[6];
  if (nb) memcpy(counts, st.data() + 8, nb * sizeof(uint64_t));
  return st[4] < hi ? SIEVE_PENDING : SIEVE_OK;
}

extern "C" int sieve_primes_to_file(sieve_ctx *ctx, uint64_t lo, uint64_t hi, const char *path,
                                    size_t segment_primes, int resume, uint64_t max_segments,
                                    uint64_t *n_written) {
  if (!ctx || !path || lo > hi) {
    set_error("sieve_primes_to_file: NULL argument or lo > hi");
    return SIEVE_ERR_INVALID;
  }
  if (segment_primes == 0) segment_primes = 125000000;  // 1 GB of uint64 per store segment
  if (segment_primes < 1024) {
    set_error("sieve_primes_to_file: segment_primes must be 0 or >= 1024");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(ctx->device));
  const std::string spath = std::string(path) + ".state";
  // state: lo, hi, segment_primes, next, primes written
  std::vector<uint64_t> st;
  int got = resume ? read_record(spath, kSpillMagic, &st) : 0;
  if (got < 0) {
    set_error("sieve_primes_to_file: %s is damaged or not a list state", spath.c_str());
    return SIEVE_ERR_INVALID;
  }
  if (got == 1 && (st.size() != 5 || st[0] != lo || st[1] != hi || st[2] != segment_primes || st[3] < lo ||
                   st[3] > hi)) {
    set_error("sieve_primes_to_file: %s belongs to another job", spath.c_str());
    return SIEVE_ERR_INVALID;
  }
  if (got != 1) st = {lo, hi, (uint64_t)segment_primes, lo, 0};
  // the list file holds exactly st[4] primes: cut off whatever an interrupted
  // segment left behind (or start it empty)
  FILE *f = fopen(path, got == 1 ? "r+b" : "wb");
  if (!f) {
    set_error("sieve_primes_to_file: cannot open %s", path);
    return SIEVE_ERR_INVALID;
  }
  const uint64_t w = width_for_primes(segment_primes);
  uint64_t *d_out = nullptr, *h_out = nullptr;
  int rc = SIEVE_OK;
  do {
    if (got == 1) {
      if (fseeko(f, (off_t)(st[4] * 8), SEEK_SET) != 0 || ftruncate(fileno(f), (off_t)(st[4] * 8)) != 0) {
        set_error("sieve_primes_to_file: cannot cut %s back to %llu primes", path, (unsigned long long)st[4]);
        rc = SIEVE_ERR_INVALID;
        break;
      }
    }
    cudaError_t e;
    if ((e = cudaMalloc(&d_out, segment_primes * sizeof(uint64_t))) != cudaSuccess ||
        (e = cudaMallocHost(&h_out, segment_primes * sizeof(uint64_t))) != cudaSuccess) {
      rc = cuda_fail(e, "sieve_primes_to_file: segment buffers");
      break;
    }
    uint64_t done = 0;
    while (st[3] < hi && (max_segments == 0 || done < max_segments)) {
      const uint64_t a = st[3];
      const uint64_t b = hi - a > w ? a + w : hi;
      RangeRequest rq;
      rq.lo = a;
      rq.hi = b;
      rq.list = 1;
      rq.out_bytes = 8;
      rq.out = d_out;
      rq.cap = segment_primes;
      rq.out_on_device = 1;
      size_t n = 0;
      if ((rc = run_range(ctx, ctx->table, rq, &n)) != SIEVE_OK) break;
      if (n && (e = cudaMemcpy(h_out, d_out, n * sizeof(uint64_t), cudaMemcpyDeviceToHost)) != cudaSuccess) {
        rc = cuda_fail(e, "sieve_primes_to_file: copy to host");
        break;
      }
      if (fwrite(h_out, sizeof(uint64_t), n, f) != n || fflush(f) != 0) {
        set_error("sieve_primes_to_file: cannot write %s", path);
        rc = SIEVE_ERR_INVALID;
        break;
      }
      st[3] = b;
      st[4] += n;
      if (!write_record(spath, kSpillMagic, st)) {
        set_error("sieve_primes_to_file: cannot write %s", spath.c_str());
        rc = SIEVE_ERR_INVALID;
        break;
      }
      done++;
    }
  } while (0);
  fclose(f);
  cudaFree(d_out);
  if (h_out) cudaFreeHost(h_out);
  if (n_written) *n_written = st[4];
  if (rc != SIEVE_OK) return rc;
  return st[3] < hi ? SIEVE_PENDING : SIEVE_OK;
}
