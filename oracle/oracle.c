/*
 * oracle.c -- plain CPU reference for the prime sieve.  TEST INFRASTRUCTURE
 * ONLY (see oracle.h for who may use it and what it computes).
 *
 * Nothing here is tuned: one byte per integer, a fresh start offset for every
 * base prime in every segment, and two plain passes (count, then write) when a
 * sorted list is asked for.
 */
#define _GNU_SOURCE
#include "oracle.h"

#include <pthread.h>
#include <sched.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_SEGMENT_BYTES ((uint64_t)1 << 20) /* Section 5: 1M entries was best */

/* ------------------------------------------------------------------------ */
/* isqrt: Newton's iteration x <- (x + n/x) / 2 started above sqrt(n) decreases
 * monotonically to floor(sqrt(n)); the loop stops at the first non-decrease.
 * The two correction loops make the result exact whatever the start. */
uint64_t oracle_isqrt(uint64_t n) {
  if (n < 2) return n;
  int bits = 64 - __builtin_clzll(n);
  uint64_t x = (uint64_t)1 << ((bits + 1) / 2); /* x >= sqrt(n), x <= 2^32 */
  for (;;) {
    uint64_t y = (x + n / x) / 2;
    if (y >= x) break;
    x = y;
  }
  while (x > 0 && x > n / x) x--;                       /* x*x > n  */
  while ((x + 1) <= n / (x + 1)) x++;                   /* (x+1)^2 <= n */
  return x;
}

/* ------------------------------------------------------------------------ */
/* The primes <= n (Section 1.1: all primes from 2 through n), by the
 * definition of primality: m >= 2 is prime iff no prime q <= isqrt(m) divides
 * m.  A composite m <= n has its smallest prime factor q <= isqrt(m) <= isqrt(n)
 * and m >= q*q, so the primes <= n are what survives in [2, n] once every
 * multiple >= q*q of every prime q <= isqrt(n) is crossed off -- which is what
 * oracle_range does for [0, n + 1) given those primes.  They come from this
 * same function for isqrt(n); the chain ends at n < 4, where isqrt(n) < 2 and
 * nothing needs crossing off. */
int64_t oracle_primes_upto(uint64_t n, uint32_t *out, size_t cap) {
  if (n < 2) return 0;
  if (n > 0xFFFFFFFFull) return ORACLE_ERR_RANGE; /* primes are stored as uint32 */
  const uint64_t r = oracle_isqrt(n);
  int64_t nb = oracle_primes_upto(r, NULL, 0);
  if (nb < 0) return nb;
  uint32_t *base = (uint32_t *)malloc(((size_t)nb + 1) * sizeof(uint32_t));
  if (!base) return ORACLE_ERR_OOM;
  oracle_primes_upto(r, base, (size_t)nb);
  uint64_t count = 0;
  int rc = oracle_range(0, n + 1, base, (size_t)nb, r, 0, &count, NULL, NULL, 0, NULL, 0, NULL, 0);
  if (rc == ORACLE_OK && out && cap) {
    uint64_t *tmp = (uint64_t *)malloc(((size_t)count + 1) * sizeof(uint64_t));
    size_t got = 0;
    if (!tmp) {
      rc = ORACLE_ERR_OOM;
    } else {
      rc = oracle_range(0, n + 1, base, (size_t)nb, r, 0, NULL, NULL, tmp, (size_t)count, &got, 0, NULL, 0);
      for (size_t i = 0; rc == ORACLE_OK && i < got && i < cap; i++) out[i] = (uint32_t)tmp[i];
      free(tmp);
    }
  }
  free(base);
  return rc == ORACLE_OK ? (int64_t)count : rc;
}

/* ------------------------------------------------------------------------ */
/* One thread's share of [lo, hi): a contiguous chunk [a, b). */
typedef struct {
  uint64_t a, b;            /* chunk */
  uint64_t lo;              /* whole range start (for bin numbering) */
  const uint32_t *base;
  size_t nbase;
  uint64_t count, sum;      /* results */
  uint64_t seg_width;
  uint64_t *bins;           /* private bins (nbins), or NULL */
  size_t nbins;
  uint64_t *list;           /* second pass: where this chunk's primes go */
  int err;
} chunk_job;

/* Sieve [a, b) segment by segment; call back on each prime found.  The start
 * for prime p in the segment [s, e) is m = max(p*p, ceil(s/p)*p). */
static void sieve_chunk(chunk_job *job, int write_list) {
  uint8_t *seg = (uint8_t *)malloc(ORACLE_SEGMENT_BYTES);
  if (!seg) {
    job->err = ORACLE_ERR_OOM;
    return;
  }
  uint64_t written = 0;
  uint64_t first_bin = job->seg_width ? job->lo / job->seg_width : 0;
  for (uint64_t s = job->a; s < job->b;) {
    uint64_t e = job->b - s > ORACLE_SEGMENT_BYTES ? s + ORACLE_SEGMENT_BYTES : job->b;
    size_t len = (size_t)(e - s);
    memset(seg, 1, len);
    for (size_t i = 0; i < job->nbase; i++) {
      uint64_t p = job->base[i];
      if (p * p > e - 1) break; /* base is increasing */
      uint64_t m = ((s + p - 1) / p) * p;
      if (m < p * p) m = p * p;
      for (; m < e; m += p) seg[m - s] = 0;
    }
    for (size_t i = 0; i < len; i++) {
      uint64_t v = s + i;
      if (!seg[i] || v < 2) continue;
      job->count++;
      job->sum += v;
      if (job->bins) job->bins[v / job->seg_width - first_bin]++;
      if (write_list) job->list[written++] = v;
    }
    s = e;
  }
  free(seg);
}

static void *count_thread(void *arg) {
  sieve_chunk((chunk_job *)arg, 0);
  return NULL;
}

static void *list_thread(void *arg) {
  sieve_chunk((chunk_job *)arg, 1);
  return NULL;
}

int oracle_default_threads(void) {
  cpu_set_t set;
  if (sched_getaffinity(0, sizeof(set), &set) == 0) {
    int c = CPU_COUNT(&set);
    if (c > 0) return c;
  }
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

static int run_threads(chunk_job *jobs, int nt, void *(*fn)(void *)) {
  pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
  if (!th) return ORACLE_ERR_OOM;
  int started = 0;
  for (int t = 0; t < nt; t++) {
    if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) {
      fn(&jobs[t]); /* run inline if no thread could be made */
      th[t] = 0;
    } else {
      started++;
    }
  }
  for (int t = 0; t < nt; t++)
    if (th[t]) pthread_join(th[t], NULL);
  free(th);
  (void)started;
  for (int t = 0; t < nt; t++)
    if (jobs[t].err) return jobs[t].err;
  return ORACLE_OK;
}

int oracle_range(uint64_t lo, uint64_t hi, const uint32_t *base, size_t nbase,
                 uint64_t base_limit, int nthreads, uint64_t *count, uint64_t *sum, uint64_t *list,
                 size_t cap, size_t *n_list, uint64_t seg_width, uint64_t *bins,
                 size_t nbins) {
  if (lo > hi) return ORACLE_ERR_INVALID;
  if (count) *count = 0;
  if (sum) *sum = 0;
  if (n_list) *n_list = 0;
  if (bins && seg_width == 0) return ORACLE_ERR_INVALID;
  if (bins && hi > lo) {
    uint64_t need = (hi - 1) / seg_width - lo / seg_width + 1;
    if (nbins != need) return ORACLE_ERR_INVALID;
    memset(bins, 0, nbins * sizeof(uint64_t));
  }
  if (lo == hi) return ORACLE_OK;

  uint64_t s = oracle_isqrt(hi - 1);
  uint32_t *own = NULL;
  if (base == NULL) {
    int64_t np = oracle_primes_upto(s, NULL, 0);
    if (np < 0) return (int)np;
    own = (uint32_t *)malloc(((size_t)np + 1) * sizeof(uint32_t));
    if (!own) return ORACLE_ERR_OOM;
    oracle_primes_upto(s, own, (size_t)np);
    base = own;
    nbase = (size_t)np;
  } else if (base_limit < s) {
    return ORACLE_ERR_RANGE; /* the caller's table must hold every prime <= s */
  }

  int nt = nthreads > 0 ? nthreads : oracle_default_threads();
  uint64_t width = hi - lo;
  if ((uint64_t)nt > width) nt = (int)width;
  chunk_job *jobs = (chunk_job *)calloc((size_t)nt, sizeof(chunk_job));
  if (!jobs) {
    free(own);
    return ORACLE_ERR_OOM;
  }
  for (int t = 0; t < nt; t++) {
    jobs[t].a = lo + width / (uint64_t)nt * (uint64_t)t;
    jobs[t].b = (t == nt - 1) ? hi : lo + width / (uint64_t)nt * (uint64_t)(t + 1);
    jobs[t].lo = lo;
    jobs[t].base = base;
    jobs[t].nbase = nbase;
    jobs[t].seg_width = seg_width;
    if (bins) {
      jobs[t].bins = (uint64_t *)calloc(nbins, sizeof(uint64_t));
      jobs[t].nbins = nbins;
      if (!jobs[t].bins) jobs[t].err = ORACLE_ERR_OOM;
    }
  }
  int rc = run_threads(jobs, nt, count_thread);
  uint64_t c = 0, sm = 0;
  for (int t = 0; t < nt && rc == ORACLE_OK; t++) {
    c += jobs[t].count;
    sm += jobs[t].sum;
    if (bins)
      for (size_t i = 0; i < nbins; i++) bins[i] += jobs[t].bins[i];
  }
  if (rc == ORACLE_OK) {
    if (count) *count = c;
    if (sum) *sum = sm;
    if (n_list) *n_list = (size_t)c;
  }
  if (rc == ORACLE_OK && list) {
    if (c > cap) {
      rc = ORACLE_ERR_CAPACITY;
    } else {
      /* second pass: each chunk writes at the exclusive prefix of the counts */
      uint64_t off = 0;
      for (int t = 0; t < nt; t++) {
        jobs[t].list = list + off;
        off += jobs[t].count;
        jobs[t].count = 0;
        jobs[t].sum = 0;
        if (jobs[t].bins) {
          free(jobs[t].bins);
          jobs[t].bins = NULL;
        }
      }
      rc = run_threads(jobs, nt, list_thread);
    }
  }
  for (int t = 0; t < nt; t++) free(jobs[t].bins);
  free(jobs);
  free(own);
  return rc;
}

/* ------------------------------------------------------------------------ */
int oracle_is_prime_td(uint64_t n) {
  if (n < 2) return 0;
  for (uint64_t d = 2; d <= n / d; d++)
    if (n % d == 0) return 0;
  return 1;
}

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t m) {
  return (uint64_t)(((unsigned __int128)a * b) % m);
}

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t m) {
  uint64_t r = 1 % m;
  a %= m;
  while (e) {
    if (e & 1) r = mulmod(r, a, m);
    a = mulmod(a, a, m);
    e >>= 1;
  }
  return r;
}

int oracle_is_prime_mr(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    s++;
  }
  for (int i = 0; i < 12; i++) {
    uint64_t x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int composite = 1;
    for (int j = 1; j < s; j++) {
      x = mulmod(x, x, n);
      if (x == n - 1) {
        composite = 0;
        break;
      }
    }
    if (composite) return 0;
  }
  return 1;
}

/* ------------------------------------------------------------------------ */
uint64_t oracle_first_class_multiple(uint64_t M, uint64_t P, int r, int from_square) {
  if (from_square && M < P * P) M = P * P;
  uint64_t v = ((M + P - 1) / P) * P;
  while (v % 6 != (uint64_t)r) v += P;
  return v;
}
