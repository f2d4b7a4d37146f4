/*
 * oracle.h -- plain, slow, obviously correct CPU reference for the prime sieve.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  The GPU
 * library never links, includes or calls anything here, and nothing here
 * includes or calls the GPU library.
 *
 * What it computes is the plain definition of the Sieve of Eratosthenes
 * (Section 1.1, Figure 1) restricted to a half-open range [lo, hi): a byte
 * per integer, every multiple of every base prime p <= isqrt(hi - 1) from
 * max(p*p, first multiple >= lo) crossed off, survivors >= 2 reported.  It has
 * no 6k+1 / 6k+5 residue arrays, no Table 1 index arithmetic and no wheel.
 * The range is split into contiguous per-thread chunks (Section 2.2 / 2.3),
 * and each chunk is processed in 1 MiB byte segments (the scratch size that
 * Section 5 found best).
 *
 * Every function's pin (what fixes its value independently of this file) is
 * listed in tests/test_oracle_pins.py.
 */
#ifndef SIEVE_ORACLE_H
#define SIEVE_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (mirrors the meaning, not the header, of the GPU library). */
#define ORACLE_OK 0
#define ORACLE_ERR_INVALID (-1)
#define ORACLE_ERR_RANGE (-2)
#define ORACLE_ERR_CAPACITY (-3)
#define ORACLE_ERR_OOM (-4)

/* floor(sqrt(n)) in exact integer arithmetic (Newton iteration from above,
 * then a final +-1 correction).  Valid for every n < 2^64. */
uint64_t oracle_isqrt(uint64_t n);

/* The primes <= n (n < 2^32; Section 1.1), from the definition: m >= 2 is
 * prime iff no prime q <= isqrt(m) divides it.  The primes q <= isqrt(n) come
 * from this function itself (recursively, down to n < 4), and oracle_range
 * crosses off their multiples >= q*q in [0, n].  Writes the primes <= n
 * (increasing) to out[0..cap) and returns how many primes <= n there are
 * (which may exceed cap), or a negative status. */
int64_t oracle_primes_upto(uint64_t n, uint32_t *out, size_t cap);

/* Primes in [lo, hi) by the segmented byte sieve described above.
 *   base / nbase / base_limit : every prime <= base_limit, increasing (from
 *                    oracle_primes_upto(base_limit)), or base == NULL to let
 *                    the call build them itself.  base_limit < isqrt(hi - 1)
 *                    is ORACLE_ERR_RANGE.
 *   nthreads       : host threads; <= 0 means every core this process may use.
 *   count, sum     : number of primes and their sum modulo 2^64 (may be NULL).
 *   list, cap      : when list != NULL the primes are written in increasing
 *                    order to list[0..cap); *n_list receives the number found.
 *                    If that number exceeds cap the call returns
 *                    ORACLE_ERR_CAPACITY and list is unspecified.
 *   seg_width, bins, nbins : when bins != NULL, bins[i] counts the primes p of
 *                    the range with floor(p / seg_width) - floor(lo / seg_width)
 *                    == i; nbins must equal
 *                    floor((hi - 1) / seg_width) - floor(lo / seg_width) + 1.
 * lo > hi is ORACLE_ERR_INVALID; lo == hi gives zero of everything.
 * Valid for hi <= 2^63. */
int oracle_range(uint64_t lo, uint64_t hi, const uint32_t *base, size_t nbase,
                 uint64_t base_limit, int nthreads, uint64_t *count, uint64_t *sum, uint64_t *list,
                 size_t cap, size_t *n_list, uint64_t seg_width, uint64_t *bins,
                 size_t nbins);

/* Trial division by every d with d*d <= n: the definition of primality. */
int oracle_is_prime_td(uint64_t n);

/* Deterministic Miller-Rabin for 64-bit n with the first twelve primes as
 * bases (deterministic far beyond 2^64), 128-bit modular products. */
int oracle_is_prime_mr(uint64_t n);

/* Smallest v >= M with v % P == 0 and v % 6 == r (r in {1, 5}, P coprime to
 * 6): the plain definition of the start index that Table 1 produces.  With
 * from_square != 0 the search starts at max(M, P*P) instead (Section 2.4: a
 * prime starts sieving only at its square). */
uint64_t oracle_first_class_multiple(uint64_t M, uint64_t P, int r, int from_square);

/* Number of host threads oracle_range uses when nthreads <= 0. */
int oracle_default_threads(void);

#ifdef __cplusplus
}
#endif

#endif
