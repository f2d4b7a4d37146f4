// cluster.cuh -- cluster segments: one segment of C consecutive tiles sieved
// by a thread-block cluster of C CTAs through distributed shared memory.
//
// Sections 2.2-2.3 give each worker one contiguous chunk and Section 5 varies
// the chunk (array) size.  On a GB300 a CTA's chunk is one tile in its own
// shared memory (at most 227 KB); a cluster of C CTAs (up to 8 portable, 16
// opt-in) can address the tiles of all its members, so the C tiles form one
// segment of C L indices per class:
//
//   * Every CTA presieves its own tile and strikes the primes up to
//     cluster_threshold x L into it itself (warp band and one-lane band, as
//     in the plain tile path).
//   * The primes above that are split over the cluster's C CTAs (prime i to
//     rank i / BLOCK mod C, one lane per prime): each is located once per
//     segment (its first class-1 and class-5 index at or after max(segment
//     start, P^2), from the inverse-of-6 constants) and walked through the
//     segment by steps of P.  A hit in the CTA's own tile is a shared-memory
//     atomic AND; a hit in another member's tile is a `red.shared::cluster`
//     AND into that member's shared memory (the address from `mapa`).
//   * Two cluster barriers per segment: after every member's presieve (so no
//     remote strike lands before the pattern copy) and after all strikes (so
//     every remote strike has landed before a member reads its tile).  The
//     barriers release and acquire at cluster scope, which orders the remote
//     ANDs before the owner's reads.
//
// A prime is thus located once per C tiles instead of once per tile, at the
// price of remote strikes, which the GB300's SM-to-SM network serves far
// more slowly than an SM serves its own shared memory.
#pragma once

#include "tile.cuh"

namespace sieve {

// Both barrier halves, by every thread of every CTA of the cluster (the
// .aligned forms: all threads of a warp execute them together).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::
          : "memory");
}

// Rank of this CTA in its (one-dimensional) cluster.
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// The shared::cluster address of the word at shared::cta address `saddr` in
// the shared memory of cluster member `rank`.
__device__ __forceinline__ uint32_t cluster_map(uint32_t saddr, uint32_t rank) {
  uint32_t a;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(a) : "r"(saddr), "r"(rank));
  return a;
}

__device__ __forceinline__ void cluster_and(uint32_t caddr, uint32_t mask) {
  asm volatile("red.relaxed.cluster.shared::cluster.and.b32 [%0], %1;" ::"r"(caddr), "r"(mask) : "memory");
}

// Strike the primes with table index in [i_lo, np_seg) whose share falls to
// this CTA (rank `rank` of C) into the segment of `slen` indices per class
// starting at class index Ks, whose tile j (L = 2^(logW + 5) indices) is the
// shared memory of member j.  s1 / s5 are this CTA's class bitmaps; every
// member has them at the same shared-memory offsets.  Needs P < 2^31 for
// every prime (starts_from_inverse) and C L <= 2^31.
template <int BLOCK>
__device__ __forceinline__ void cluster_strike(uint32_t *s1, uint32_t *s5, uint32_t logW, uint64_t Ks, uint32_t slen,
                                               uint32_t rank, uint32_t C, const uint32_t *__restrict__ primes,
                                               const uint64_t *__restrict__ magic, const uint2 *__restrict__ cinv,
                                               uint32_t i_lo, uint32_t np_seg) {
  const uint32_t logL = logW + 5, lmask = (1u << logL) - 1, wmask = (1u << logW) - 1;
  const uint32_t a1 = (uint32_t)__cvta_generic_to_shared(s1), a5 = (uint32_t)__cvta_generic_to_shared(s5);
  auto hit = [&](uint32_t k, uint32_t *s, uint32_t a) {
    const uint32_t owner = k >> logL, kl = k & lmask;
    const uint32_t m = rotl32(0xFFFFFFFEu, kl >> logW);
    if (owner == rank)
      atomicAnd(s + (kl & wmask), m);
    else
      cluster_and(cluster_map(a + 4u * (kl & wmask), owner), m);
  };
  auto one = [&](uint32_t P, uint64_t m, uint2 c) {
    const uint64_t Kc = ((uint64_t)P * P - 1) / 6;  // P^2 = 6 Kc + 1: nothing to strike below P^2
    const uint64_t K0 = Ks > Kc ? Ks : Kc;
    if (K0 >= Ks + slen) return;
    uint32_t r1, r5;
    starts_from_inverse(K0, P, m, c, r1, r5);
    const uint64_t base = K0 - Ks;
    for (uint64_t k = base + r1; k < slen; k += P) hit((uint32_t)k, s1, a1);
    for (uint64_t k = base + r5; k < slen; k += P) hit((uint32_t)k, s5, a5);
  };
  // one lane per prime; the next prime's table entries are loaded before the
  // current one is struck, so that their latency overlaps the strikes (a
  // segment streams the whole table above i_lo)
  const uint64_t step = (uint64_t)C * BLOCK;
  uint64_t i = (uint64_t)i_lo + (uint64_t)rank * BLOCK + threadIdx.x;
  uint32_t P = 0;
  uint64_t m = 0;
  uint2 c = make_uint2(0, 0);
  if (i < np_seg) {
    P = __ldg(primes + i);
    m = __ldg(magic + i);
    c = __ldg(cinv + i);
  }
  while (i < np_seg) {
    const uint64_t in = i + step;
    uint32_t Pn = 0;
    uint64_t mn = 0;
    uint2 cn = make_uint2(0, 0);
    if (in < np_seg) {
      Pn = __ldg(primes + in);
      mn = __ldg(magic + in);
      cn = __ldg(cinv + in);
    }
    one(P, m, c);
    P = Pn;
    m = mn;
    c = cn;
    i = in;
  }
}

}  // namespace sieve
