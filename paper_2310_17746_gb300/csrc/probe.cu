// probe.cu -- measurement of the device resource the strike loops are bound
// by: 32-bit shared-memory atomic AND throughput.  Used for roofline reporting;
// the paper has no counterpart.
//
// One CTA of 1024 threads per SM fills 128 KB of shared memory, then every
// thread issues `iters` atomic ANDs, either conflict-free (lane l of a warp
// always hits bank l) or at pseudo-random words; thread 0 times the loop with
// clock64.  Every index is masked into the buffer.  The result is lane
// operations per SM clock (clock-independent).
#include <cstdint>

#include "sieve_internal.cuh"

namespace {

constexpr uint32_t kProbeWords = 32768;  // 128 KB
constexpr int kProbeIters = 4096;

__global__ void __launch_bounds__(1024, 1) smem_atomics_probe(unsigned long long *cycles, uint32_t *sink, int mode) {
  extern __shared__ uint32_t s[];
  for (uint32_t w = threadIdx.x; w < kProbeWords; w += blockDim.x) s[w] = 0xFFFFFFFFu;
  __syncthreads();
  uint32_t x = threadIdx.x * 2654435761u + blockIdx.x;
  const long long t0 = clock64();
  if (mode == 0) {
    uint32_t k = threadIdx.x;  // consecutive lanes, consecutive words: 32 banks
#pragma unroll 8
    for (int i = 0; i < kProbeIters; i++) {
      atomicAnd(s + (k & (kProbeWords - 1)), ~(1u << (i & 31)));
      k += 1056;
    }
  } else {
#pragma unroll 8
    for (int i = 0; i < kProbeIters; i++) {
      x = x * 1664525u + 1013904223u;
      atomicAnd(s + (x >> 17), ~(1u << (i & 31)));  // x >> 17 < 32768
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
  for (uint32_t w = threadIdx.x; w < kProbeWords; w += blockDim.x) acc ^= s[w];
  if (threadIdx.x == 0) {
    cycles[blockIdx.x] = (unsigned long long)(t1 - t0);
    sink[blockIdx.x] = acc;  // keeps the loop's effect observable
  }
}

}  // namespace

using namespace sieve;

extern "C" int sieve_measure_smem_atomics(int device, double *conflict_free, double *random_banks) {
  if (!conflict_free || !random_banks) {
    set_error("sieve_measure_smem_atomics: NULL argument");
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaSetDevice(device));
  int sms = 0, optin = 0;
  SIEVE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  SIEVE_CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
  const size_t smem = kProbeWords * sizeof(uint32_t);
  if ((size_t)optin < smem) {
    set_error("device offers %d bytes of shared memory per block; the probe needs %zu", optin, smem);
    return SIEVE_ERR_INVALID;
  }
  SIEVE_CUDA_TRY(cudaFuncSetAttribute(smem_atomics_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  unsigned long long *d_cycles = nullptr;
  uint32_t *d_sink = nullptr;
  SIEVE_CUDA_TRY(cudaMalloc(&d_cycles, (size_t)sms * sizeof(unsigned long long)));
  cudaError_t e = cudaMalloc(&d_sink, (size_t)sms * sizeof(uint32_t));
  double rate[2] = {0.0, 0.0};
  std::vector<unsigned long long> h(sms);
  for (int mode = 0; mode < 2 && e == cudaSuccess; mode++) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // the first run warms up
      smem_atomics_probe<<<sms, 1024, smem>>>(d_cycles, d_sink, mode);
      e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), d_cycles, (size_t)sms * sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) {
      unsigned long long worst = 1;
      for (unsigned long long c : h) worst = c > worst ? c : worst;
      rate[mode] = 1024.0 * kProbeIters / (double)worst;
    }
  }
  cudaFree(d_cycles);
  cudaFree(d_sink);
  if (e != cudaSuccess) return cuda_fail(e, "smem_atomics_probe");
  *conflict_free = rate[0];
  *random_banks = rate[1];
  return SIEVE_OK;
}
