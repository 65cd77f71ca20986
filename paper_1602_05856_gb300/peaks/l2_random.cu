// Roofline denominators for the filter kernels: the rate at which this GPU
// serves random 32-byte sector reads and random 64-bit atomic ORs from a
// buffer of a given size (L2-resident when it is smaller than L2).
// Not part of the junction method; the benchmark calls it before timing.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

__device__ __forceinline__ uint64_t mix(uint64_t z) {
  z ^= z >> 33;
  z *= 0xff51afd7ed558ccdull;
  z ^= z >> 33;
  z *= 0xc4ceb9fe1a85ec53ull;
  z ^= z >> 33;
  return z;
}

__global__ void __launch_bounds__(256) sector_reads(const ulonglong2* __restrict__ buf,
                                                   uint64_t block_mask, int iters,
                                                   unsigned long long* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t acc = 0;
  uint64_t h = mix(tid + 1);
  for (int it = 0; it < iters; ++it) {
    h = mix(h + 0x9e3779b97f4a7c15ull);
    const uint64_t b = h & block_mask;
    const ulonglong2 a = __ldcg(buf + 2 * b), c = __ldcg(buf + 2 * b + 1);
    acc ^= a.x ^ a.y ^ c.x ^ c.y;
  }
  if (acc == 0x1234567ull) sink[0] = acc;  // keeps the loads alive
}

__global__ void __launch_bounds__(256) word_reads(const unsigned long long* __restrict__ buf,
                                                 uint64_t word_mask, int iters,
                                                 unsigned long long* sink) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t acc = 0;
  uint64_t h = mix(tid + 3);
  for (int it = 0; it < iters; ++it) {
    h = mix(h + 0x9e3779b97f4a7c15ull);
    acc ^= __ldcg(buf + (h & word_mask));
  }
  if (acc == 0x1234567ull) sink[0] = acc;
}

__global__ void __launch_bounds__(256) sector_ors(unsigned long long* __restrict__ buf,
                                                 uint64_t block_mask, int iters) {
  const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint64_t h = mix(tid + 7);
  for (int it = 0; it < iters; ++it) {
    h = mix(h + 0x9e3779b97f4a7c15ull);
    const uint64_t b = h & block_mask;
    atomicOr(buf + 4 * b + ((h >> 40) & 3), 1ull << ((h >> 48) & 63));
  }
}

// The same three access kinds with cheap addresses: a 32-bit linear
// congruential sequence per thread (Numerical Recipes' constants; one
// multiply-add per access), its high bits scaled to the buffer. Four
// independent accesses per step keep more requests in flight; nothing depends
// on loaded data, so the loop issues as fast as the memory system takes it.
__device__ __forceinline__ uint32_t lcg(uint32_t x) { return x * 1664525u + 1013904223u; }

__global__ void __launch_bounds__(256) sector_reads_lcg(const ulonglong2* __restrict__ buf, int lg_units,
                                                        int iters, unsigned long long* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[4];
  for (int j = 0; j < 4; ++j) x[j] = (uint32_t)mix(4ull * tid + j + 1);
  uint64_t acc = 0;
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = lcg(x[j]);
      const uint64_t b = lg_units ? (x[j] >> (32 - lg_units)) : 0;
      const ulonglong2 a = __ldcg(buf + 2 * b), c = __ldcg(buf + 2 * b + 1);
      acc ^= a.x ^ a.y ^ c.x ^ c.y;
    }
  }
  if (acc == 0x1234567ull) sink[0] = acc;
}

__global__ void __launch_bounds__(256) word_reads_lcg(const unsigned long long* __restrict__ buf, int lg_units,
                                                      int iters, unsigned long long* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[4];
  for (int j = 0; j < 4; ++j) x[j] = (uint32_t)mix(4ull * tid + j + 3);
  uint64_t acc = 0;
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = lcg(x[j]);
      acc ^= __ldcg(buf + (lg_units ? (x[j] >> (32 - lg_units)) : 0));
    }
  }
  if (acc == 0x1234567ull) sink[0] = acc;
}

__global__ void __launch_bounds__(256) sector_ors_lcg(unsigned long long* __restrict__ buf, int lg_units,
                                                      int iters) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t x[4];
  for (int j = 0; j < 4; ++j) x[j] = (uint32_t)mix(4ull * tid + j + 7);
  for (int it = 0; it < iters; it += 4) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      x[j] = lcg(x[j]);
      const uint64_t b = lg_units ? (x[j] >> (32 - lg_units)) : 0;
      atomicOr(buf + 4 * b + (x[j] & 3u), 1ull << ((x[j] >> 2) & 63u));
    }
  }
}

int log2_of(uint64_t x) {
  int l = 0;
  while ((1ull << l) < x) ++l;
  return l;
}

}  // namespace

extern "C" {

// mode 0: random 32-byte sector reads; mode 1: random 64-bit ORs (one per
// sector); mode 2: random 8-byte reads; modes 3, 4, 5: the same with the
// linear-congruential addresses (iters a multiple of 4; buffers of at most
// 2^32 units of 32 or 8 bytes).
// buf_bytes: power of two >= 32. Returns sector operations per second, or a
// negative value on a CUDA error. Allocates and frees its own buffer.
double peaks_l2_random_rate(int mode, uint64_t buf_bytes, int iters, int reps) {
  void* buf = nullptr;
  unsigned long long* sink = nullptr;
  if (cudaMalloc(&buf, buf_bytes) != cudaSuccess) return -1.0;
  if (cudaMalloc(&sink, 8) != cudaSuccess) { cudaFree(buf); return -1.0; }
  cudaMemset(buf, 0, buf_bytes);
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (mode == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sector_reads, 256, 0);
  else if (mode == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sector_ors, 256, 0);
  else if (mode == 2) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, word_reads, 256, 0);
  else if (mode == 3) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sector_reads_lcg, 256, 0);
  else if (mode == 4) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sector_ors_lcg, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, word_reads_lcg, 256, 0);
  if (mode < 0 || mode > 5 || (mode >= 3 && (iters % 4 || buf_bytes / 8 > (1ull << 32)))) {
    cudaFree(sink);
    cudaFree(buf);
    return -1.0;
  }
  const unsigned grid = (unsigned)(sms * (per_sm > 0 ? per_sm : 1));
  const uint64_t mask = buf_bytes / 32 - 1;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 0.0;
  for (int r = 0; r <= reps; ++r) {  // first launch is a warm-up
    cudaEventRecord(a);
    if (mode == 0) sector_reads<<<grid, 256>>>(static_cast<const ulonglong2*>(buf), mask, iters, sink);
    else if (mode == 1) sector_ors<<<grid, 256>>>(static_cast<unsigned long long*>(buf), mask, iters);
    else if (mode == 2)
      word_reads<<<grid, 256>>>(static_cast<const unsigned long long*>(buf), buf_bytes / 8 - 1, iters, sink);
    else if (mode == 3)
      sector_reads_lcg<<<grid, 256>>>(static_cast<const ulonglong2*>(buf), log2_of(buf_bytes / 32), iters, sink);
    else if (mode == 4)
      sector_ors_lcg<<<grid, 256>>>(static_cast<unsigned long long*>(buf), log2_of(buf_bytes / 32), iters);
    else
      word_reads_lcg<<<grid, 256>>>(static_cast<const unsigned long long*>(buf), log2_of(buf_bytes / 8), iters,
                                    sink);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double rate = (double)grid * 256.0 * iters / (ms * 1e-3);
    if (r > 0 && rate > best) best = rate;
  }
  const bool bad = cudaGetLastError() != cudaSuccess;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(sink);
  cudaFree(buf);
  return bad ? -1.0 : best;
}

}  // extern "C"
