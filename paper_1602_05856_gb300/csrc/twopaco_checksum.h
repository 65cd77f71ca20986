// Checksum of a checkpoint's payload (host code only, no CUDA): a damaged,
// truncated-and-padded or reordered payload changes it, so that a checkpoint
// whose bits changed on disk is refused instead of resuming from wrong state.
#ifndef TWOPACO_CHECKSUM_H_
#define TWOPACO_CHECKSUM_H_

#include <cstdint>
#include <cstring>

namespace twopaco {

// splitmix64's output function (Steele, Lea & Flood, "Fast splittable
// pseudorandom number generators", 2014): a bijection on 64-bit words that
// spreads every input bit over the whole output.
inline uint64_t checksum_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// Order-dependent sum of n bytes: every 8-byte little-endian word (the last
// one zero-padded) is folded into the running state together with its
// offset, and the length seeds the state.
inline uint64_t payload_checksum(const void* data, uint64_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(data);
  uint64_t h = checksum_mix(n ^ 0x9e3779b97f4a7c15ull);
  uint64_t i = 0;
  for (; i + 8 <= n; i += 8) {
    uint64_t w;
    std::memcpy(&w, b + i, 8);
    h = checksum_mix(h ^ w) + i;
  }
  if (i < n) {
    uint64_t w = 0;
    std::memcpy(&w, b + i, n - i);
    h = checksum_mix(h ^ w) + i;
  }
  return checksum_mix(h);
}

}  // namespace twopaco

#endif  // TWOPACO_CHECKSUM_H_
