// Diagnostic kernel of the library: one bounded device wait made to run out
// (twopaco_selftest_bounded_wait), so that the failure path of the emit's
// look-back -- give up after a poll limit and report, never hang -- is tested.
#include "twopaco_internal.h"

namespace twopaco {
namespace {

// The emit's poll limit (kSpinLimit in twopaco_kernels.cu) and back-off.
constexpr uint32_t kPolls = 1u << 22;

// Polls *word, which nothing sets, like the emit's look-back polls a tile's
// status: *status = 1 when it gives up, 2 if it saw the word set.
__global__ void bounded_wait_kernel(volatile unsigned long long* word, unsigned int* status) {
  uint32_t spins = 0;
  for (;;) {
    if (*word) {
      *status = 2;
      return;
    }
    if (++spins > kPolls) {
      *status = 1;
      return;
    }
    __nanosleep(32);
  }
}

}  // namespace

int launch_bounded_wait(unsigned long long* word, unsigned int* status, cudaStream_t s) {
  bounded_wait_kernel<<<1, 1, 0, s>>>(word, status);
  if (cudaPeekAtLastError() != cudaSuccess) return -1;
  count_launches(1);
  return 1;
}

}  // namespace twopaco
