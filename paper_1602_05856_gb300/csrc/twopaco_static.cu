// twopaco_run_device_noalloc: the device-resident run with its workspace in a
// fixed, statically allocated device buffer instead of caller memory, for
// callers that cannot allocate device memory themselves.
#include <mutex>

#include "twopaco.h"
#include "twopaco_internal.h"

namespace {

// The scratch workspace. Every GPU that loads this library holds these
// TWOPACO_NOALLOC_SCRATCH_BYTES until the process exits. Host code may not use
// the symbol's name as a device address: it takes the address from
// cudaGetSymbolAddress, once per device, in scratch_address() below.
static __device__ __align__(256) unsigned char g_scratch[TWOPACO_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_address[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up on the first
// call made on that device (with the device current) and reused afterwards.
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TWOPACO_ECUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_address[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return TWOPACO_ECUDA;
    g_address[dev] = p;
  }
  *out = g_address[dev];
  return TWOPACO_OK;
}

}  // namespace

extern "C" int twopaco_run_device_noalloc(const uint8_t* d_bases, const uint64_t* d_offsets,
                                          uint64_t n_seqs, uint64_t total_bases, int k,
                                          uint64_t filter_bits, int rounds,
                                          const twopaco_options* opt, uint64_t* d_out_offsets,
                                          uint64_t* d_out_positions, uint64_t out_capacity,
                                          twopaco_stats* stats) {
  uint64_t need = 0;
  int rc = twopaco_workspace_size(total_bases, n_seqs, k, filter_bits, rounds, opt, &need);
  if (rc) return rc;
  if (need > TWOPACO_NOALLOC_SCRATCH_BYTES) return TWOPACO_ESCRATCH;
  void* ws = nullptr;
  if ((rc = scratch_address(&ws))) return rc;
  rc = twopaco_run_device(d_bases, d_offsets, n_seqs, total_bases, k, filter_bits, rounds, opt, ws,
                          TWOPACO_NOALLOC_SCRATCH_BYTES, d_out_offsets, d_out_positions, out_capacity);
  if (rc) return rc;
  twopaco_stats st{};
  rc = twopaco_read_stats(ws, opt ? opt->cuda_stream : nullptr, &st);
  if (stats) *stats = st;
  return rc;
}
