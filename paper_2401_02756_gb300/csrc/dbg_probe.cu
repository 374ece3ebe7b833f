// K5: random 32-byte-sector traffic, the measured ceiling the insert kernel
// is rated against.  The insert touches one random slot (one sector) per
// vertex; these kernels do exactly that and nothing else, over a buffer the
// size of the table, so that their rate is the best the memory system gives
// for the access pattern.
#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

__global__ void k_probe(Slot *buf, uint64_t n_slots, uint64_t n_ops, uint64_t seed, int mode,
                        unsigned long long *sink) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  unsigned long long acc = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride) {
    const uint64_t h = fmix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
    const uint64_t s = __umul64hi(h, n_slots);
    const uint32_t w = (uint32_t)(h >> 62);
    if (mode == 0) {
      atomicAdd(&buf[s].cnt[w], 1u);
    } else if (mode == 1) {
      const unsigned long long v = ld_relaxed_u64(&buf[s].key);
      atomicAdd(&buf[s].cnt[w], (uint32_t)(v & 1ull) | 1u);  // depends on the load
    } else {
      acc += atomicCAS(&buf[s].key, (unsigned long long)s, (unsigned long long)(s ^ 1ull));
    }
  }
  if (mode == 2 && acc == 0x5a5a5a5a5a5a5a5aull) *sink = acc;  // keep the CAS results live
}

// Load + atomicAdd on a random slot of a window of `window` slots that
// slides linearly across the buffer as the operation index grows: the access
// pattern of a region-ordered stream of table updates.
// `scale` = floor((n_slots - window) * 2^64 / n_ops), so that the window
// start of operation i is mulhi(i, scale).
__global__ void k_probe_window(Slot *buf, uint64_t n_slots, uint64_t n_ops, uint64_t window,
                               uint64_t scale, uint64_t seed, int flags) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t pol = l2_policy_evict_last();
  const int evict_last = flags & 1;
  unsigned long long acc = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_ops; i += stride) {
    const uint64_t h = fmix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
    const uint64_t start = __umul64hi(i, scale);
    const uint64_t s = start + __umul64hi(h, window);
    if (flags & 2) {  // loads only
      acc += ld_relaxed_u64(&buf[s].key);
    } else if (flags & 4) {  // adds only
      atomicAdd(&buf[s].cnt[(uint32_t)(h >> 62)], 1u);
    } else if (evict_last) {
      const unsigned long long v = ld_relaxed_u64_hint(&buf[s].key, pol);
      red_add_u32_hint(&buf[s].cnt[(uint32_t)(h >> 62)], (uint32_t)(v & 1ull) | 1u, pol);
    } else {
      const unsigned long long v = ld_relaxed_u64(&buf[s].key);
      atomicAdd(&buf[s].cnt[(uint32_t)(h >> 62)], (uint32_t)(v & 1ull) | 1u);
    }
  }
  if (acc == 0x5a5a5a5a5a5a5a5aull) buf[0].pad[0] = 1u;  // keep the loads live
}

}  // namespace
}  // namespace dbg

extern "C" int dbg_probe_window(void *buf, uint64_t n_slots, uint64_t n_ops, uint64_t window_slots,
                                uint64_t seed, int flags, void *stream) {
  using namespace dbg;
  if (!buf || n_slots == 0 || window_slots == 0 || window_slots > n_slots || ((uintptr_t)buf & 31u) ||
      flags < 0 || flags > 7)
    return DBG_ERR_INVALID_ARG;
  if (n_ops == 0) return DBG_OK;
  int dev = 0, sms = 0, per_sm = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe_window, 256, 0));
  const uint64_t want = (n_ops + 255) / 256;
  const int grid = (int)std::min<uint64_t>(want, (uint64_t)std::max(1, per_sm) * sms);
  const uint64_t scale =
      (uint64_t)((((unsigned __int128)(n_slots - window_slots)) << 64) / n_ops);
  k_probe_window<<<std::max(1, grid), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<Slot *>(buf), n_slots, n_ops, window_slots, scale, seed, flags);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

extern "C" int dbg_probe_random_sectors(void *buf, uint64_t n_slots, uint64_t n_ops, uint64_t seed,
                                        int mode, void *stream) {
  using namespace dbg;
  if (!buf || n_slots == 0 || mode < 0 || mode > 2 || ((uintptr_t)buf & 31u))
    return DBG_ERR_INVALID_ARG;
  if (n_ops == 0) return DBG_OK;
  int dev = 0, sms = 0, per_sm = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe, 256, 0));
  const uint64_t want = (n_ops + 255) / 256;
  const int grid = (int)std::min<uint64_t>(want, (uint64_t)std::max(1, per_sm) * sms);
  k_probe<<<std::max(1, grid), 256, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<Slot *>(buf), n_slots, n_ops, seed, mode,
      reinterpret_cast<unsigned long long *>(buf));
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}
