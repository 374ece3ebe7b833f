// Sorted export of a graph (K3 compaction, K4 radix sort, gather): the
// (vertex, counters) table of the paper's Fig. 1 in key order, which is
// lexicographic order with A < C < G < T because keys hold the first base in
// their most significant bits.  Not on the timed insert path.
//
// The radix sort is CUB's DeviceRadixSort (open-source CCCL headers shipped
// with the CUDA toolkit); compaction and gather are this file's kernels.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

// K3: append (key, slot index) of every occupied slot; one atomicAdd per warp.
__global__ void k_compact(const Slot *t, uint64_t n_slots, unsigned long long *keys,
                          unsigned long long *idx, unsigned long long *count, uint64_t cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (((uint64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (uint64_t base = w0 * 32; base < n_slots; base += warps * 32) {
    const uint64_t i = base + lane;
    unsigned long long key = kEmpty;
    if (i < n_slots) key = __ldcs(&t[i].key);
    const bool occ = key != kEmpty;
    const unsigned mask = __ballot_sync(0xffffffffu, occ);
    unsigned long long pos = 0;
    if (lane == 0 && mask) pos = atomicAdd(count, (unsigned long long)__popc(mask));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const unsigned long long at = pos + __popc(mask & ((1u << lane) - 1u));
    if (occ && at < cap) {  // cap: vertices counted before; never write past the buffers
      keys[at] = key;
      idx[at] = i;
    }
  }
}

// Counters of the sorted vertices, in key order.
__global__ void k_gather(const Slot *t, const unsigned long long *idx, uint4 *counts, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    // the counters sit at byte 8 of the slot: 8-byte aligned, not 16
    const uint2 *c = reinterpret_cast<const uint2 *>(&t[idx[i]].cnt[0]);
    const uint2 lo = c[0], hi = c[1];
    counts[i] = make_uint4(lo.x, lo.y, hi.x, hi.y);
  }
}

struct Guard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit Guard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = err == cudaSuccess;
    }
  }
  ~Guard() {
    if (changed) cudaSetDevice(prev);
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace dbg

extern "C" int dbg_export_sorted(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                                 uint64_t max_n, uint64_t *n_out, void *stream) {
  using namespace dbg;
  if (!h || !n_out) return DBG_ERR_INVALID_ARG;
  Guard g(h->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  uint64_t D = 0;
  int st = dbg_stats(h, &D, nullptr, stream);
  if (st != DBG_OK) return st;
  *n_out = D;
  if (D > max_n) return DBG_ERR_BUFFER_TOO_SMALL;
  if (D == 0) return DBG_OK;
  if (h->k > 32) return export_sorted_wide(h, D, keys_out, counts_out, s);

  const int end_bit = 2 * (h->k - 1);
  size_t temp_bytes = 0;
  DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr, (int64_t)D, 0, end_bit, s));
  const size_t kb = align256(D * sizeof(unsigned long long));
  const size_t cb = align256(D * sizeof(uint4));
  const size_t total = 4 * kb + cb + 256 + align256(temp_bytes);
  char *buf = nullptr;
  DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), total, s));
  unsigned long long *keys_a = reinterpret_cast<unsigned long long *>(buf);
  unsigned long long *keys_b = reinterpret_cast<unsigned long long *>(buf + kb);
  unsigned long long *idx_a = reinterpret_cast<unsigned long long *>(buf + 2 * kb);
  unsigned long long *idx_b = reinterpret_cast<unsigned long long *>(buf + 3 * kb);
  uint4 *counts = reinterpret_cast<uint4 *>(buf + 4 * kb);
  unsigned long long *count = reinterpret_cast<unsigned long long *>(buf + 4 * kb + cb);
  void *temp = buf + 4 * kb + cb + 256;

  int rc = DBG_OK;
  do {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    const int grid = std::max(1, h->sm_count) * 8;
    k_compact<<<grid, 256, 0, s>>>(h->table, h->n_slots, keys_a, idx_a, count, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_compact"); break; }
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, keys_a, keys_b, idx_a, idx_b, (int64_t)D,
                                        0, end_bit, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceRadixSort::SortPairs"); break; }
    k_gather<<<grid, 256, 0, s>>>(h->table, idx_b, counts, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_gather"); break; }
    if (keys_out) {
      e = cudaMemcpyAsync(keys_out, keys_b, D * sizeof(uint64_t), cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(keys)"); break; }
    }
    if (counts_out) {
      e = cudaMemcpyAsync(counts_out, counts, D * sizeof(uint4), cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
    }
  } while (0);
  cudaError_t e = cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}
