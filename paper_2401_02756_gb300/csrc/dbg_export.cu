// Sorted export of a graph (K3 compaction, K4 radix sort, gather): the
// (vertex, counters) table of the paper's Fig. 1 in key order, which is
// lexicographic order with A < C < G < T because keys hold the first base in
// their most significant bits.  Not on the timed insert path.
//
// The radix sort is CUB's DeviceRadixSort (open-source CCCL headers shipped
// with the CUDA toolkit); compaction and gather are this file's kernels.
//
// Memory.  The sort orders (key, slot index) pairs -- 8 + 4 bytes a vertex
// while the table has fewer than 2^32 slots -- and needs a second buffer of
// each.  When both outputs are device buffers they hold all four: keys_out
// is the first key buffer, and counts_out (16 bytes a vertex) holds the
// second key buffer and both index buffers until the gather overwrites it.
// The only temporary memory is then one index array (4 bytes a vertex: the
// gather cannot read its indices from the buffer it writes) and the sort's
// small histogram space.  Host outputs go through temporary device buffers.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr int kCompactBlock = 256;
constexpr int kCompactPer = 8;  // slots per thread per round: 2048 per CTA round

// K3: (key, slot index) of every occupied slot, at most `cap` of them (the
// vertices counted beforehand; nothing is ever written past the buffers).
// Each CTA round takes 2048 consecutive slots; every warp ranks its occupied
// slots with ballots, the warps' totals are summed in shared memory, and one
// atomicAdd per round places the CTA's run -- so a warp's writes of one
// ballot are 32 consecutive entries.  The order of the runs does not matter:
// the sort follows.
template <class I>
__global__ void __launch_bounds__(kCompactBlock)
    k_compact(const Slot *t, uint64_t n_slots, unsigned long long *keys, I *idx,
              unsigned long long *count, uint64_t cap) {
  constexpr int W = kCompactBlock / 32;
  __shared__ uint32_t s_w[W];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  constexpr uint64_t kRound = (uint64_t)kCompactBlock * kCompactPer;
  for (uint64_t base = (uint64_t)blockIdx.x * kRound; base < n_slots;
       base += (uint64_t)gridDim.x * kRound) {
    unsigned long long k[kCompactPer];
    unsigned bal[kCompactPer];
    uint32_t wcount = 0;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      const uint64_t i = base + (uint64_t)r * kCompactBlock + threadIdx.x;
      k[r] = i < n_slots ? __ldcs(&t[i].key) : kEmpty;
      bal[r] = __ballot_sync(0xffffffffu, k[r] != kEmpty);
      wcount += (uint32_t)__popc(bal[r]);
    }
    if (lane == 0) s_w[warp] = wcount;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const uint32_t v = s_w[j];
      before += j < warp ? v : 0u;
      total += v;
    }
    if (threadIdx.x == 0) s_base = total ? atomicAdd(count, (unsigned long long)total) : 0ull;
    __syncthreads();
    uint64_t pos = s_base + before;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      if (k[r] != kEmpty) {
        const uint64_t at = pos + (uint64_t)__popc(bal[r] & lt);
        if (at < cap) {
          keys[at] = k[r];
          idx[at] = (I)(base + (uint64_t)r * kCompactBlock + threadIdx.x);
        }
      }
      pos += (uint64_t)__popc(bal[r]);
    }
    __syncthreads();  // s_w and s_base are rewritten by the next round
  }
}

// Counters of the sorted vertices, in key order.
template <class I>
__global__ void k_gather(const Slot *t, const I *__restrict__ idx, uint4 *counts, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    // the counters sit at byte 8 of the slot: 8-byte aligned, not 16
    const uint2 *c = reinterpret_cast<const uint2 *>(&t[__ldcs(idx + i)].cnt[0]);
    const uint2 lo = c[0], hi = c[1];
    __stcs(counts + i, make_uint4(lo.x, lo.y, hi.x, hi.y));
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

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // (an unregistered host pointer on older runtimes)
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The export of D vertices with slot indices of type I (k <= 32).
template <class I>
int export_pairs(dbg_handle h, uint64_t D, uint64_t *keys_out, uint32_t *counts_out,
                 cudaStream_t s) {
  const int end_bit = 2 * (h->k - 1);
  // in place: both outputs on the device, 16-byte aligned (keys_out needs 8,
  // the uint4 rows of counts_out 16), and the index buffers fit beside the
  // second key buffer in counts_out
  const bool in_place = sizeof(I) == 4 && is_device_ptr(keys_out) && is_device_ptr(counts_out) &&
                        ((uintptr_t)keys_out & 15u) == 0 && ((uintptr_t)counts_out & 15u) == 0;
  size_t temp_bytes = 0;
  {
    cub::DoubleBuffer<unsigned long long> dk(nullptr, nullptr);
    cub::DoubleBuffer<I> dv(nullptr, nullptr);
    DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, dk, dv, (int64_t)D, 0, end_bit, s));
  }
  const size_t kb = align256(D * sizeof(unsigned long long));
  const size_t ib = align256(D * sizeof(I));
  const size_t cb = align256(D * sizeof(uint4));
  // scratch: [count][sort temp], then in place [final indices], otherwise
  // [keys a][keys b][indices a][indices b][counters]
  const size_t head = 256 + align256(temp_bytes);
  const size_t total = head + (in_place ? ib : 2 * kb + 2 * ib + cb);
  char *buf = nullptr;
  DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), total, s));
  unsigned long long *count = reinterpret_cast<unsigned long long *>(buf);
  void *temp = buf + 256;
  I *idx_final = reinterpret_cast<I *>(buf + head);  // (in place only)
  unsigned long long *keys_a, *keys_b;
  I *idx_a, *idx_b;
  uint4 *counts;
  if (in_place) {
    char *c = reinterpret_cast<char *>(counts_out);
    keys_a = reinterpret_cast<unsigned long long *>(keys_out);
    keys_b = reinterpret_cast<unsigned long long *>(c);
    idx_a = reinterpret_cast<I *>(c + D * 8);
    idx_b = reinterpret_cast<I *>(c + D * 12);
    counts = reinterpret_cast<uint4 *>(counts_out);
  } else {
    char *p = buf + head;
    keys_a = reinterpret_cast<unsigned long long *>(p);
    keys_b = reinterpret_cast<unsigned long long *>(p + kb);
    idx_a = reinterpret_cast<I *>(p + 2 * kb);
    idx_b = reinterpret_cast<I *>(p + 2 * kb + ib);
    counts = reinterpret_cast<uint4 *>(p + 2 * kb + 2 * ib);
  }

  int rc = DBG_OK;
  do {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    const int sms = std::max(1, h->sm_count);
    k_compact<I><<<sms * 8, kCompactBlock, 0, s>>>(h->table, h->n_slots, keys_a, idx_a, count, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_compact"); break; }
    cub::DoubleBuffer<unsigned long long> dk(keys_a, keys_b);
    cub::DoubleBuffer<I> dv(idx_a, idx_b);
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, dk, dv, (int64_t)D, 0, end_bit, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceRadixSort::SortPairs"); break; }
    // in place, the gather writes counts_out, which holds the sorted indices
    // (and maybe the sorted keys): move them out first
    const I *gidx = dv.Current();
    if (in_place) {
      e = cudaMemcpyAsync(idx_final, dv.Current(), D * sizeof(I), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(indices)"); break; }
      gidx = idx_final;
    }
    if (keys_out && (!in_place || dk.Current() != keys_a)) {
      e = cudaMemcpyAsync(keys_out, dk.Current(), D * sizeof(uint64_t), cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(keys)"); break; }
    }
    if (counts_out) {
      k_gather<I><<<sms * 8, 256, 0, s>>>(h->table, gidx, counts, D);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_gather"); break; }
      if (!in_place) {
        e = cudaMemcpyAsync(counts_out, counts, D * sizeof(uint4), cudaMemcpyDefault, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
      }
    }
  } while (0);
  cudaError_t e = cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}

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
  if (h->n_slots <= 0xFFFFFFFFull) return export_pairs<uint32_t>(h, D, keys_out, counts_out, s);
  return export_pairs<unsigned long long>(h, D, keys_out, counts_out, s);
}
