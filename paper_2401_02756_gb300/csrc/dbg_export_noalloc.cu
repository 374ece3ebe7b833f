// dbg_export_sorted_noalloc: the sorted export for callers that must not
// allocate device memory.
//
// Who needs it: code that exports graphs from a loop that has to run without
// touching the device allocator -- a serving loop working inside a fixed
// memory budget that another component accounts for, a host framework that
// owns every device allocation itself, or a caller that cannot afford the
// device-wide synchronisation cudaMalloc/cudaFree may cause.  dbg_export_sorted
// takes about 48 bytes per vertex of temporary memory from the stream-ordered
// allocator; this variant takes none.
//
// Its temporary memory is one file-scope device array of
// DBG_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library
// holds until the process exits.  That bounds the graphs it can export to
// DBG_NOALLOC_EXPORT_MAX_VERTICES (2^19) vertices.  Host code cannot use the
// array's name as a device address, so the first call on each device looks
// the address up with cudaGetSymbolAddress (with that device current) and
// keeps it for later calls.  All calls share the array and it keeps the
// previous call's contents; the compaction counter is cleared on every call.
#include <cub/device/device_radix_sort.cuh>

#include <mutex>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr uint64_t kNoallocMaxVertices = DBG_NOALLOC_EXPORT_MAX_VERTICES;
constexpr size_t kNoallocBytes = DBG_NOALLOC_SCRATCH_BYTES;

// layout: keys (8 B/vertex) | slot indices | second slot-index buffer | counter | sort temp
constexpr size_t kKeysOff = 0;
constexpr size_t kIdxOff = kKeysOff + 8 * kNoallocMaxVertices;
constexpr size_t kIdxSortedOff = kIdxOff + 8 * kNoallocMaxVertices;
constexpr size_t kCounterOff = kIdxSortedOff + 8 * kNoallocMaxVertices;
constexpr size_t kTempOff = kCounterOff + 256;
static_assert(kTempOff < kNoallocBytes, "no room for the sort's temporary storage");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// The device address of g_noalloc_scratch on the current device, looked up
// once per device.
int scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return DBG_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return DBG_OK;
}

// Occupied slots -> (key, slot index) in the scratch array, at most `cap` of them.
__global__ void k_compact_noalloc(const Slot *t, uint64_t n_slots, unsigned char *scratch,
                                  uint64_t cap) {
  unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch + kKeysOff);
  unsigned long long *idx = reinterpret_cast<unsigned long long *>(scratch + kIdxOff);
  unsigned long long *count = reinterpret_cast<unsigned long long *>(scratch + kCounterOff);
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (((uint64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (uint64_t base = w0 * 32; base < n_slots; base += warps * 32) {
    const uint64_t i = base + lane;
    const unsigned long long key = i < n_slots ? __ldcs(&t[i].key) : kEmpty;
    const bool occ = key != kEmpty;
    const unsigned mask = __ballot_sync(0xffffffffu, occ);
    unsigned long long pos = 0;
    if (lane == 0 && mask) pos = atomicAdd(count, (unsigned long long)__popc(mask));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const unsigned long long at = pos + __popc(mask & ((1u << lane) - 1u));
    if (occ && at < cap) {
      keys[at] = key;
      idx[at] = i;
    }
  }
}

// Counters of the sorted vertices straight into the caller's buffer.
__global__ void k_gather_noalloc(const Slot *t, const unsigned long long *idx, uint32_t *counts,
                                 uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const Slot &s = t[idx[i]];
    counts[4 * i + 0] = s.cnt[0];
    counts[4 * i + 1] = s.cnt[1];
    counts[4 * i + 2] = s.cnt[2];
    counts[4 * i + 3] = s.cnt[3];
  }
}

}  // namespace
}  // namespace dbg

extern "C" int dbg_export_sorted_noalloc(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                                         uint64_t max_n, uint64_t *n_out, void *stream) {
  using namespace dbg;
  if (!h || !n_out || !keys_out || !counts_out || h->k > 32) return DBG_ERR_INVALID_ARG;
  int prev = 0;
  DBG_CK(cudaGetDevice(&prev));
  if (prev != h->device) DBG_CK(cudaSetDevice(h->device));
  struct Restore {
    int dev, prev;
    ~Restore() {
      if (dev != prev) cudaSetDevice(prev);
    }
  } restore{h->device, prev};
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  unsigned char *scratch = nullptr;
  int st = scratch_address(h->device, &scratch);
  if (st != DBG_OK) return st;

  uint64_t D = 0;
  st = dbg_stats(h, &D, nullptr, stream);  // uses only memory the handle already owns
  if (st != DBG_OK) return st;
  *n_out = D;
  if (D > kNoallocMaxVertices) return DBG_ERR_NOALLOC_LIMIT;
  if (D > max_n) return DBG_ERR_BUFFER_TOO_SMALL;
  if (D == 0) return DBG_OK;

  unsigned long long *keys = reinterpret_cast<unsigned long long *>(scratch + kKeysOff);
  unsigned long long *idx = reinterpret_cast<unsigned long long *>(scratch + kIdxOff);
  unsigned long long *idx_alt = reinterpret_cast<unsigned long long *>(scratch + kIdxSortedOff);
  // ping-pong buffers: the caller's keys_out is the keys' second buffer, so
  // the sort needs only histogram and look-back space in the scratch
  cub::DoubleBuffer<unsigned long long> dk(keys, reinterpret_cast<unsigned long long *>(keys_out));
  cub::DoubleBuffer<unsigned long long> dv(idx, idx_alt);
  const int end_bit = 2 * (h->k - 1);
  size_t temp_bytes = 0;
  DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, dk, dv, (int64_t)D, 0, end_bit, s));
  if (temp_bytes > kNoallocBytes - kTempOff) return DBG_ERR_NOALLOC_LIMIT;

  DBG_CK(cudaMemsetAsync(scratch + kCounterOff, 0, sizeof(unsigned long long), s));
  const int grid = (h->sm_count > 0 ? h->sm_count : 1) * 8;
  k_compact_noalloc<<<grid, 256, 0, s>>>(h->table, h->n_slots, scratch, D);
  DBG_CK(cudaGetLastError());
  DBG_CK(cub::DeviceRadixSort::SortPairs(scratch + kTempOff, temp_bytes, dk, dv, (int64_t)D, 0,
                                         end_bit, s));
  if (dk.Current() != reinterpret_cast<unsigned long long *>(keys_out))
    DBG_CK(cudaMemcpyAsync(keys_out, dk.Current(), D * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
  k_gather_noalloc<<<grid, 256, 0, s>>>(h->table, dv.Current(), counts_out, D);
  DBG_CK(cudaGetLastError());
  DBG_CK(cudaStreamSynchronize(s));
  return DBG_OK;
}
