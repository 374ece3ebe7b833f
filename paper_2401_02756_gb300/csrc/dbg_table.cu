// Handle lifecycle, table kernels (K2 init, stats) and the host-side entry
// points of the C ABI declared in include/dbg.h.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <thread>
#include <new>
#include <vector>

#include "dbg_binned.cuh"
#include "dbg_internal.cuh"

namespace dbg {

static thread_local char g_last_error[512];

int cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_last_error, sizeof(g_last_error), "%s: %s (%s)", what, cudaGetErrorName(e),
           cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DBG_ERR_OOM : DBG_ERR_CUDA;
}

// Temporary device memory of the export and contig passes: a stream-ordered
// pool per device, owned by the library, that keeps up to kScratchKeep
// bytes across synchronisations (the default pool would give every byte
// back at each one, so a loop of exports would map and unmap memory each
// time).  Anything above that is released as usual.  4 GiB covers the
// export of a graph of about 900 million vertices into device buffers (4
// bytes a vertex plus the sort's histograms).
namespace {
constexpr uint64_t kScratchKeep = 4ull << 30;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
}  // namespace

int scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  DBG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return DBG_ERR_INVALID_ARG;
  cudaMemPool_t pool;
  {
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pools[dev]) {
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      DBG_CK(cudaMemPoolCreate(&g_pools[dev], &props));
      uint64_t keep = kScratchKeep;
      DBG_CK(cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep));
    }
    pool = g_pools[dev];
  }
  DBG_CK(cudaMallocFromPoolAsync(p, bytes, pool, s));
  return DBG_OK;
}

uint64_t pool_reserved_bytes(int dev) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (dev < 0 || dev >= 64 || !g_pools[dev]) return 0;
  uint64_t v = 0;
  if (cudaMemPoolGetAttribute(g_pools[dev], cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess)
    return 0;
  return v;
}

int release_scratch_pools() {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  int prev = 0;
  DBG_CK(cudaGetDevice(&prev));
  for (int d = 0; d < 64; ++d) {
    if (!g_pools[d]) continue;
    DBG_CK(cudaSetDevice(d));
    DBG_CK(cudaDeviceSynchronize());
    DBG_CK(cudaMemPoolTrimTo(g_pools[d], 0));
  }
  DBG_CK(cudaSetDevice(prev));
  return DBG_OK;
}

namespace {

struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = err == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

// K2: every slot EMPTY with zero counters; two 16-byte stores per slot.
__global__ void k_table_init(uint4 *t, uint64_t n_vec, const uint32_t *gate) {
  if (gate != nullptr && ld_volatile_u32(gate) != 0u) return;
  const uint4 head = make_uint4(0xffffffffu, 0xffffffffu, 0u, 0u);
  const uint4 tail = make_uint4(0u, 0u, 0u, 0u);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += stride)
    t[i] = (i & 1) ? tail : head;
}

// Vertices (occupied slots) and edges (sum of counters) of a table.
// (wide: keys of k > 32 take two words, so the counters sit at byte 16)
__global__ void k_stats(const Slot *t, uint64_t n_slots, unsigned long long *acc, int wide) {
  unsigned long long nv = 0, ne = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_slots; i += stride) {
    const uint4 *p = reinterpret_cast<const uint4 *>(t + i);
    const uint4 a = __ldcs(p), b = __ldcs(p + 1);
    const unsigned long long key = (unsigned long long)a.x | ((unsigned long long)a.y << 32);
    if (key != kEmpty) {
      nv += 1;
      ne += wide ? (unsigned long long)b.x + b.y + b.z + b.w
                 : (unsigned long long)a.z + a.w + b.x + b.y;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    nv += __shfl_down_sync(0xffffffffu, nv, d);
    ne += __shfl_down_sync(0xffffffffu, ne, d);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(acc, nv);
    atomicAdd(acc + 1, ne);
  }
}

int stream_grid(int sm_count, int per_sm) { return std::max(1, sm_count) * per_sm; }

}  // namespace

int launch_table_init(Slot *table, uint64_t n_slots, cudaStream_t stream, const uint32_t *gate) {
  int dev = 0, sms = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const uint64_t n_vec = n_slots * 2;
  uint64_t want = (n_vec + 255) / 256;
  const int grid = (int)std::min<uint64_t>(want, (uint64_t)stream_grid(sms, 8));
  k_table_init<<<std::max(grid, 1), 256, 0, stream>>>(reinterpret_cast<uint4 *>(table), n_vec,
                                                      gate);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

int launch_stats(const Slot *table, uint64_t n_slots, unsigned long long *acc, cudaStream_t stream,
                 bool wide) {
  int dev = 0, sms = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBG_CK(cudaMemsetAsync(acc, 0, 2 * sizeof(unsigned long long), stream));
  const uint64_t want = (n_slots + 255) / 256;
  const int grid = (int)std::min<uint64_t>(want, (uint64_t)stream_grid(sms, 8));
  k_stats<<<std::max(grid, 1), 256, 0, stream>>>(table, n_slots, acc, wide ? 1 : 0);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

static void timer_free(dbg_handle h) {
  if (h->timer_ev) {
    for (int i = 0; i < h->timer_cap * kTimerMarks; ++i)
      if (h->timer_ev[i]) cudaEventDestroy(h->timer_ev[i]);
  }
  delete[] h->timer_ev;
  delete[] h->timer_mark_set;
  h->timer_ev = nullptr;
  h->timer_mark_set = nullptr;
  h->timer_cap = 0;
  h->timer_calls = 0;
}

int timer_begin_call(dbg_handle h) {
  if (h->timer_cap <= 0) return -1;
  const int call = h->timer_calls % h->timer_cap;
  h->timer_calls += 1;
  for (int m = 0; m < kTimerMarks; ++m) h->timer_mark_set[call * kTimerMarks + m] = 0;
  return call;
}

void timer_mark(dbg_handle h, int call, int m, cudaStream_t s) {
  if (call < 0 || h->timer_cap <= 0) return;
  if (cudaEventRecord(h->timer_ev[call * kTimerMarks + m], s) == cudaSuccess)
    h->timer_mark_set[call * kTimerMarks + m] = 1;
}

void destroy_timer(dbg_handle h) { timer_free(h); }

ItemDesc make_item(dbg_handle h, const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads,
                   uint64_t origin) {
  ItemDesc it{};
  it.packed = packed;
  it.offsets = offsets;
  it.n_reads = n_reads;
  it.origin = origin;
  it.table = h->table;
  it.n_slots = h->n_slots;
  it.status = h->d_status;
  it.max_probes = h->max_probes;
  it.k = h->k;
  it.tile_begin = 0;
  it.vec_ok = ((uintptr_t)packed & 15u) == 0 ? 1 : 0;
  it.spill = h->d_spill;
  it.spill_cap = h->spill_cap;
  it.spill_count = h->d_spill_count;
  return it;
}

}  // namespace dbg

using dbg::DeviceGuard;

// ---------------------------------------------------------------------------
// lifecycle
// ---------------------------------------------------------------------------

namespace {

// The host-staging stream and events of dbg_insert_reads_host, made on first use.
int ensure_copy_stream(dbg_handle h) {
  if (h->copy_stream) return DBG_OK;
  DBG_CK(cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    DBG_CK(cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming));
    DBG_CK(cudaEventCreateWithFlags(&h->ev_consumed[i], cudaEventDisableTiming));
  }
  for (cudaEvent_t &e : h->ev_part) DBG_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return DBG_OK;
}

int check_create_args(int k, uint64_t capacity, dbg_handle *out) {
  if (!out) return DBG_ERR_INVALID_ARG;
  *out = nullptr;
  if (k < 2 || k > 64 || capacity == 0 || capacity > (~0ull / sizeof(dbg::Slot)) - 256)
    return DBG_ERR_INVALID_ARG;
  return DBG_OK;
}

dbg_graph *new_graph(int k, uint64_t capacity, uint32_t max_probes) {
  dbg_graph *h = new (std::nothrow) dbg_graph();
  if (!h) return nullptr;
  h->k = k;
  h->n_slots = capacity;
  h->max_probes = max_probes ? max_probes
                             : (uint32_t)std::min<uint64_t>(capacity, dbg::kDefaultMaxProbes);
  h->max_probes_auto = max_probes == 0;
  return h;
}

int device_of(dbg_handle h) {
  DBG_CK(cudaGetDevice(&h->device));
  DBG_CK(cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device));
  return DBG_OK;
}

void carve_small(dbg_handle h, void *small) {
  h->d_status = static_cast<uint32_t *>(small);
  h->d_acc = reinterpret_cast<unsigned long long *>(static_cast<char *>(small) + dbg::kSmallAcc);
  h->d_spill_count =
      reinterpret_cast<unsigned long long *>(static_cast<char *>(small) + dbg::kSmallSpill);
}

constexpr uint64_t kSmallBytes = 64;   // the small block: status, flag, counters (dbg::kSmall*)
constexpr uint64_t kOnMemTail = 256;   // the same block at the end of caller memory

}  // namespace

extern "C" int dbg_create_ex(int k, uint64_t capacity, uint32_t max_probes, dbg_handle *out) {
  int st = check_create_args(k, capacity, out);
  if (st != DBG_OK) return st;
  dbg_graph *h = new_graph(k, capacity, max_probes);
  if (!h) return DBG_ERR_OOM;
  do {
    st = device_of(h);
    if (st != DBG_OK) break;
    cudaError_t e = cudaMalloc(&h->table, capacity * sizeof(dbg::Slot));
    if (e != cudaSuccess) { h->table = nullptr; st = dbg::cuda_fail(e, "cudaMalloc(table)"); break; }
    void *small = nullptr;
    e = cudaMalloc(&small, kSmallBytes);
    if (e != cudaSuccess) { st = dbg::cuda_fail(e, "cudaMalloc(status)"); break; }
    carve_small(h, small);
    st = ensure_copy_stream(h);
    if (st != DBG_OK) break;
    st = dbg::launch_table_init(h->table, h->n_slots, h->copy_stream);
    if (st != DBG_OK) break;
    e = cudaMemsetAsync(h->d_status, 0, kSmallBytes, h->copy_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->copy_stream);
    if (e != cudaSuccess) { st = dbg::cuda_fail(e, "table init"); break; }
  } while (0);
  if (st != DBG_OK) {
    dbg_destroy(h);
    return st;
  }
  *out = h;
  return DBG_OK;
}

extern "C" int dbg_create(int k, uint64_t capacity, dbg_handle *out) {
  return dbg_create_ex(k, capacity, 0, out);
}

extern "C" uint64_t dbg_table_bytes(uint64_t capacity) {
  if (capacity == 0 || capacity > (~0ull / sizeof(dbg::Slot)) - 256) return 0;
  return capacity * sizeof(dbg::Slot) + kOnMemTail;
}

extern "C" int dbg_create_on(int k, uint64_t capacity, uint32_t max_probes, void *mem,
                             uint64_t mem_bytes, void *stream, dbg_handle *out) {
  int st = check_create_args(k, capacity, out);
  if (st != DBG_OK) return st;
  if (!mem || ((uintptr_t)mem & 255u) || mem_bytes < dbg_table_bytes(capacity))
    return DBG_ERR_INVALID_ARG;
  dbg_graph *h = new_graph(k, capacity, max_probes);
  if (!h) return DBG_ERR_OOM;
  h->owns_slots = h->owns_small = false;
  h->table = static_cast<dbg::Slot *>(mem);
  carve_small(h, static_cast<char *>(mem) + capacity * sizeof(dbg::Slot));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  st = device_of(h);
  if (st == DBG_OK) st = dbg::launch_table_init(h->table, h->n_slots, s);
  if (st == DBG_OK) {
    cudaError_t e = cudaMemsetAsync(h->d_status, 0, kSmallBytes, s);
    if (e != cudaSuccess) st = dbg::cuda_fail(e, "cudaMemsetAsync");
  }
  if (st != DBG_OK) {
    delete h;
    return st;
  }
  *out = h;
  return DBG_OK;
}

extern "C" void dbg_destroy(dbg_handle h) {
  if (!h) return;
  DeviceGuard g(h->device);
  // cudaFree waits for the device anyway; a handle on caller memory that
  // allocated nothing itself frees only host state and does not wait
  const bool owns_device_memory = h->owns_slots || h->owns_small || h->stage_packed[0] ||
                                  h->stage_offsets[0] || h->bin.ev || h->bin.meta || h->d_spill ||
                                  h->bin.ev2 || h->bin.aux;
  if (owns_device_memory) cudaDeviceSynchronize();
  if (h->owns_slots) cudaFree(h->table);
  if (h->owns_small) cudaFree(h->d_status);
  for (int i = 0; i < 2; ++i) {
    cudaFree(h->stage_packed[i]);
    cudaFree(h->stage_offsets[i]);
    if (h->ev_copied[i]) cudaEventDestroy(h->ev_copied[i]);
    if (h->ev_consumed[i]) cudaEventDestroy(h->ev_consumed[i]);
  }
  for (cudaEvent_t e : h->ev_part)
    if (e) cudaEventDestroy(e);
  if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
  dbg::free_bin_scratch(h->bin);
  cudaFree(h->d_spill);
  dbg::destroy_timer(h);
  delete h;
}

extern "C" int dbg_reset(dbg_handle h, void *stream) {
  if (!h) return DBG_ERR_INVALID_ARG;
  h->built_counts = false;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = dbg::launch_table_init(h->table, h->n_slots, s);
  if (st != DBG_OK) return st;
  DBG_CK(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s));
  DBG_CK(cudaMemsetAsync(h->d_spill_count, 0, sizeof(unsigned long long), s));
  return DBG_OK;
}

extern "C" int dbg_set_tuning(dbg_handle h, const dbg_tuning *t) {
  if (!h) return DBG_ERR_INVALID_ARG;
  if (!t) {
    h->tuning = dbg_tuning{};
    return DBG_OK;
  }
  dbg_tuning r = *t;
  if (r.block_threads != 0 && r.block_threads != 128 && r.block_threads != 256 &&
      r.block_threads != 512)
    return DBG_ERR_INVALID_ARG;
  const int bt = r.block_threads ? r.block_threads : 256;
  if (r.tile_reads < 0 || r.tile_reads > bt) return DBG_ERR_INVALID_ARG;
  if (r.grid_ctas < 0) return DBG_ERR_INVALID_ARG;
  if (r.warp_aggregate < -1 || r.warp_aggregate > 1) return DBG_ERR_INVALID_ARG;
  if (r.insert_path < 0 || r.insert_path > 2) return DBG_ERR_INVALID_ARG;
  if (r.apply_unroll != 0 && r.apply_unroll != 2 && r.apply_unroll != 4 && r.apply_unroll != 8)
    return DBG_ERR_INVALID_ARG;
  if (r.apply_chunk != 0 && r.apply_chunk != 4 && r.apply_chunk != 8 && r.apply_chunk != 16)
    return DBG_ERR_INVALID_ARG;
  if (r.apply_ctas < 0 || r.apply_ctas > 32) return DBG_ERR_INVALID_ARG;
  if (r.apply_counters < 0 || r.apply_counters > 64) return DBG_ERR_INVALID_ARG;
  if (r.region_log2 != 0 && (r.region_log2 < 16 || r.region_log2 > 26)) return DBG_ERR_INVALID_ARG;
  if (r.apply_group < 0) return DBG_ERR_INVALID_ARG;
  if (r.apply_mode < 0 || r.apply_mode > 2) return DBG_ERR_INVALID_ARG;
  if (r.scatter_reads != 0 && (r.scatter_reads < 32 || r.scatter_reads > 512))
    return DBG_ERR_INVALID_ARG;
  if (r.split_threads != 0 && r.split_threads != 256 && r.split_threads != 512 &&
      r.split_threads != 1024)
    return DBG_ERR_INVALID_ARG;
  h->tuning = r;
  return DBG_OK;
}

extern "C" int dbg_get_info(dbg_handle h, dbg_info *out) {
  if (!h || !out) return DBG_ERR_INVALID_ARG;
  out->k = h->k;
  out->n_slots = h->n_slots;
  out->table_bytes = h->n_slots * sizeof(dbg::Slot);
  out->max_probes = h->max_probes;
  out->device = h->device;
  out->event_capacity = h->bin.cap ? h->bin.cap : h->bin_want;
  out->spill_capacity = h->spill_cap;
  return DBG_OK;
}

extern "C" int dbg_set_spill(dbg_handle h, uint64_t records) {
  if (!h || (h->k > 32 && records > 0)) return DBG_ERR_INVALID_ARG;  // 64-bit spill records
  h->built_counts = false;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  DBG_CK(cudaDeviceSynchronize());
  unsigned long long pending = 0;
  DBG_CK(cudaMemcpy(&pending, h->d_spill_count, sizeof(pending), cudaMemcpyDeviceToHost));
  if (pending > 0) return DBG_ERR_NEEDS_GROW;  // records would be lost
  cudaFree(h->d_spill);
  h->d_spill = nullptr;
  h->spill_cap = 0;
  if (records == 0) return DBG_OK;
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, records * sizeof(dbg::SpillRecord));
  if (e != cudaSuccess) return dbg::cuda_fail(e, "cudaMalloc(spill)");
  h->d_spill = static_cast<dbg::SpillRecord *>(p);
  h->spill_cap = records;
  return DBG_OK;
}

extern "C" int dbg_grow(dbg_handle h, uint64_t new_capacity, void *stream) {
  if (!h || h->k > 32) return DBG_ERR_INVALID_ARG;
  h->built_counts = false;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  return dbg::launch_grow(h, new_capacity, static_cast<cudaStream_t>(stream));
}

extern "C" int dbg_enable_kernel_timing(dbg_handle h, int calls) {
  if (!h || calls < 0) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  DBG_CK(cudaDeviceSynchronize());
  dbg::destroy_timer(h);
  if (calls == 0) return DBG_OK;
  h->timer_ev = new (std::nothrow) cudaEvent_t[(size_t)calls * dbg::kTimerMarks]();
  h->timer_mark_set = new (std::nothrow) signed char[(size_t)calls * dbg::kTimerMarks]();
  if (!h->timer_ev || !h->timer_mark_set) {
    dbg::destroy_timer(h);
    return DBG_ERR_OOM;
  }
  h->timer_cap = calls;
  for (int i = 0; i < calls * dbg::kTimerMarks; ++i) {
    cudaError_t e = cudaEventCreate(&h->timer_ev[i]);
    if (e != cudaSuccess) {
      dbg::destroy_timer(h);
      return dbg::cuda_fail(e, "cudaEventCreate(timer)");
    }
  }
  return DBG_OK;
}

extern "C" int dbg_kernel_times(dbg_handle h, float *out_ms, int max_calls, int *n_calls) {
  if (!h || !n_calls || max_calls < 0 || (max_calls > 0 && !out_ms)) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  const int kept = std::min(h->timer_calls, h->timer_cap);
  const int first = h->timer_calls - kept;  // oldest kept call
  const int n = std::min(kept, max_calls);
  for (int c = 0; c < n; ++c) {
    const int slot = (first + c) % h->timer_cap;
    const cudaEvent_t *ev = h->timer_ev + (size_t)slot * dbg::kTimerMarks;
    const signed char *set = h->timer_mark_set + (size_t)slot * dbg::kTimerMarks;
    for (int kk = 0; kk < dbg::kTimerKernels; ++kk) {
      float ms = -1.0f;
      // kernel kk spans mark kk to the next recorded mark
      if (set[kk]) {
        int nx = kk + 1;
        while (nx < dbg::kTimerMarks && !set[nx]) ++nx;
        if (nx < dbg::kTimerMarks) {
          DBG_CK(cudaEventSynchronize(ev[nx]));
          DBG_CK(cudaEventElapsedTime(&ms, ev[kk], ev[nx]));
        }
      }
      out_ms[(size_t)c * dbg::kTimerKernels + kk] = ms;
    }
  }
  *n_calls = n;
  return DBG_OK;
}

extern "C" int dbg_binned_counters(dbg_handle h, uint64_t *out) {
  if (!h || !out) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  return dbg::binned_counters(h, out);
}

extern "C" int dbg_reserve_events(dbg_handle h, uint64_t events) {
  if (!h) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  // room for the buckets' margins (3 % and more per region) on top of the
  // positions asked for
  if (events > 0) events += events / 16 + 65536 + 256 * 2048;
  h->bin_want = events;
  // a buffer of another size goes now; the new one comes with the first
  // single-read-set binned insert (batches use the library's own)
  if (h->bin.ev && h->bin.cap != dbg::bin_events_wanted(h)) {
    DBG_CK(cudaDeviceSynchronize());
    dbg::free_bin_scratch(h->bin);
  }
  return DBG_OK;
}

namespace {

// Path for one read set into h: binned when asked for, or automatically for
// large tables; never for k = 32 (keys of 62 bits do not fit an event).
bool want_binned(dbg_handle h) {
  if (h->k > 31) return false;
  const int path = h->tuning.insert_path;
  if (path == 1) return false;
  if (path == 2) return true;
  return h->n_slots * sizeof(dbg::Slot) >= dbg::kBinMinTableBytes;
}

// fresh: the table's contents are discarded first (dbg_build_reads); the
// binned path folds that into its tiled apply, the others empty the table
// with the init kernel before they insert.
// `input`: the read set's bases arrive in parts (see dbg::InputParts); only
// the binned scatter takes them part by part, every other kernel waits for all.
int insert_one(dbg_handle h, const dbg::ItemDesc &it, uint64_t tiles, cudaStream_t s,
               bool fresh = false, const dbg::InputParts *input = nullptr) {
  h->built_counts = false;  // (set again by a rebuild on the tiled binned path)
  const int call = dbg::timer_begin_call(h);
  const bool binned = h->k <= 32 && want_binned(h) &&
                      (h->bin.cap == dbg::bin_events_wanted(h) ||
                       dbg::ensure_bin_scratch(h, 0) == DBG_OK);
  if (binned) return dbg::launch_binned(h, it, tiles, h->tuning, s, call, fresh, input);
  DBG_TRY(dbg::wait_input(input, s));
  if (fresh) DBG_TRY(dbg::launch_table_init(h->table, h->n_slots, s));
  if (h->k > 32) {  // 128-bit keys: their own kernel
    dbg::timer_mark(h, call, 0, s);
    const int st = dbg::launch_insert_wide(it, h->sm_count, s);
    dbg::timer_mark(h, call, 1, s);
    return st;
  }
  dbg::timer_mark(h, call, 0, s);
  const int st = dbg::launch_insert(&it, 1, tiles, h->tuning, h->sm_count, s);
  dbg::timer_mark(h, call, 1, s);  // direct call: kernel 0 spans marks 0..1
  return st;
}

}  // namespace

// ---------------------------------------------------------------------------
// inserts
// ---------------------------------------------------------------------------

extern "C" int dbg_insert_reads(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                                uint64_t n_reads, void *stream) {
  if (!h) return DBG_ERR_INVALID_ARG;
  if (n_reads == 0) return DBG_OK;
  if (!packed || !offsets) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  const dbg_tuning t = dbg::resolve_tuning(h->tuning);
  const uint64_t tiles = (n_reads + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
  const dbg::ItemDesc it = dbg::make_item(h, packed, offsets, n_reads, 0);
  return insert_one(h, it, tiles, static_cast<cudaStream_t>(stream));
}

namespace {

// The sticky status and the spill count back to zero, stream-ordered (the
// part of dbg_reset that is not the table).
// (the start of every rebuild: its counts, if any, are set by its insert)
int clear_status(dbg_handle h, cudaStream_t s) {
  h->built_counts = false;
  DBG_CK(cudaMemsetAsync(h->d_status, 0, sizeof(uint32_t), s));
  DBG_CK(cudaMemsetAsync(h->d_spill_count, 0, sizeof(unsigned long long), s));
  return DBG_OK;
}

}  // namespace

extern "C" int dbg_build_reads(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                               uint64_t n_reads, void *stream) {
  if (!h) return DBG_ERR_INVALID_ARG;
  if (n_reads > 0 && (!packed || !offsets)) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBG_TRY(clear_status(h, s));
  if (n_reads == 0) return dbg::launch_table_init(h->table, h->n_slots, s);
  const dbg_tuning t = dbg::resolve_tuning(h->tuning);
  const uint64_t tiles = (n_reads + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
  const dbg::ItemDesc it = dbg::make_item(h, packed, offsets, n_reads, 0);
  return insert_one(h, it, tiles, s, /*fresh=*/true);
}

namespace {

constexpr uint64_t kStageAllBytes = 4ull << 30;  // inputs up to this size are staged whole
constexpr uint64_t kStageBytes = 256ull << 20;   // otherwise: packed bytes per host chunk
constexpr uint64_t kStageReads = 1ull << 22;     // otherwise: reads per host chunk
constexpr int kInputParts = 8;                    // a whole input is copied in at most 8 parts
constexpr uint64_t kPartBytes = 128ull << 20;     // of at least this many packed bytes

int grow_stage(dbg_handle h, uint64_t bytes, uint64_t reads) {
  const int st = ensure_copy_stream(h);
  if (st != DBG_OK) return st;
  if (bytes > h->stage_packed_bytes) {
    DBG_CK(cudaStreamSynchronize(h->copy_stream));
    DBG_CK(cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i) {
      cudaFree(h->stage_packed[i]);
      h->stage_packed[i] = nullptr;
    }
    h->stage_packed_bytes = 0;
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaMalloc(&h->stage_packed[i], bytes);
      if (e != cudaSuccess) return dbg::cuda_fail(e, "cudaMalloc(staging)");
    }
    h->stage_packed_bytes = bytes;
  }
  if (reads + 1 > h->stage_offsets_count) {
    DBG_CK(cudaDeviceSynchronize());
    for (int i = 0; i < 2; ++i) {
      cudaFree(h->stage_offsets[i]);
      h->stage_offsets[i] = nullptr;
    }
    h->stage_offsets_count = 0;
    for (int i = 0; i < 2; ++i) {
      cudaError_t e = cudaMalloc(&h->stage_offsets[i], (reads + 1) * sizeof(uint64_t));
      if (e != cudaSuccess) return dbg::cuda_fail(e, "cudaMalloc(staging)");
    }
    h->stage_offsets_count = reads + 1;
  }
  return DBG_OK;
}

}  // namespace

// offsets[0..n_reads] never decrease.  Branch-free (vectorisable) scans,
// split over up to 16 host threads for inputs of millions of reads.
static bool offsets_non_decreasing(const uint64_t *offsets, uint64_t n_reads) {
  auto scan = [offsets](uint64_t r0, uint64_t r1) {
    uint64_t bad = 0;
    for (uint64_t r = r0; r < r1; ++r) bad |= (uint64_t)(offsets[r + 1] < offsets[r]);
    return bad == 0;
  };
  constexpr uint64_t kReadsPerThread = 1ull << 20;
  const uint64_t hw = std::max(1u, std::thread::hardware_concurrency());
  const uint64_t nt = std::min<uint64_t>(std::min<uint64_t>(hw, 16),
                                         (n_reads + kReadsPerThread - 1) / kReadsPerThread);
  if (nt <= 1) return scan(0, n_reads);
  std::vector<char> ok(nt, 0);
  std::vector<std::thread> pool;
  pool.reserve(nt - 1);
  for (uint64_t i = 1; i < nt; ++i)
    pool.emplace_back([&, i] { ok[i] = scan(n_reads * i / nt, n_reads * (i + 1) / nt); });
  ok[0] = scan(0, n_reads / nt);
  for (std::thread &t : pool) t.join();
  return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
}

// The whole input staged at once (one insert: the binned path needs to see
// the whole read set).  The offsets are copied first, then the packed bases
// in parts of at least kPartBytes, each recorded by an event, so that the
// binned scatter starts on a part as soon as it has arrived.  The host checks
// the offsets while the copies run; no kernel is launched before the check
// passes (a refused call waits for its copies, so that the caller may reuse
// its buffers).
static int insert_whole(dbg_handle h, const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads,
                        uint64_t all_bytes, const dbg_tuning &t, cudaStream_t s, bool fresh) {
  DBG_TRY(grow_stage(h, std::max<uint64_t>(16, (all_bytes + 15) & ~15ull), n_reads));
  const uint64_t byte0 = offsets[0] >> 2, end = (offsets[n_reads] + 3) >> 2;
  DBG_CK(cudaStreamWaitEvent(h->copy_stream, h->ev_consumed[0], 0));
  DBG_CK(cudaMemcpyAsync(h->stage_offsets[0], offsets, (n_reads + 1) * sizeof(uint64_t),
                         cudaMemcpyHostToDevice, h->copy_stream));
  DBG_CK(cudaEventRecord(h->ev_copied[0], h->copy_stream));
  // parts: the reads cut where the bytes pass equal shares
  const int n_parts =
      (int)std::min<uint64_t>(kInputParts, std::max<uint64_t>(1, all_bytes / kPartBytes));
  uint64_t read_cut[kInputParts + 1];
  read_cut[0] = 0;
  read_cut[n_parts] = n_reads;
  for (int c = 1; c < n_parts; ++c) {
    const uint64_t target = byte0 + all_bytes * (uint64_t)c / (uint64_t)n_parts;
    uint64_t lo = read_cut[c - 1], hi = n_reads;  // the first read starting at or past it
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if ((offsets[mid] >> 2) < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    read_cut[c] = lo;
  }
  uint64_t copied = byte0;  // bytes [byte0, copied) are on their way
  for (int c = 0; c < n_parts; ++c) {
    const uint64_t upto =
        c + 1 == n_parts
            ? end
            : std::max(copied, std::min(end, (offsets[read_cut[c + 1]] + 3) >> 2));
    if (upto > copied)
      DBG_CK(cudaMemcpyAsync(h->stage_packed[0] + (copied - byte0), packed + copied, upto - copied,
                             cudaMemcpyHostToDevice, h->copy_stream));
    copied = upto;
    DBG_CK(cudaEventRecord(h->ev_part[c], h->copy_stream));
  }
  if (!offsets_non_decreasing(offsets, n_reads)) {
    DBG_CK(cudaStreamSynchronize(h->copy_stream));
    return DBG_ERR_INVALID_ARG;
  }
  if (fresh) DBG_TRY(clear_status(h, s));
  DBG_CK(cudaStreamWaitEvent(s, h->ev_copied[0], 0));
  const dbg::ItemDesc it =
      dbg::make_item(h, h->stage_packed[0], h->stage_offsets[0], n_reads, byte0 * 4);
  const uint64_t tiles = (n_reads + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
  dbg::InputParts input;
  input.n = n_parts;
  input.read_cut = read_cut;
  input.ready = h->ev_part;
  if (n_parts == 1) DBG_CK(cudaStreamWaitEvent(s, h->ev_part[0], 0));
  DBG_TRY(insert_one(h, it, tiles, s, fresh, n_parts > 1 ? &input : nullptr));
  DBG_CK(cudaEventRecord(h->ev_consumed[0], s));
  return DBG_OK;
}

// dbg_insert_reads_host, or with `fresh` dbg_build_reads_host: the first
// chunk's insert then discards the table's contents (later chunks add to it).
static int insert_reads_host(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                             uint64_t n_reads, void *stream, bool fresh) {
  if (!h) return DBG_ERR_INVALID_ARG;
  if (n_reads > 0 && (!packed || !offsets)) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_reads == 0) {
    if (!fresh) return DBG_OK;
    DBG_TRY(clear_status(h, s));
    return dbg::launch_table_init(h->table, h->n_slots, s);
  }
  const dbg_tuning t = dbg::resolve_tuning(h->tuning);

  // the whole input when it is small enough (one insert, which the binned
  // path needs to see the whole read set at once), else chunks of at most
  // kStageReads reads and about kStageBytes bytes
  if (offsets[n_reads] >= offsets[0]) {
    const uint64_t all_bytes = ((offsets[n_reads] + 3) >> 2) - (offsets[0] >> 2);
    if (all_bytes + (n_reads + 1) * sizeof(uint64_t) <= kStageAllBytes)
      return insert_whole(h, packed, offsets, n_reads, all_bytes, t, s, fresh);
  }
  if (!offsets_non_decreasing(offsets, n_reads)) return DBG_ERR_INVALID_ARG;
  if (fresh) DBG_TRY(clear_status(h, s));
  std::vector<uint64_t> cuts{0};
  uint64_t max_bytes = 0, max_reads = 0;
  for (uint64_t r0 = 0; cuts.back() != n_reads && r0 < n_reads;) {
    const uint64_t b0 = offsets[r0] >> 2;
    uint64_t r1 = std::min(n_reads, r0 + kStageReads);
    // shrink until the chunk's bytes fit (always keep at least one read)
    uint64_t lo = r0 + 1, hi = r1;
    while (lo < hi) {
      const uint64_t mid = (lo + hi + 1) / 2;
      if (((offsets[mid] + 3) >> 2) - b0 <= kStageBytes)
        lo = mid;
      else
        hi = mid - 1;
    }
    r1 = lo;
    max_bytes = std::max(max_bytes, ((offsets[r1] + 3) >> 2) - b0);
    max_reads = std::max(max_reads, r1 - r0);
    cuts.push_back(r1);
    r0 = r1;
  }
  int st = grow_stage(h, std::max<uint64_t>(16, (max_bytes + 15) & ~15ull), max_reads);
  if (st != DBG_OK) return st;

  for (size_t c = 0; c + 1 < cuts.size(); ++c) {
    const int b = (int)(c & 1);
    const uint64_t r0 = cuts[c], r1 = cuts[c + 1];
    const uint64_t byte0 = offsets[r0] >> 2;
    const uint64_t nbytes = ((offsets[r1] + 3) >> 2) - byte0;
    DBG_CK(cudaStreamWaitEvent(h->copy_stream, h->ev_consumed[b], 0));
    DBG_CK(cudaMemcpyAsync(h->stage_offsets[b], offsets + r0, (r1 - r0 + 1) * sizeof(uint64_t),
                           cudaMemcpyHostToDevice, h->copy_stream));
    if (nbytes)
      DBG_CK(cudaMemcpyAsync(h->stage_packed[b], packed + byte0, nbytes, cudaMemcpyHostToDevice,
                             h->copy_stream));
    DBG_CK(cudaEventRecord(h->ev_copied[b], h->copy_stream));
    DBG_CK(cudaStreamWaitEvent(s, h->ev_copied[b], 0));
    const dbg::ItemDesc it =
        dbg::make_item(h, h->stage_packed[b], h->stage_offsets[b], r1 - r0, byte0 * 4);
    const uint64_t tiles = (r1 - r0 + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
    st = insert_one(h, it, tiles, s, fresh && c == 0);
    if (st != DBG_OK) return st;
    DBG_CK(cudaEventRecord(h->ev_consumed[b], s));
  }
  return DBG_OK;
}

extern "C" int dbg_insert_reads_host(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                                     uint64_t n_reads, void *stream) {
  return insert_reads_host(h, packed, offsets, n_reads, stream, false);
}

extern "C" int dbg_build_reads_host(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                                    uint64_t n_reads, void *stream) {
  return insert_reads_host(h, packed, offsets, n_reads, stream, true);
}

// Many read sets into many graphs: graphs with k <= 31 go through binned
// chains (all of a chain's tables in one launch of each binned kernel) unless
// their tuning asks for the direct path; those and the graphs with k = 32
// share direct insert launches of up to kBatchItems items, and graphs with
// k > 32 take their own kernel one by one.  `fresh`: every graph is emptied
// first (dbg_build_batch).  (On the 256-sample batched workload every table
// in the chains built 1.5x faster than the default single-table choice --
// binned from 256 MiB up, the small tables direct.)
static int insert_batch(const dbg_batch_item *items, int n_items, void *stream, bool fresh) {
  if (n_items < 0 || (n_items > 0 && !items)) return DBG_ERR_INVALID_ARG;
  if (n_items == 0) return DBG_OK;
  const int dev = items[0].graph ? items[0].graph->device : -1;
  for (int i = 0; i < n_items; ++i) {
    if (!items[i].graph || items[i].graph->device != dev) return DBG_ERR_INVALID_ARG;
    if (items[i].n_reads > 0 && (!items[i].packed || !items[i].offsets)) return DBG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < n_items; ++i) items[i].graph->built_counts = false;  // (dbg_stats counts)
  DeviceGuard g(dev);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const dbg_tuning t = dbg::resolve_tuning(items[0].graph->tuning);
  const int sms = items[0].graph->sm_count;
  std::vector<dbg::ItemDesc> group, binned;
  std::vector<uint64_t> wants;
  group.reserve(dbg::kBatchItems);
  uint64_t tiles = 0;
  for (int i = 0; i <= n_items; ++i) {
    const bool flush = (i == n_items) || (int)group.size() == dbg::kBatchItems;
    if (flush && !group.empty()) {
      if (fresh) DBG_TRY(dbg::launch_tables_init(group.data(), (int)group.size(), sms, s));
      DBG_TRY(dbg::launch_insert(group.data(), (int)group.size(), tiles, t, sms, s));
      group.clear();
      tiles = 0;
    }
    if (i == n_items) break;
    dbg_handle h = items[i].graph;
    dbg::ItemDesc it = dbg::make_item(h, items[i].packed, items[i].offsets, items[i].n_reads, 0);
    if (h->k > 32) {  // 128-bit keys: their own kernel, one item at a time
      if (fresh) {
        DBG_TRY(clear_status(h, s));
        DBG_TRY(dbg::launch_table_init(h->table, h->n_slots, s));
      }
      if (items[i].n_reads == 0) continue;
      const dbg_tuning th = dbg::resolve_tuning(h->tuning);
      DBG_TRY(insert_one(h, it, (items[i].n_reads + th.tile_reads - 1) / th.tile_reads, s));
      continue;
    }
    if (h->k <= 31 && h->tuning.insert_path != 1) {  // binned chains below (an empty read
                                                     // set still empties a build)
      binned.push_back(it);
      wants.push_back(dbg::bin_events_wanted(h));
      continue;
    }
    if (items[i].n_reads == 0 && !fresh) continue;
    it.tile_begin = tiles;
    tiles += (items[i].n_reads + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
    group.push_back(it);
  }
  return dbg::launch_binned_batch(binned.data(), wants.data(), (int)binned.size(), t, sms, s,
                                  fresh);
}

extern "C" int dbg_insert_batch(const dbg_batch_item *items, int n_items, void *stream) {
  return insert_batch(items, n_items, stream, false);
}

extern "C" int dbg_build_batch(const dbg_batch_item *items, int n_items, void *stream) {
  return insert_batch(items, n_items, stream, true);
}

extern "C" uint64_t dbg_scratch_bytes(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  return dbg::batch_scratch_bytes(dev) + dbg::pool_reserved_bytes(dev);
}

extern "C" int dbg_release_scratch(void) {
  int st = dbg::release_batch_scratch();
  if (st != DBG_OK) return st;
  return dbg::release_scratch_pools();
}

// ---------------------------------------------------------------------------
// status and stats
// ---------------------------------------------------------------------------

extern "C" int dbg_get_status(dbg_handle h, void *stream) {
  if (!h) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t st = 0;
  unsigned long long spilled = 0;
  DBG_CK(cudaMemcpyAsync(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaMemcpyAsync(&spilled, h->d_spill_count, sizeof(spilled), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaStreamSynchronize(s));
  if (st == DBG_OK && spilled > 0) return DBG_ERR_NEEDS_GROW;
  return (int)st;
}

extern "C" int dbg_stats(dbg_handle h, uint64_t *n_vertices, uint64_t *n_edges, void *stream) {
  if (!h) return DBG_ERR_INVALID_ARG;
  DeviceGuard g(h->device);
  if (g.err != cudaSuccess) return dbg::cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (h->built_counts) {
    // the graph was last rebuilt on the tiled binned path, which counted its
    // new vertices and its edges: read them unless the build fell back
    uint32_t head[2] = {0, 0};  // status, counted flag
    unsigned long long built[2] = {0, 0}, spilled = 0;
    DBG_CK(cudaMemcpyAsync(head, h->d_status, sizeof(head), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaMemcpyAsync(built, dbg::small_built(h->d_status), sizeof(built),
                           cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaMemcpyAsync(&spilled, h->d_spill_count, sizeof(spilled), cudaMemcpyDeviceToHost, s));
    DBG_CK(cudaStreamSynchronize(s));
    if (head[1] == 1u && head[0] == DBG_OK && spilled == 0) {
      if (n_vertices) *n_vertices = built[0];
      if (n_edges) *n_edges = built[1];
      return DBG_OK;
    }
  }
  int st = dbg::launch_stats(h->table, h->n_slots, h->d_acc, s, h->k > 32);
  if (st != DBG_OK) return st;
  unsigned long long acc[2] = {0, 0};
  uint32_t status = 0;
  unsigned long long spilled = 0;
  DBG_CK(cudaMemcpyAsync(acc, h->d_acc, sizeof(acc), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaMemcpyAsync(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaMemcpyAsync(&spilled, h->d_spill_count, sizeof(spilled), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaStreamSynchronize(s));
  if (n_vertices) *n_vertices = acc[0];
  if (n_edges) *n_edges = acc[1];
  if (status == DBG_OK && spilled > 0) return DBG_ERR_NEEDS_GROW;
  return (int)status;
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------

extern "C" int dbg_pack_ascii(const char *ascii, uint64_t n, uint8_t *out, int phase,
                              uint64_t *bad_index) {
  if ((n > 0 && (!ascii || !out)) || phase < 0 || phase > 3) return DBG_ERR_INVALID_ARG;
  for (uint64_t i = 0; i < n; ++i) {
    unsigned code;
    switch (ascii[i]) {
      case 'A': code = 0; break;
      case 'C': code = 1; break;
      case 'G': code = 2; break;
      case 'T': code = 3; break;
      default:
        if (bad_index) *bad_index = i;
        return DBG_ERR_INVALID_ARG;
    }
    const uint64_t p = i + (uint64_t)phase;
    const unsigned sh = 2u * (unsigned)(p & 3u);
    uint8_t &byte = out[p >> 2];
    byte = (uint8_t)((byte & ~(3u << sh)) | (code << sh));
  }
  return DBG_OK;
}

extern "C" const char *dbg_strerror(int code) {
  switch (code) {
    case DBG_OK: return "ok";
    case DBG_ERR_INVALID_ARG: return "invalid argument";
    case DBG_ERR_OOM: return "out of memory";
    case DBG_ERR_CAPACITY: return "table full: a vertex found no free slot within max_probes";
    case DBG_ERR_CUDA: return "CUDA error";
    case DBG_ERR_BUFFER_TOO_SMALL: return "output buffer too small";
    case DBG_ERR_BAD_OFFSETS: return "offsets are not non-decreasing";
    case DBG_ERR_NOALLOC_LIMIT: return "graph larger than the no-alloc export's fixed scratch";
    case DBG_ERR_NEEDS_GROW: return "vertices were spilled: call dbg_grow to complete the graph";
    case DBG_ERR_TIMEOUT: return "a kernel gave up a bounded wait on an asynchronous copy";
    default: return "unknown status";
  }
}

extern "C" const char *dbg_last_cuda_error(void) { return dbg::g_last_error; }

extern "C" int dbg_binary_version(int *out) {
  if (!out) return DBG_ERR_INVALID_ARG;
  *out = 0;
  cudaFuncAttributes a{};
  DBG_CK(cudaFuncGetAttributes(&a, dbg::k_table_init));
  *out = a.binaryVersion;
  return DBG_OK;
}
