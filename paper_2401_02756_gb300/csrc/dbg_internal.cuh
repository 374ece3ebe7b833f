// Internal definitions of libdbg: the device table layout, the item
// descriptor the insert kernel consumes, and the handle.
//
// Table (replaces the paper's array of N atomic list heads with chained
// Nodes, Section "Graph data structure", Fig. 2): an open-addressing array of
// 32-byte slots, one slot per 32-byte DRAM sector, so that a vertex touch --
// claim, find and count -- is one sector.  A slot holds the vertex key (the
// paper's stored (k-1)-mer, here 2 bits per base) and the four out-edge
// counters; the paper's four edge pointers are not stored, because the
// target of label b from key v is ((v << 2) | b) masked to 2(k-1) bits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dbg.h"

namespace dbg {

constexpr unsigned long long kEmpty = ~0ull;  // never a key: keys have <= 62 bits
constexpr uint32_t kDefaultMaxProbes = 8192;

struct __align__(32) Slot {
  unsigned long long key;  // kEmpty or the vertex key
  uint32_t cnt[4];         // out-edge counters, labels A, C, G, T
  uint32_t pad[2];         // zero; keeps one slot per 32-byte sector
};
static_assert(sizeof(Slot) == 32, "slot must be one 32-byte sector");

// A vertex position that found no slot within max_probes, kept for dbg_grow.
struct SpillRecord {
  unsigned long long key;
  unsigned long long info;  // bit 2: the position starts a k-mer; bits 0-1: its label
};

// Keep a vertex that found no slot, or fail with DBG_ERR_CAPACITY when there
// is no spill buffer or it is full.  Returns true when the insert must stop.
__device__ __forceinline__ bool spill_or_fail(SpillRecord *spill, uint64_t spill_cap,
                                              unsigned long long *spill_count, uint32_t *status,
                                              uint64_t key, bool edge, uint32_t label) {
  if (spill != nullptr) {
    const unsigned long long at = atomicAdd(spill_count, 1ull);
    if (at < spill_cap) {
      spill[at].key = key;
      spill[at].info = ((unsigned long long)edge << 2) | label;
      return false;
    }
  }
  atomicCAS(status, 0u, (uint32_t)DBG_ERR_CAPACITY);
  return true;
}

// One read set to insert into one table (a batch is an array of these).
struct ItemDesc {
  const uint8_t *packed;     // 2-bit stream, byte 0 holds base `origin`
  const uint64_t *offsets;   // n_reads + 1 base positions
  uint64_t n_reads;
  uint64_t origin;           // base position of packed[0] (multiple of 4)
  Slot *table;
  uint64_t n_slots;
  uint32_t *status;          // sticky device status word
  uint32_t max_probes;
  int k;
  uint64_t tile_begin;       // first global tile index of this item
  int vec_ok;                // packed is 16-byte aligned: vector loads allowed
  int region0;               // binned insert: the item's first region in its chain
  SpillRecord *spill;        // vertices that found no slot go here (null: fail instead)
  uint64_t spill_cap;
  unsigned long long *spill_count;
};

// MurmurHash3's 64-bit finalizer (Appleby, public domain): a bijective mix
// so that nearby keys land on unrelated slots.
__host__ __device__ __forceinline__ uint64_t fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdull;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ull;
  x ^= x >> 33;
  return x;
}

// The table's key hash: a multiplication by 2^64 / golden ratio (Knuth's
// multiplicative hashing) whose high bits choose the home slot, with the high
// half folded into the low one so that the low byte is mixed too (the tiled
// apply's slot fingerprints).
__host__ __device__ __forceinline__ uint64_t key_hash(uint64_t key) {
  const uint64_t x = key * 0x9E3779B97F4A7C15ull;
  return x ^ (x >> 32);
}

__device__ __forceinline__ uint64_t home_slot(uint64_t key, uint64_t n_slots) {
  return __umul64hi(key_hash(key), n_slots);
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// An L2 cache policy that keeps the lines it touches ahead of others
// (evict_last) for the whole access.
__device__ __forceinline__ uint64_t l2_policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

__device__ __forceinline__ unsigned long long ld_relaxed_u64_hint(const unsigned long long *p,
                                                                   uint64_t pol) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.L2::cache_hint.u64 %0, [%1], %2;"
               : "=l"(v)
               : "l"(p), "l"(pol)
               : "memory");
  return v;
}

__device__ __forceinline__ void red_add_u32_hint(uint32_t *p, uint32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.u32 [%0], %1, %2;" ::"l"(p), "r"(v),
               "l"(pol)
               : "memory");
}

__device__ __forceinline__ unsigned long long cas_u64_hint(unsigned long long *p,
                                                           unsigned long long cmp,
                                                           unsigned long long val, uint64_t pol) {
  unsigned long long old;
  asm volatile("atom.relaxed.gpu.global.cas.L2::cache_hint.b64 %0, [%1], %2, %3, %4;"
               : "=l"(old)
               : "l"(p), "l"(cmp), "l"(val), "l"(pol)
               : "memory");
  return old;
}

__device__ __forceinline__ uint32_t ld_volatile_u32(const uint32_t *p) {
  return *(const volatile uint32_t *)p;
}

__device__ __forceinline__ void set_sticky(uint32_t *status, uint32_t code) {
  atomicCAS(status, 0u, code);
}

// Reverse the order of the 32 two-bit groups of a 64-bit word.
__device__ __forceinline__ uint64_t reverse_pairs(uint64_t x) {
  x = __brevll(x);
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// Key of the m bases starting at base q of a little-endian 2-bit stream whose
// 64-bit words (32 bases each) are w[]: first base most significant.
__device__ __forceinline__ uint64_t key_from_words(uint64_t lo, uint64_t hi, uint32_t sh, int m) {
  uint64_t x = sh ? ((lo >> sh) | (hi << (64u - sh))) : lo;
  return reverse_pairs(x) >> (64 - 2 * m);
}

// Find the slot holding `key`, claiming an empty one if the key is absent
// (Alg. 4's search and Alg. 3's insertion, as open addressing: linear
// probing from the home slot, a relaxed load first, atomicCAS only on EMPTY).
// Returns false after max_probes slots without success.
// `claimed` (optional): set when this call claimed the slot (a new vertex).
__device__ __forceinline__ bool find_or_claim(Slot *table, uint64_t n_slots, uint32_t max_probes,
                                              uint64_t key, uint64_t &slot_out,
                                              bool *claimed = nullptr) {
  uint64_t s = home_slot(key, n_slots);
  for (uint32_t i = 0; i < max_probes; ++i) {
    unsigned long long cur = ld_relaxed_u64(&table[s].key);
    if (cur == key) {
      slot_out = s;
      return true;
    }
    if (cur == kEmpty) {
      unsigned long long prev = atomicCAS(&table[s].key, kEmpty, (unsigned long long)key);
      if (prev == kEmpty || prev == key) {
        slot_out = s;
        if (claimed) *claimed = prev == kEmpty;
        return true;
      }
    }
    if (++s == n_slots) s = 0;
  }
  return false;
}


// Every graph's small block of device memory (64 bytes beside its table):
// the sticky status (u32) at byte 0; a flag at 4 set by a rebuild from empty
// on the tiled binned path whose vertex and edge counts at 40 and 48 are then
// exact (cleared when the build falls back to the direct insert); the stats
// accumulators (2 x u64) at 16; the spill count (u64) at 32.  Kernels reach
// the flag and the counts from an item's status pointer.
constexpr size_t kSmallCounted = 4, kSmallAcc = 16, kSmallSpill = 32, kSmallBuilt = 40;
__host__ __device__ inline uint32_t *small_counted(uint32_t *status) {
  return reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(status) + kSmallCounted);
}
__host__ __device__ inline unsigned long long *small_built(uint32_t *status) {
  return reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(status) + kSmallBuilt);
}

// Scratch of the binned insert: event buffers and bookkeeping, owned by a
// handle (its single-read-set inserts) or by the library (batched inserts).
struct BinScratch {
  uint64_t *ev = nullptr;               // events, 8 bytes each
  uint64_t cap = 0;                     // capacity in events
  uint64_t *ev2 = nullptr;              // tiled apply: events again, grouped by table tile
  void *aux = nullptr;                  // tiled apply: units, tile buckets, region table
  uint64_t aux_bytes = 0;
  unsigned long long *meta = nullptr;   // region counts, ranges, cursors, flag
  unsigned long long *counters = nullptr;  // the last call's overflow and deferred counts
                                           // (tiled apply; null otherwise)
  cudaEvent_t done = nullptr;           // orders the calls that share the scratch
};

// Release a scratch's buffers (the caller synchronises first).
void free_bin_scratch(BinScratch &sc);

}  // namespace dbg

// The handle.
struct dbg_graph {
  int k = 0;
  int device = 0;
  uint64_t n_slots = 0;
  uint32_t max_probes = 0;
  bool max_probes_auto = true;  // max_probes follows the table size
  dbg::Slot *table = nullptr;
  bool owns_slots = true;               // table allocated by the handle (not dbg_create_on's)
  bool owns_small = true;               // status block allocated by the handle
  uint32_t *d_status = nullptr;
  unsigned long long *d_acc = nullptr;  // [2]: vertices, edges (stats)
  unsigned long long *d_spill_count = nullptr;  // spilled vertex positions
  dbg::SpillRecord *d_spill = nullptr;
  uint64_t spill_cap = 0;
  dbg_tuning tuning{};                  // as set by the user (0 = auto)
  int sm_count = 0;
  // staging for dbg_insert_reads_host
  uint8_t *stage_packed[2] = {nullptr, nullptr};
  uint64_t *stage_offsets[2] = {nullptr, nullptr};
  uint64_t stage_packed_bytes = 0;
  uint64_t stage_offsets_count = 0;
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_copied[2] = {nullptr, nullptr};
  cudaEvent_t ev_consumed[2] = {nullptr, nullptr};
  cudaEvent_t ev_part[8] = {};                // parts of a whole-input copy (kInputParts)
  // binned insert scratch (allocated when a single-read-set binned insert
  // first needs it; batched inserts use the library's own)
  dbg::BinScratch bin;
  uint64_t bin_want = 0;                    // events asked for by dbg_reserve_events (0: default)
  // the last call that changed the graph was a rebuild on the tiled binned
  // path, which counts its vertices and edges (see small_counted): dbg_stats
  // then reads them instead of counting the table
  bool built_counts = false;
  // optional per-kernel timing of insert calls (dbg_enable_kernel_timing)
  int timer_cap = 0;                        // calls kept
  int timer_calls = 0;                      // calls recorded (may exceed timer_cap)
  cudaEvent_t *timer_ev = nullptr;          // timer_cap * kTimerMarks events
  signed char *timer_mark_set = nullptr;    // which marks of each call were recorded
};

namespace dbg {

// Kernel boundaries of one insert call for the optional timer: mark i is
// recorded before kernel i; the last mark after the last kernel.
//   0 direct insert | 1 bin count | 2 bin scan | 3 bin scatter | 4 bin split |
//   5 bin apply | 6 bin deferred | 7 gated direct insert (binned fall-back) | 8 end
constexpr int kTimerMarks = 9;
constexpr int kTimerKernels = kTimerMarks - 1;

// Start recording a call (no-op when timing is off); returns the ring slot.
int timer_begin_call(dbg_handle h);
// Record mark `m` of ring slot `call` on stream s (no-op when call < 0).
void timer_mark(dbg_handle h, int call, int m, cudaStream_t s);

// Error plumbing shared by the entry points (host side).
int cuda_fail(cudaError_t e, const char *what);
// Temporary device memory from the library's stream-ordered pool (free it
// with cudaFreeAsync on a stream).
int scratch_alloc(void **p, size_t bytes, cudaStream_t s);
// Give the pools' cached memory back to the device (synchronising each device).
int release_scratch_pools();
// Device bytes the pool of device `dev` holds now.
uint64_t pool_reserved_bytes(int dev);
int launch_grow(dbg_handle h, uint64_t new_capacity, cudaStream_t s);

// Propagate a non-OK status from a library call.
#define DBG_TRY(...)               \
  do {                             \
    const int st_ = (__VA_ARGS__); \
    if (st_ != DBG_OK) return st_; \
  } while (0)

#define DBG_CK(call)                                        \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return dbg::cuda_fail(e_, #call); \
  } while (0)

// Fill an ItemDesc for a handle and a read set.
ItemDesc make_item(dbg_handle h, const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads,
                   uint64_t origin);

// Items passed to one insert launch by value (kernel parameter space), so a
// launch needs no descriptor upload.  N = 1 for a single read set; batches
// are cut into launches of at most kBatchItems items (ItemPack<128> is 14 KB
// of the 32 KB parameter space).
constexpr int kBatchItems = 128;
template <int N>
struct ItemPack {
  int n_items;
  int pad_;
  uint64_t total_tiles;
  ItemDesc d[N];
};

// Launch the insert kernel over host-side descriptors items[0..n_items)
// (tile_begin already set, total_tiles their sum); n_items <= kBatchItems.
// `gate`: if not null, the kernel does nothing when *gate != 0 (read on the
// device when it runs).
int launch_insert(const ItemDesc *items, int n_items, uint64_t total_tiles,
                  const dbg_tuning &tuning, int sm_count, cudaStream_t stream,
                  const uint32_t *gate = nullptr);

// Resolved tuning (defaults filled in).
dbg_tuning resolve_tuning(const dbg_tuning &t);

// Table kernels.
// (gate: if not null, the kernel does nothing when *gate != 0, read on the
// device when it runs -- the binned path's "binned kernels did the work" flag)
int launch_table_init(Slot *table, uint64_t n_slots, cudaStream_t stream,
                      const uint32_t *gate = nullptr);
int launch_stats(const Slot *table, uint64_t n_slots, unsigned long long *acc, cudaStream_t stream,
                 bool wide);
// Graphs with k > 32 (128-bit keys, dbg_wide.cu).
int launch_insert_wide(const ItemDesc &it, int sm_count, cudaStream_t s);
int export_sorted_wide(dbg_handle h, uint64_t D, uint64_t *keys_out, uint32_t *counts_out,
                       cudaStream_t s);

}  // namespace dbg
