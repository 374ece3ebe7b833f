// K1 (direct path): the fused read-tile insert kernel -- Alg. 2 "makeGraph"
// with Alg. 3 "addLeftVertex", Alg. 4 "findVertex" and the addRightVertex
// prose, done the GPU way.  The tile walk, shared-memory staging and key
// extraction are in dbg_tiles.cuh; this file is what happens to a vertex:
//
//   find or claim the key's slot: linear probing from the hash's home slot,
//   a relaxed load first and atomicCAS(EMPTY -> key) only on an empty slot,
//   so that a found vertex costs one L2 read and no atomic; then, if the
//   position starts a k-mer (j <= len - k), add 1 to the slot's counter for
//   the label s_{k-1} (a fire-and-forget atomicAdd at L2).
//
// Counters start at zero (table init), so a thread that loses the CAS race
// for a key can count at once: no allocate/retry/free loop (Alg. 3's
// do-while) is needed, and the result is independent of thread order.
//
// Warp aggregation (__match_any_sync; on unless the tuning turns it off):
// lanes of a warp holding the same key probe once (the lowest lane), and
// lanes adding to the same (slot, label) counter issue one atomicAdd of the
// group size.
//
// Probing is bounded by max_probes; a vertex that finds neither its key nor
// an empty slot sets the sticky DBG_ERR_CAPACITY and the CTA stops, and later
// tiles of the item are skipped, so an overfull table never spins.
#include <algorithm>

#include "dbg_tiles.cuh"

namespace dbg {
namespace {

template <bool AGG>
struct InsertVisitor {
  static constexpr bool kUniformRounds = false;
  volatile uint32_t *s_cap_hit;

  __device__ void tile_begin() {
    if (threadIdx.x == 0) *s_cap_hit = 0u;
  }
  __device__ bool stop(int) {
    if (AGG) return __any_sync(kFull, *s_cap_hit != 0u);
    return *s_cap_hit != 0u;
  }
  __device__ void round_end() {}

  __device__ void vertex(bool valid, uint64_t key, bool edge, uint32_t label, int lane, int,
                         const VertexCtx &c) {
    if (!AGG) {
      if (valid) {
        uint64_t slot;
        if (find_or_claim(c.table, c.n_slots, c.max_probes, key, slot)) {
          if (edge) atomicAdd(&c.table[slot].cnt[label], 1u);
        } else if (spill_or_fail(c.spill, c.spill_cap, c.spill_count, c.status, key, edge, label)) {
          *s_cap_hit = 1u;
        }
      }
    } else {
      const unsigned long long mk = valid ? key : kEmpty;
      const unsigned peers = __match_any_sync(kFull, mk);
      const int leader = __ffs(peers) - 1;
      uint64_t slot = 0;
      int ok = 0;
      if (valid && lane == leader) {
        ok = find_or_claim(c.table, c.n_slots, c.max_probes, key, slot) ? 1 : 0;
        if (!ok) {
          // every lane of the group spills its own position below
          ok = -1;
        }
      }
      slot = __shfl_sync(kFull, slot, leader);
      ok = __shfl_sync(kFull, ok, leader);
      if (valid && ok < 0) {
        if (spill_or_fail(c.spill, c.spill_cap, c.spill_count, c.status, key, edge, label))
          *s_cap_hit = 1u;
        ok = 0;
      }
      const bool add = valid && ok > 0 && edge;
      const unsigned long long ek = add ? ((slot << 2) | label) : kEmpty;
      const unsigned grp = __match_any_sync(kFull, ek);
      if (add && lane == __ffs(grp) - 1)
        atomicAdd(&c.table[slot].cnt[label], (uint32_t)__popc(grp));
    }
  }
};

template <int BLOCK, bool AGG, int N>
__global__ void __launch_bounds__(BLOCK)
    k_insert(const __grid_constant__ ItemPack<N> pk, int tile_reads, const uint32_t *gate) {
  if (gate != nullptr && ld_volatile_u32(gate) != 0u) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ volatile uint32_t s_cap_hit;
  InsertVisitor<AGG> vis{&s_cap_hit};
  for_each_vertex<BLOCK, N, 1>(pk, tile_reads, smem_raw, vis, blockIdx.x, pk.total_tiles,
                               gridDim.x);
}

template <int BLOCK, bool AGG, int N>
int launch_one(const ItemPack<N> &pk, int tile_reads, int grid_ctas, int sm_count,
               cudaStream_t stream, const uint32_t *gate) {
  auto kern = k_insert<BLOCK, AGG, N>;
  const size_t smem = tile_smem_bytes(tile_reads);
  if (smem > 48 * 1024) {
    DBG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  int grid = grid_ctas;
  if (grid <= 0) {
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BLOCK, smem));
    grid = std::max(1, per_sm) * std::max(1, sm_count);
  }
  if ((uint64_t)grid > pk.total_tiles) grid = (int)pk.total_tiles;
  kern<<<grid, BLOCK, smem, stream>>>(pk, tile_reads, gate);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

template <int N>
int launch_pack(const ItemPack<N> &pk, const dbg_tuning &t, int sm_count, cudaStream_t stream,
                const uint32_t *gate) {
  const bool agg = t.warp_aggregate != 0;
#define DBG_LAUNCH(B)                                                                           \
  return agg ? launch_one<B, true, N>(pk, t.tile_reads, t.grid_ctas, sm_count, stream, gate)   \
             : launch_one<B, false, N>(pk, t.tile_reads, t.grid_ctas, sm_count, stream, gate)
  switch (t.block_threads) {
    case 128: DBG_LAUNCH(128);
    case 256: DBG_LAUNCH(256);
    case 512: DBG_LAUNCH(512);
    default: return DBG_ERR_INVALID_ARG;
  }
#undef DBG_LAUNCH
}

}  // namespace

dbg_tuning resolve_tuning(const dbg_tuning &t) {
  dbg_tuning r = t;
  if (r.block_threads <= 0) r.block_threads = 256;
  if (r.tile_reads <= 0 || r.tile_reads > r.block_threads) r.tile_reads = r.block_threads;
  // warp aggregation on by default: it costs nothing where a warp's keys
  // differ (100 Mbp direct insert: 155.9 ms either way) and merges repeats
  // (microsatellite reads: 0.85 -> 0.18 ms)
  if (r.warp_aggregate < 0) r.warp_aggregate = 1;
  if (r.apply_unroll <= 0) r.apply_unroll = 4;
  if (r.apply_chunk <= 0) r.apply_chunk = 8;
  if (r.apply_counters <= 0) r.apply_counters = 16;
  return r;
}

int launch_insert(const ItemDesc *items, int n_items, uint64_t total_tiles,
                  const dbg_tuning &tuning, int sm_count, cudaStream_t stream,
                  const uint32_t *gate) {
  if (total_tiles == 0 || n_items <= 0) return DBG_OK;
  if (n_items > kBatchItems) return DBG_ERR_INVALID_ARG;
  const dbg_tuning t = resolve_tuning(tuning);
  if (n_items == 1) {
    ItemPack<1> pk{};
    pk.n_items = 1;
    pk.total_tiles = total_tiles;
    pk.d[0] = items[0];
    return launch_pack(pk, t, sm_count, stream, gate);
  }
  ItemPack<kBatchItems> pk{};
  pk.n_items = n_items;
  pk.total_tiles = total_tiles;
  for (int i = 0; i < n_items; ++i) pk.d[i] = items[i];
  return launch_pack(pk, t, sm_count, stream, gate);
}

}  // namespace dbg
