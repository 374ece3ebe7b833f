// K1: the fused read-tile insert kernel -- Alg. 2 "makeGraph" with Alg. 3
// "addLeftVertex", Alg. 4 "findVertex" and the addRightVertex prose, done the
// GPU way.
//
// Work unit: a tile of `tile_reads` consecutive reads of one item.  A CTA
//   1. stages the tile's offsets in shared memory, computes each read's vertex
//      count (len - k + 2 for len >= k, else 0; the last vertex of a read is a
//      target only) and a block-wide prefix sum of them;
//   2. stages the packed bases the tile spans in shared memory with coalesced
//      16-byte loads (a tile too wide for the window is cut into sub-tiles;
//      a single read wider than the window reads its bases from global memory);
//   3. maps one thread to one vertex position of the flattened tile, extracts
//      the vertex key (k-1 bases, first base most significant) from two
//      64-bit words of the window with a funnel shift and a pair reversal;
//   4. finds or claims the key's slot: linear probing from the hash's home
//      slot, a relaxed load first and atomicCAS(EMPTY -> key) only on an
//      empty slot, so that a found vertex costs one L2 read and no atomic;
//   5. if the position starts a k-mer (j <= len - k), adds 1 to the slot's
//      counter for the label s_{k-1} (a fire-and-forget RED at L2).
// Counters start at zero (table init), so a thread that loses the CAS race
// for a key can count at once: no allocate/retry/free loop (Alg. 3's
// do-while) is needed, and the result is independent of thread order.
//
// Optional warp aggregation (__match_any_sync): lanes of a warp holding the
// same key probe once (the lowest lane), and lanes adding to the same
// (slot, label) counter issue one atomicAdd of the group size.
//
// Probing is bounded by max_probes; a vertex that finds neither its key nor
// an empty slot sets the sticky DBG_ERR_CAPACITY and the CTA stops, and later
// tiles of the item are skipped, so an overfull table never spins.
#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr int kWinWords = 2048;  // 16 KB window of packed bases per CTA (64 Ki bases)
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint4 ldg_stream_v4(const uint8_t *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Find the slot holding `key`, claiming an empty one if the key is absent
// (Alg. 3 lines "FindVertex"/"CAS" as open addressing).  Returns false after
// max_probes slots without success.
__device__ __forceinline__ bool find_or_claim(Slot *table, uint64_t n_slots, uint32_t max_probes,
                                              uint64_t key, uint64_t &slot_out) {
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
        return true;
      }
    }
    if (++s == n_slots) s = 0;
  }
  return false;
}

template <bool AGG>
__device__ __forceinline__ void insert_vertex(bool valid, uint64_t key, bool edge, uint32_t label,
                                              Slot *table, uint64_t n_slots, uint32_t max_probes,
                                              uint32_t *status, volatile uint32_t *s_cap_hit,
                                              int lane) {
  if (!AGG) {
    if (valid) {
      uint64_t slot;
      if (find_or_claim(table, n_slots, max_probes, key, slot)) {
        if (edge) atomicAdd(&table[slot].cnt[label], 1u);
      } else {
        set_sticky(status, DBG_ERR_CAPACITY);
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
      ok = find_or_claim(table, n_slots, max_probes, key, slot) ? 1 : 0;
      if (!ok) {
        set_sticky(status, DBG_ERR_CAPACITY);
        *s_cap_hit = 1u;
      }
    }
    slot = __shfl_sync(kFull, slot, leader);
    ok = __shfl_sync(kFull, ok, leader);
    const bool add = valid && ok && edge;
    const unsigned long long ek = add ? ((slot << 2) | label) : kEmpty;
    const unsigned grp = __match_any_sync(kFull, ek);
    if (add && lane == __ffs(grp) - 1) atomicAdd(&table[slot].cnt[label], (uint32_t)__popc(grp));
  }
}

// Key (and label) of the vertex at base p, read from global memory: used only
// for a read wider than the shared-memory window.
__device__ __forceinline__ uint64_t key_from_global(const uint8_t *packed, uint64_t nbytes,
                                                    uint64_t p, int m, uint32_t &label) {
  const uint64_t b0 = p >> 2;
  uint64_t lo = 0, hi = 0;
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    const uint64_t b = b0 + i;
    const uint64_t x = b < nbytes ? (uint64_t)__ldg(packed + b) : 0ull;
    if (i < 8)
      lo |= x << (8 * i);
    else
      hi |= x << (8 * (i - 8));
  }
  const uint32_t sh = (uint32_t)(p & 3) * 2;
  const uint32_t rel = (uint32_t)(p & 3) + (uint32_t)m;  // label base, relative
  label = (uint32_t)((rel < 32 ? (lo >> (2 * rel)) : (hi >> (2 * rel - 64))) & 3ull);
  return key_from_words(lo, hi, sh, m);
}

template <int N>
__device__ __forceinline__ int find_item(const ItemPack<N> &pk, uint64_t t) {
  if (N == 1) return 0;
  int lo = 0, hi = pk.n_items - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pk.d[mid].tile_begin <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <int BLOCK, bool AGG, int N>
__global__ void __launch_bounds__(BLOCK) k_insert(const __grid_constant__ ItemPack<N> pk, int tile_reads) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  uint64_t *s_win = reinterpret_cast<uint64_t *>(smem_raw);  // kWinWords + 2
  uint64_t *s_off = s_win + kWinWords + 2;                     // tile_reads + 1
  uint64_t *s_vpre = s_off + tile_reads + 1;                   // tile_reads + 1

  __shared__ ItemDesc s_item;
  __shared__ int s_item_idx;
  __shared__ uint32_t s_stop;
  __shared__ uint64_t s_nbytes;
  __shared__ uint64_t s_warp[BLOCK / 32];
  __shared__ int s_rb, s_global;
  __shared__ uint64_t s_wb0;
  __shared__ volatile uint32_t s_cap_hit;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_item_idx = -1;

  const uint64_t total_tiles = pk.total_tiles;
  for (uint64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    if (tid == 0) {
      const int ii = find_item(pk, t);
      if (ii != s_item_idx) {
        s_item = pk.d[ii];
        s_item_idx = ii;
        const uint64_t last = s_item.offsets[s_item.n_reads];
        s_nbytes = last >= s_item.origin ? (last - s_item.origin + 3) >> 2 : 0;
        if (last < s_item.origin) set_sticky(s_item.status, DBG_ERR_BAD_OFFSETS);
      }
      s_stop = ld_volatile_u32(s_item.status);
      s_cap_hit = 0u;
    }
    __syncthreads();
    if (s_stop == 0u) {
      const uint8_t *packed = s_item.packed;
      const uint64_t origin = s_item.origin;
      Slot *table = s_item.table;
      const uint64_t n_slots = s_item.n_slots;
      const uint32_t max_probes = s_item.max_probes;
      uint32_t *status = s_item.status;
      const int k = s_item.k, m = k - 1;
      const uint64_t nbytes = s_nbytes;
      const int vec_ok = s_item.vec_ok;
      const uint64_t r0 = (t - s_item.tile_begin) * (uint64_t)tile_reads;
      const int nr = (int)min((uint64_t)tile_reads, s_item.n_reads - r0);

      // 1. offsets, vertex counts, exclusive prefix
      for (int i = tid; i <= nr; i += BLOCK) s_off[i] = s_item.offsets[r0 + i];
      __syncthreads();
      uint64_t nv = 0;
      int bad = 0;
      if (tid < nr) {
        const uint64_t a = s_off[tid], b = s_off[tid + 1];
        if (b < a || a < origin) {
          bad = 1;
        } else {
          const uint64_t len = b - a;
          nv = len >= (uint64_t)k ? len - (uint64_t)k + 2 : 0;
        }
      }
      bad = __syncthreads_or(bad);
      if (!bad) {
        uint64_t incl = nv;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint64_t o = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += o;
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        if (warp == 0) {
          uint64_t w = lane < BLOCK / 32 ? s_warp[lane] : 0;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += o;
          }
          if (lane < BLOCK / 32) s_warp[lane] = w;  // inclusive over warps
        }
        __syncthreads();
        const uint64_t excl = incl - nv + (warp > 0 ? s_warp[warp - 1] : 0);
        if (tid < nr) s_vpre[tid] = excl;
        if (tid == nr - 1) s_vpre[nr] = excl + nv;
        __syncthreads();

        // 2-5. sub-tiles whose bases fit the window
        const uint64_t cap_bytes = (uint64_t)kWinWords * 8 - 16;
        int ra = 0;
        while (ra < nr) {
          if (tid == 0) {
            const uint64_t wb0 = ((s_off[ra] - origin) >> 2) & ~15ull;
            auto fits = [&](int rb) {
              return ((s_off[rb] - origin + 3) >> 2) - wb0 <= cap_bytes;
            };
            int rb;
            if (!fits(ra + 1)) {
              rb = ra + 1;
              s_global = 1;
            } else {
              int lo = ra + 1, hi = nr;  // largest rb in [lo, hi] that fits
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (fits(mid))
                  lo = mid;
                else
                  hi = mid - 1;
              }
              rb = lo;
              s_global = 0;
            }
            s_rb = rb;
            s_wb0 = wb0;
          }
          __syncthreads();
          const int rb = s_rb;
          const bool gmode = s_global != 0;
          const uint64_t wb0 = s_wb0;
          if (!gmode) {
            const uint64_t need_end = (s_off[rb] - origin + 3) >> 2;
            const uint64_t wend = min(need_end, nbytes);
            const uint64_t nb = wend > wb0 ? wend - wb0 : 0;
            unsigned char *wbytes = reinterpret_cast<unsigned char *>(s_win);
            uint64_t done = 0;
            if (vec_ok) {
              const uint64_t nvec = nb >> 4;
              uint4 *wv = reinterpret_cast<uint4 *>(s_win);
              for (uint64_t i = tid; i < nvec; i += BLOCK) wv[i] = ldg_stream_v4(packed + wb0 + 16 * i);
              done = nvec << 4;
            }
            for (uint64_t i = done + tid; i < nb; i += BLOCK) wbytes[i] = __ldg(packed + wb0 + i);
            __syncthreads();
          }
          const uint64_t v_lo = s_vpre[ra], v_hi = s_vpre[rb];
          int r = ra;
          for (uint64_t base = v_lo; base < v_hi; base += BLOCK) {
            if (AGG) {
              if (__any_sync(kFull, s_cap_hit != 0u)) break;
            } else if (s_cap_hit != 0u) {
              break;
            }
            const uint64_t v = base + tid;
            const bool valid = v < v_hi;
            uint64_t key = kEmpty;
            bool edge = false;
            uint32_t label = 0;
            if (valid) {
              while (s_vpre[r + 1] <= v) ++r;
              const uint64_t j = v - s_vpre[r];
              const uint64_t rs = s_off[r];
              const uint64_t len = s_off[r + 1] - rs;
              const uint64_t p = rs - origin + j;
              edge = j + (uint64_t)k <= len;
              if (!gmode) {
                const uint64_t q = p - (wb0 << 2);
                const uint32_t wi = (uint32_t)(q >> 5);
                key = key_from_words(s_win[wi], s_win[wi + 1], (uint32_t)(q & 31) * 2, m);
                const uint64_t qe = q + (uint64_t)m;
                label = (uint32_t)(s_win[qe >> 5] >> ((qe & 31) * 2)) & 3u;
              } else {
                key = key_from_global(packed, nbytes, p, m, label);
              }
            }
            insert_vertex<AGG>(valid, key, edge, label, table, n_slots, max_probes, status,
                               &s_cap_hit, lane);
          }
          __syncthreads();
          ra = rb;
        }
      } else if (tid == 0) {
        set_sticky(status, DBG_ERR_BAD_OFFSETS);
      }
    }
    __syncthreads();
  }
}

template <int BLOCK, bool AGG, int N>
int launch_one(const ItemPack<N> &pk, int tile_reads, int grid_ctas, int sm_count,
               cudaStream_t stream) {
  auto kern = k_insert<BLOCK, AGG, N>;
  const size_t smem = (size_t)(kWinWords + 2) * 8 + (size_t)(tile_reads + 1) * 16;
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
  kern<<<grid, BLOCK, smem, stream>>>(pk, tile_reads);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

template <int N>
int launch_pack(const ItemPack<N> &pk, const dbg_tuning &t, int sm_count, cudaStream_t stream) {
  const bool agg = t.warp_aggregate != 0;
#define DBG_LAUNCH(B)                                                                      \
  return agg ? launch_one<B, true, N>(pk, t.tile_reads, t.grid_ctas, sm_count, stream)    \
             : launch_one<B, false, N>(pk, t.tile_reads, t.grid_ctas, sm_count, stream)
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
  if (r.warp_aggregate < 0) r.warp_aggregate = 0;
  return r;
}

int launch_insert(const ItemDesc *items, int n_items, uint64_t total_tiles,
                  const dbg_tuning &tuning, int sm_count, cudaStream_t stream) {
  if (total_tiles == 0 || n_items <= 0) return DBG_OK;
  if (n_items > kBatchItems) return DBG_ERR_INVALID_ARG;
  const dbg_tuning t = resolve_tuning(tuning);
  if (n_items == 1) {
    ItemPack<1> pk{};
    pk.n_items = 1;
    pk.total_tiles = total_tiles;
    pk.d[0] = items[0];
    return launch_pack(pk, t, sm_count, stream);
  }
  ItemPack<kBatchItems> pk{};
  pk.n_items = n_items;
  pk.total_tiles = total_tiles;
  for (int i = 0; i < n_items; ++i) pk.d[i] = items[i];
  return launch_pack(pk, t, sm_count, stream);
}

}  // namespace dbg
