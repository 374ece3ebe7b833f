// The binned insert: the same table updates as the direct insert kernel
// (find or claim the prefix and suffix vertices, count the label -- Alg. 2-4
// and the addRightVertex prose), issued in an order that keeps them on chip.
//
// A random 32-byte slot of a table far larger than L2 costs a DRAM round trip
// that fetches a whole line, which caps the direct insert near the
// random-sector rate of HBM.  So for a large table the insert runs as:
//   buckets -- the read set's vertex positions, and for every table region
//              (2^shift slots, at most 2048 regions) a bucket of its
//              expected events plus a margin of several standard deviations;
//   scatter -- walk the read tiles, compute every vertex's key and home
//              slot, and write one 8-byte event per vertex,
//              (key << 3) | (edge << 2) | label, into its region's bucket
//              (block-local counting sort in shared memory; each flush's
//              run appended to its bucket with one atomic);
//   split   -- per region, regroup the events into per-tile buckets of the
//              region's mean per 2048-slot tile plus a margin (a counting
//              sort per chunk in shared memory, one atomic per tile and
//              chunk; what does not fit goes to an overflow area);
//   apply   -- one CTA per tile: a bulk copy brings the tile into shared
//              memory, the tile's events are applied there with
//              shared-memory CAS and add, a bulk copy writes it back;
//   deferred -- the events whose probe left their tile and those of the
//              overflow area, from their home slot, with the global
//              find-or-claim.
// The earlier streaming apply (all CTAs sweep the region-ordered events with
// global atomics inside an L2-resident window) remains as apply_mode = 1; it
// needs gap-free region ranges, so it keeps an exact count pass (histogram
// per slice of tiles) and its scan ahead of the scatter.
// The result is identical to the direct insert (additions commute).  Events
// hold a key of at most 60 bits, so the binned path serves k <= 31.  If the
// buckets do not fit the handle's event buffer, or one of them fills up,
// every later binned kernel returns at once and the direct insert kernel,
// launched last with the same flag as its gate, does the work instead.
#include <algorithm>
#include <mutex>
#include <vector>

#include "dbg_binned.cuh"
#include "dbg_tiles.cuh"
#include "dbg_tma.cuh"

namespace dbg {
namespace {

constexpr int kMaxParts = kBinMaxParts;
constexpr int kRun = 8;             // consecutive vertex positions per thread (rolled keys)

constexpr int kTileLog2 = 11;
constexpr int kTileSlots = 1 << kTileLog2;  // 2048 slots: 64 KB as 32-byte slots, 48 KB split
constexpr int kMaxTilesPerRegion = 4096;    // beyond this the streaming apply is used
constexpr int kTiledShift = 21;             // automatic regions of the tiled path: 1024 tiles

// The tiled path's bookkeeping for one chain of items (one or many tables).
// Regions never span two tables: item i's table is cut into regions
// region0_i, region0_i + 1, ... of 2^shift slots (the last one shorter), and
// every region into tiles of kTileSlots slots (the last one shorter).  Tiles
// are numbered compactly, region after region.
struct TileAux {
  unsigned long long *unit_base;     // [parts + 1] units of the regions before p
  unsigned long long *region_base;   // [parts + 1] region p's first bucket; [parts]: overflow area
  uint32_t *tile_cap;                // [parts] events one tile bucket of region p holds
  uint32_t *fill;                    // [tiles] events each tile received (zeroed per call)
  uint32_t *region_item;             // [parts] the item (table) of region p
  unsigned long long *region_first;  // [parts] region p's first slot in its table
  unsigned long long *region_nslots; // [parts] slots of that table
  uint32_t *region_tile0;            // [parts + 1] compact index of region p's first tile
  uint16_t *tile_region;             // [tiles] region of every tile (chains of many tables)
  unsigned long long *deferred_n;    // [parts] events of region p whose probe left their tile
  unsigned long long *overflow;      // [1] events in the overflow area
  unsigned long long *deferred;      // [1] events whose probe left their tile, in all
};

__device__ __forceinline__ uint64_t make_event(uint64_t key, bool edge, uint32_t label) {
  return (key << 3) | ((uint64_t)edge << 2) | (uint64_t)label;
}

// Work is cut into `slices` equal runs of consecutive tiles; CTAs take slices
// (count, scatter) or event chunks (apply) from counters in the meta area, so
// that every CTA works near the others: the apply pass then touches a narrow,
// L2-resident window of the table.

// The next work unit from counter *ctr, the same for every thread of the CTA;
// ~0 when `status` (if given) holds an error, so the CTA stops as one.
__device__ __forceinline__ uint64_t grab(unsigned long long *ctr, const uint32_t *status = nullptr) {
  __shared__ unsigned long long s_next;
  if (threadIdx.x == 0) {
    s_next = (status != nullptr && ld_volatile_u32(status) != 0u) ? ~0ull : atomicAdd(ctr, 1ull);
  }
  __syncthreads();
  const uint64_t v = s_next;
  __syncthreads();
  return v;
}

// --- K1b --------------------------------------------------------------------

struct CountVisitor {
  static constexpr bool kUniformRounds = false;
  uint32_t *s_hist;
  int shift;
  __device__ void tile_begin() {}
  __device__ bool stop(int) { return false; }
  __device__ void vertex(bool valid, uint64_t key, bool, uint32_t, int, int, const VertexCtx &c) {
    if (valid) atomicAdd(&s_hist[home_slot(key, c.n_slots) >> shift], 1u);
  }
  __device__ void round_end() {}
};

// hist[slice][region]: vertex positions of each slice that fall in each
// region; counts[region]: their sum over the slices.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_bin_count(const __grid_constant__ ItemPack<1> pk, int tile_reads, int shift, int parts,
                uint64_t slices, uint32_t *hist, unsigned long long *counts,
                unsigned long long *ctr) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_hist = reinterpret_cast<uint32_t *>(smem + tile_smem_bytes(tile_reads));
  const uint64_t T = pk.total_tiles;
  CountVisitor vis{s_hist, shift};
  for (;;) {
    const uint64_t sl = grab(&ctr[0]);
    if (sl >= slices) break;
    for (int p = threadIdx.x; p < parts; p += BLOCK) s_hist[p] = 0;
    __syncthreads();
    for_each_vertex<BLOCK, 1, kRun>(pk, tile_reads, smem, vis, sl * T / slices,
                                    (sl + 1) * T / slices, 1);
    __syncthreads();
    for (int p = threadIdx.x; p < parts; p += BLOCK) {
      const uint32_t h = s_hist[p];
      hist[sl * parts + p] = h;
      if (h) atomicAdd(&counts[p], (unsigned long long)h);
    }
  }
}

// --- K1c --------------------------------------------------------------------

// One CTA of 1024 threads (parts <= 2048: two regions per thread):
// begin[p] = events of regions < p, begin[parts] = total, cursor[p] = begin[p],
// *use_binned = total <= cap; resets the scatter and apply counters.
__global__ void __launch_bounds__(1024)
    k_bin_scan(const unsigned long long *counts, int parts, unsigned long long *begin,
               unsigned long long *cursor, uint64_t cap, unsigned long long *ctr,
               uint32_t *use_binned) {
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p0 = 2 * tid;  // regions p0 and p0 + 1
  const unsigned long long ca = p0 < parts ? counts[p0] : 0ull;
  const unsigned long long cb = p0 + 1 < parts ? counts[p0 + 1] : 0ull;
  const unsigned long long local = ca + cb;
  unsigned long long incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = s_warp[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(kFull, w, d);
      if (lane >= d) w += o;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const unsigned long long b = incl - local + (warp > 0 ? s_warp[warp - 1] : 0ull);
  if (p0 < parts) begin[p0] = cursor[p0] = b;
  if (p0 + 1 < parts) begin[p0 + 1] = cursor[p0 + 1] = b + ca;
  if (tid == 0) {
    const unsigned long long total = s_warp[31];
    begin[parts] = total;
    *use_binned = total <= cap ? 1u : 0u;
    ctr[1] = 0;
    ctr[2] = 0;
  }
}

// --- bucketed reservation (the tiled path's replacement of K1b/K1c) -----------
//
// The tiled apply re-partitions every region's events by tile, so it needs
// each region's events together but not in an exact, gap-free range.  The
// count pass can then go: each region gets a bucket of its expected events
// (its share of the table's slots) with a margin, and the scatter appends
// every flush's run to its bucket.  Regions are drawn by the hash per
// distinct key, not per position, so a region's count varies with the keys'
// multiplicities (about the coverage for genomic keys): its standard
// deviation is sqrt(expected x mean squared multiplicity / mean multiplicity),
// about 10^4 events for the 100 Mbp workload's 4-million-event regions.  The
// margin, 3 % + 16 sqrt(expected) + 256, is several such deviations.  A
// bucket that fills up anyway (inputs dominated by a few heavily repeated
// keys) clears the use-binned flag, and the direct insert does the call
// instead, exactly as when the events exceed the buffer.

// totals[i] = vertex positions of item i's reads, sum of max(0, len - k + 2),
// and edges[i] = its k-mers, sum of max(0, len - k + 1) (grid: x strides over
// the item's reads, y = item).
// clear: also zero every item's sticky status and spill count (a rebuild
// from empty; this is the chain's first kernel, so every later one sees it).
template <int N>
__global__ void k_bin_totals(const __grid_constant__ ItemPack<N> pk, unsigned long long *totals,
                             unsigned long long *edges, int clear) {
  const int i = blockIdx.y;
  if (i >= pk.n_items) return;
  if (clear && blockIdx.x == 0 && threadIdx.x == 0) {
    *pk.d[i].status = 0u;
    *pk.d[i].spill_count = 0ull;
  }
  const uint64_t *offsets = pk.d[i].offsets;
  const uint64_t n_reads = pk.d[i].n_reads;
  const int k = pk.d[i].k;
  unsigned long long v = 0, ne = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += stride) {
    const uint64_t a = offsets[r], b = offsets[r + 1];
    const uint64_t len = b > a ? b - a : 0;
    if (len >= (uint64_t)k) {
      v += len - k + 2;
      ne += len - k + 1;
    }
  }
  for (int d = 16; d > 0; d >>= 1) {
    v += __shfl_down_sync(kFull, v, d);
    ne += __shfl_down_sync(kFull, ne, d);
  }
  if ((threadIdx.x & 31) == 0 && v) {
    atomicAdd(&totals[i], v);
    atomicAdd(&edges[i], ne);
  }
}

// Exclusive prefix over a CTA of 1024 threads; `total` receives the sum.
__device__ __forceinline__ unsigned long long cta1024_exclusive_scan(unsigned long long local,
                                                                     unsigned long long *s_warp,
                                                                     unsigned long long &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = s_warp[lane];
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(kFull, w, d);
      if (lane >= d) w += o;
    }
    s_warp[lane] = w;
  }
  __syncthreads();
  const unsigned long long ex = incl - local + (warp > 0 ? s_warp[warp - 1] : 0ull);
  total = s_warp[31];
  __syncthreads();  // s_warp is free again
  return ex;
}

// One CTA of 1024 threads (two regions each).  Region p belongs to the last
// item i with region0 <= p; it covers slots [first, first + slots) of that
// item's table and ceil(slots / kTileSlots) tiles.  Its bucket holds its
// share of the item's vertex positions plus the margin, and starts at
// begin[p]; cursor[p] = begin[p].  The region table (item, first slot, table
// size, first tile) is written for the later passes.  The flag says whether
// all buckets fit the buffer; the scatter's slice counter is reset.
template <int N>
__global__ void __launch_bounds__(1024)
    k_bin_buckets(const __grid_constant__ ItemPack<N> pk, const unsigned long long *totals,
                  const unsigned long long *edges, int fresh, int shift, int parts,
                  unsigned long long *begin, unsigned long long *cursor, uint64_t cap,
                  unsigned long long *ctr, uint32_t *use_binned, TileAux aux) {
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x;
  if (tid < pk.n_items) {  // a rebuild counts its vertices (its claims) and its edges
    uint32_t *st = pk.d[tid].status;
    *small_counted(st) = fresh ? 1u : 0u;
    if (fresh) {
      small_built(st)[0] = 0ull;
      small_built(st)[1] = edges[tid];
    }
  }
  unsigned long long bk[2], nt[2];
  for (int j = 0; j < 2; ++j) {
    const int p = 2 * tid + j;
    bk[j] = nt[j] = 0ull;
    if (p >= parts) continue;
    int lo = 0, hi = pk.n_items - 1;  // the last item whose first region is <= p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pk.d[mid].region0 <= p)
        lo = mid;
      else
        hi = mid - 1;
    }
    const uint64_t ns = pk.d[lo].n_slots;
    const uint64_t first = (uint64_t)(p - pk.d[lo].region0) << shift;
    const uint64_t slots = min((uint64_t)1 << shift, ns - first);
    const double expected = (double)totals[lo] * (double)slots / (double)ns;
    bk[j] = (unsigned long long)ceil(expected * 1.03 + 16.0 * sqrt(expected) + 256.0);
    nt[j] = (slots + kTileSlots - 1) >> kTileLog2;
    aux.region_item[p] = (uint32_t)lo;
    aux.region_first[p] = first;
    aux.region_nslots[p] = ns;
  }
  unsigned long long all, tiles;
  const unsigned long long b = cta1024_exclusive_scan(bk[0] + bk[1], s_warp, all);
  const unsigned long long t0 = cta1024_exclusive_scan(nt[0] + nt[1], s_warp, tiles);
  const int p0 = 2 * tid;
  if (p0 < parts) {
    begin[p0] = cursor[p0] = b;
    aux.region_tile0[p0] = (uint32_t)t0;
  }
  if (p0 + 1 < parts) {
    begin[p0 + 1] = cursor[p0 + 1] = b + bk[0];
    aux.region_tile0[p0 + 1] = (uint32_t)(t0 + nt[0]);
  }
  if (tid == 0) {
    begin[parts] = all;
    aux.region_tile0[parts] = (uint32_t)tiles;
    *use_binned = all <= cap ? 1u : 0u;
    ctr[1] = 0;
  }
}

// --- K1d --------------------------------------------------------------------

// Exclusive prefix of `local` over a CTA of BLOCK threads with one barrier:
// every warp scans the per-warp totals itself (no second pass by one warp).
// `total` receives the CTA's sum.  s_w (BLOCK / 32 words) must not be
// written again before the caller's next barrier.
template <int BLOCK>
__device__ __forceinline__ uint32_t cta_exclusive_prefix(uint32_t local, uint32_t *s_w,
                                                         uint32_t &total) {
  static_assert(BLOCK % 32 == 0 && BLOCK <= 1024, "whole warps, at most 32 of them");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_w[warp] = incl;
  __syncthreads();
  uint32_t w = lane < BLOCK / 32 ? s_w[lane] : 0u;
  for (int d = 1; d < BLOCK / 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(kFull, w, d);
    if (lane >= d) w += o;
  }
  total = __shfl_sync(kFull, w, BLOCK / 32 - 1);
  const uint32_t before = __shfl_sync(kFull, w, (warp + 31) & 31);  // warp - 1's inclusive sum
  return incl - local + (warp > 0 ? before : 0u);
}

// A round of the tile walk gives every thread kRun events; each keeps them in
// registers with its region and its rank in the region (a shared-memory
// atomic), then the round is flushed: an exclusive prefix of the region
// counts places the events in region order in shared memory (counting
// sort), and they are written out as runs.  A run's position: without a
// count pass (the tiled path), one atomic on the region's bucket cursor per
// round; after a count pass, the slice's run start in the region (reserved
// at the start of the slice) + the events of the region already placed.
template <int BLOCK>
struct ScatterVisitor {
  static constexpr bool kUniformRounds = true;
  static constexpr int kRound = BLOCK * kRun;  // events of one round = one flush
  uint64_t *sorted;    // kRound, in region order
  uint16_t *spid;      // region of sorted[j]
  uint32_t *hist;      // parts: events per region in this round
  uint32_t *off;       // parts: exclusive prefix of hist
  unsigned long long *cur;    // parts: next global position of each region (this slice)
  unsigned long long *gbase;  // parts: cur[p] - off[p] for this round
  uint64_t *out;
  uint64_t cap;  // events the buffer holds: never store past it
  int shift, parts;
  // bucketed mode: runs are appended to per-region buckets at flush time
  unsigned long long *bucket_cursor = nullptr;     // parts: next free position
  const unsigned long long *bucket_end = nullptr;  // parts: end of each bucket
  uint32_t *use_binned = nullptr;                  // cleared when a bucket overflows
  uint64_t ev[kRun];     // this thread's events of the round
  uint32_t where[kRun];  // region << 16 | rank, or ~0 for no event

  __device__ void tile_begin() {}
  __device__ bool stop(int) { return false; }
  __device__ void vertex(bool valid, uint64_t key, bool edge, uint32_t label, int, int sub,
                         const VertexCtx &c) {
    if (valid) {
      const uint32_t p = (uint32_t)c.region0 + (uint32_t)(home_slot(key, c.n_slots) >> shift);
      ev[sub] = make_event(key, edge, label);
      where[sub] = (p << 16) | atomicAdd(&hist[p], 1u);
    } else {
      where[sub] = ~0u;
    }
  }
  __device__ void round_end() {
    __shared__ uint32_t s_w[BLOCK / 32];
    __syncthreads();
    const int tid = threadIdx.x;
    // exclusive prefix over the regions; each region's place in the output
    const int per = (parts + BLOCK - 1) / BLOCK;
    const int p0 = min(parts, tid * per), p1 = min(parts, p0 + per);
    uint32_t local = 0;
    for (int p = p0; p < p1; ++p) local += hist[p];
    uint32_t total;
    uint32_t run = cta_exclusive_prefix<BLOCK>(local, s_w, total);
    for (int p = p0; p < p1; ++p) {
      const uint32_t h = hist[p];
      off[p] = run;
      if (bucket_cursor == nullptr) {
        gbase[p] = cur[p] - run;
        cur[p] += h;
      } else if (h) {
        const unsigned long long at = atomicAdd(&bucket_cursor[p], (unsigned long long)h);
        if (at + h > bucket_end[p]) {  // the bucket is full: the direct insert takes over
          atomicExch(use_binned, 0u);
          gbase[p] = ~0ull;
        } else {
          gbase[p] = at - run;
        }
      }
      run += h;
      hist[p] = 0;  // read by no one after this prefix: ready for the next round
    }
    __syncthreads();
    // counting sort of the registers into region order
#pragma unroll
    for (int sub = 0; sub < kRun; ++sub) {
      const uint32_t w = where[sub];
      if (w != ~0u) {
        const uint32_t p = w >> 16;
        const uint32_t j = off[p] + (w & 0xFFFFu);
        sorted[j] = ev[sub];
        spid[j] = (uint16_t)p;
      }
    }
    __syncthreads();
    for (uint32_t j = tid; j < total; j += BLOCK) {
      const unsigned long long g = gbase[spid[j]];
      const unsigned long long at = g + j;
      if (g != ~0ull && at < cap) __stcs(out + at, sorted[j]);
    }
    // no barrier here: the next round only touches hist (already cleared)
    // before its first barrier, and sorted / spid / gbase / s_w after it
  }
};

constexpr int kScatterTileReads = 416;  // reads per scatter tile without a count pass (<= 512)

int scatter_tile_reads(const dbg_tuning &t) {
  return t.scatter_reads > 0 ? t.scatter_reads : kScatterTileReads;
}

template <int BLOCK>
constexpr size_t scatter_smem(int tile_reads, int parts) {
  return tile_smem_bytes(tile_reads) + (size_t)BLOCK * kRun * (8 + 2) +
         (size_t)parts * (4 + 4 + 8 + 8) + 64;
}

template <int BLOCK, int N>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
    k_bin_scatter(const __grid_constant__ ItemPack<N> pk, int tile_reads, int shift, int parts,
                  uint64_t t0, uint64_t t1, uint64_t slices, const uint32_t *hist,
                  unsigned long long *cursor, uint64_t *out, uint64_t cap,
                  unsigned long long *ctr, uint32_t *use_binned,
                  const unsigned long long *bucket_end) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem + tile_smem_bytes(tile_reads);
  ScatterVisitor<BLOCK> vis;
  vis.sorted = reinterpret_cast<uint64_t *>(p);
  p += (size_t)ScatterVisitor<BLOCK>::kRound * 8;
  vis.gbase = reinterpret_cast<unsigned long long *>(p);
  p += (size_t)parts * 8;
  vis.cur = reinterpret_cast<unsigned long long *>(p);
  p += (size_t)parts * 8;
  vis.hist = reinterpret_cast<uint32_t *>(p);
  p += (size_t)parts * 4;
  vis.off = reinterpret_cast<uint32_t *>(p);
  p += (size_t)parts * 4;
  vis.spid = reinterpret_cast<uint16_t *>(p);
  vis.out = out;
  vis.cap = cap;
  vis.shift = shift;
  vis.parts = parts;
  if (bucket_end != nullptr) {  // bucketed: no count pass, runs appended per flush
    vis.bucket_cursor = cursor;
    vis.bucket_end = bucket_end;
    vis.use_binned = use_binned;
  }
  const uint64_t T = t1 - t0;  // this launch's read tiles: [t0, t1)
  for (int q = threadIdx.x; q < parts; q += BLOCK) vis.hist[q] = 0;
  for (;;) {
    const uint64_t sl = grab(&ctr[1]);
    if (sl >= slices) break;
    if (bucket_end == nullptr) {
      // reserve this slice's run in every region it reaches (counted by K1b)
      for (int q = threadIdx.x; q < parts; q += BLOCK) {
        const uint32_t h = hist[sl * parts + q];
        vis.cur[q] = h ? atomicAdd(&cursor[q], (unsigned long long)h) : 0ull;
      }
    }
    __syncthreads();
    for_each_vertex<BLOCK, N, kRun>(pk, tile_reads, smem, vis, t0 + sl * T / slices,
                                    t0 + (sl + 1) * T / slices, 1);
  }
}

// --- K1e --------------------------------------------------------------------

// One launch applies the events of a group of consecutive regions (by
// default all of them).  Each warp streams chunks of 32*M consecutive events
// (no block barriers).
// Chunk j is handed out by counter j % n_ctr: the counters advance side by
// side, so the chunks in flight stay close together in the event order (the
// table window they touch stays in L2) while no single counter is hammered
// by every warp.  Every lane keeps U probe slots.  A round first looks, in
// every slot, at the key word that arrived (a match counts the label; an
// empty slot gets an atomicCAS; another key moves the probe on), then the
// whole warp refills the free slots from the staged chunk -- lane by lane in
// ballot order, so no lane idles while the chunk has events -- and, half way
// through a chunk, loads the next chunk into registers so that it is ready
// when the staged one runs out.
template <int BLOCK, int U, int M>
__global__ void __launch_bounds__(BLOCK)
    k_bin_apply(const uint64_t *__restrict__ ev_all, const unsigned long long *begin,
                int part_first, int part_end, const uint32_t *use_binned, Slot *table,
                uint64_t n_slots, uint32_t max_probes, uint32_t *status, unsigned long long *ctrs,
                int n_ctr, SpillRecord *spill, uint64_t spill_cap,
                unsigned long long *spill_count) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  __shared__ uint64_t s_ev[BLOCK / 32][32 * M];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  uint64_t *buf = s_ev[wib];
  // this launch's events: those of regions [part_first, part_end)
  const uint64_t e0 = begin[part_first];
  const uint64_t total = begin[part_end] - e0;
  const uint64_t *__restrict__ ev = ev_all + e0;
  constexpr uint64_t kChunk = 32 * M;
  const uint64_t n_chunks = (total + kChunk - 1) / kChunk;
  const int gwarp = (int)((blockIdx.x * (uint64_t)BLOCK + threadIdx.x) >> 5);
  int k = gwarp % n_ctr;  // the counter this warp draws from (lane 0's copy counts)
  int tried = 0;          // counters found exhausted
  auto draw = [&]() -> uint64_t {  // lane 0 only
    while (tried < n_ctr) {
      if (ld_volatile_u32(status) != 0u) return n_chunks;
      const uint64_t j = atomicAdd(&ctrs[k], 1ull) * (uint64_t)n_ctr + (uint64_t)k;
      if (j < n_chunks) return j;
      ++tried;
      k = (k + 1) % n_ctr;
    }
    return n_chunks;
  };
  auto load_chunk = [&](uint64_t c, uint64_t (&dst)[M]) {
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const uint64_t i = c * kChunk + (uint64_t)j * 32 + lane;
      dst[j] = (c < n_chunks && i < total) ? __ldcs(ev + i) : kEmpty;
    }
  };

  unsigned long long c = 0, nc = 0;
  if (lane == 0) {
    c = draw();
    nc = draw();
  }
  c = __shfl_sync(kFull, c, 0);
  nc = __shfl_sync(kFull, nc, 0);
  uint64_t pre[M];
  load_chunk(c, pre);
#pragma unroll
  for (int j = 0; j < M; ++j) buf[j * 32 + lane] = pre[j];
  __syncwarp();
  uint32_t head = 0;                                      // next staged event to hand out
  uint32_t avail = c < n_chunks ? (uint32_t)kChunk : 0u;  // staged events
  bool have_pre = false;

  uint64_t e[U], s[U];
  unsigned long long cur[U];
  uint32_t probes[U];
  uint32_t active = 0, cas_done = 0;
  for (;;) {
    // 1. look at what arrived; issue each slot's next operation
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!(active & (1u << u))) continue;
      const unsigned long long key = e[u] >> 3;
      if (cur[u] == key) {
        if (e[u] & 4ull) atomicAdd(&table[s[u]].cnt[e[u] & 3ull], 1u);
        active &= ~(1u << u);
      } else if (cur[u] == kEmpty && !(cas_done & (1u << u))) {
        const unsigned long long prev = atomicCAS(&table[s[u]].key, kEmpty, key);
        cur[u] = prev == kEmpty ? key : prev;
        cas_done |= 1u << u;
      } else {
        if (++probes[u] >= max_probes) {
          spill_or_fail(spill, spill_cap, spill_count, status, key, (e[u] & 4ull) != 0,
                        (uint32_t)(e[u] & 3ull));
          active &= ~(1u << u);
          continue;
        }
        if (++s[u] == n_slots) s[u] = 0;
        cur[u] = ld_relaxed_u64(&table[s[u]].key);
        cas_done &= ~(1u << u);
      }
    }
    // 2. half way through the staged chunk: fetch the next one into registers
    if (!have_pre && nc < n_chunks && 2 * head >= avail) {
      load_chunk(nc, pre);
      have_pre = true;
    }
    // 3. the warp hands out staged events to free slots, in lane order
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const bool want = !(active & (1u << u));
      const unsigned b = __ballot_sync(kFull, want);
      const uint32_t pos = head + (uint32_t)__popc(b & lt_mask);
      if (want && pos < avail) {
        e[u] = buf[pos];
        if (e[u] != kEmpty) {
          s[u] = home_slot(e[u] >> 3, n_slots);
          cur[u] = ld_relaxed_u64(&table[s[u]].key);
          probes[u] = 0;
          cas_done &= ~(1u << u);
          active |= 1u << u;
        }
      }
      head = min(avail, head + (uint32_t)__popc(b));
    }
    // 4. staged chunk used up: stage the prefetched one, draw the one after
    if (head >= avail) {
      if (have_pre) {
        __syncwarp();
#pragma unroll
        for (int j = 0; j < M; ++j) buf[j * 32 + lane] = pre[j];
        __syncwarp();
        head = 0;
        avail = (uint32_t)kChunk;
        have_pre = false;
        unsigned long long nn = 0;
        if (lane == 0) nn = draw();
        nc = __shfl_sync(kFull, nn, 0);
      } else if (!__any_sync(kFull, active != 0u)) {
        break;  // nothing staged, nothing prefetched, nothing in flight
      }
    }
  }
}

// --- tiled apply -------------------------------------------------------------
//
// The streaming apply above keeps a table window in L2, but every event is
// still a round trip to L2 (a load, then a CAS or an add): ncu shows it
// stalled on those round trips, far below both the L2 and the DRAM peaks.
// The tiled apply instead gives each table tile of kTileSlots slots (64 KB) to
// one CTA: the CTA copies the tile into shared memory, applies every event
// whose home slot lies in the tile with shared-memory CAS and add, and
// writes the tile back.  The table then moves through DRAM once, in
// coalesced 16-byte accesses, and no event leaves the SM.
//
// That needs the events grouped by tile.  The scatter pass grouped them by
// region (2^shift slots = tiles_per_region tiles); a second, region-local
// partition pass (split) groups each region's events by tile:
//   units   -- one CTA: each region's event count, its units of `unit`
//              events, and one bucket per tile of the region in the second
//              buffer (the region's mean events per tile plus a margin), the
//              buckets of all regions end to end and an overflow area after
//              them;
//   scatter -- per unit, every event appended to its tile's bucket: each
//              chunk is counting-sorted by tile in shared memory, then each
//              tile's run takes its place with one atomic; what no longer
//              fits the bucket goes to the overflow area.
// No pass counts the tiles' events beforehand: the buckets are sized from
// the region counts alone, and a tile that receives more than its bucket
// holds (a key with many copies) sends the rest to the overflow area.
// Events in the overflow area, and events whose probe sequence runs off the
// end of their tile (keys homed near the end of a full stretch of slots),
// cannot be applied in the tile: the next tile belongs to another CTA.  They
// are applied afterwards, from their home slot, with the direct insert's
// global find-or-claim; the tiles are final by then.  The second kind are
// listed in the first event buffer, which the split pass has consumed.  If
// the overflow area fills up, the device flag turns the binned kernels off
// and the direct insert does the call (nothing has touched the table yet).
// A probe that reaches max_probes inside its tile fails (or spills) exactly
// as in the direct insert, so every key stays within max_probes of its home
// slot.

constexpr int kBatch = 8;  // events each thread loads before it uses them (memory parallelism)


// One CTA of 1024 threads, two regions each.  Region p's events are those
// its bucket received (cursor - begin); they become counts[p] and are cut
// into ceil(count / unit) units (unit_base, a prefix).  The region's tiles
// (rt of them, from the region table) get buckets of mean + slack events,
// mean = count / rt, slack = 3 % + 16 sqrt(mean) + 64 (a tile's count varies
// with its keys' multiplicities, as a region's does; at the 100 Mbp, 30x
// workload 0.1 % of the events overflow).  If the buckets and an overflow area of 1/64 of the
// buffer do not fit the buffer, the slack shrinks first, then the buckets.
__global__ void __launch_bounds__(1024)
    k_tile_units(unsigned long long *counts, const unsigned long long *begin,
                 const unsigned long long *cursor, int parts, uint64_t unit, uint64_t ev2_cap,
                 TileAux aux, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  __shared__ double s_red[3][32];
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  unsigned long long n[2];
  uint32_t rt[2];
  double mean[2], slack[2];
  double sums[3] = {0.0, 0.0, 0.0};  // events, slack over all buckets, buckets
  for (int i = 0; i < 2; ++i) {
    const int p = 2 * tid + i;
    n[i] = 0ull;
    rt[i] = 0u;
    mean[i] = slack[i] = 0.0;
    if (p < parts) {
      n[i] = cursor[p] - begin[p];
      counts[p] = n[i];
      rt[i] = aux.region_tile0[p + 1] - aux.region_tile0[p];
      if (n[i]) {
        mean[i] = (double)n[i] / (double)rt[i];
        slack[i] = 0.03 * mean[i] + 16.0 * sqrt(mean[i]) + 64.0;
        sums[0] += (double)n[i];
        sums[1] += slack[i] * (double)rt[i];
        sums[2] += (double)rt[i];
      }
    }
  }
  for (int j = 0; j < 3; ++j) {
    double v = sums[j];
    for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
    if (lane == 0) s_red[j][warp] = v;
  }
  __syncthreads();
  if (warp == 0) {
    for (int j = 0; j < 3; ++j) {
      double v = s_red[j][lane];
      for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
      if (lane == 0) s_red[j][0] = v;
    }
  }
  __syncthreads();
  const double N = s_red[0][0], D = s_red[1][0], R = s_red[2][0];
  const double avail = (double)(ev2_cap - ev2_cap / 64);
  const double f = D > 0.0 ? fmin(1.0, fmax(0.0, (avail - N - R) / D)) : 0.0;
  const double want = N + f * D;
  const double g = want > avail ? avail / want : 1.0;
  uint32_t cap[2];
  for (int i = 0; i < 2; ++i) cap[i] = n[i] ? (uint32_t)floor((mean[i] + f * slack[i]) * g) : 0u;

  const unsigned long long ua = (n[0] + unit - 1) / unit, ub = (n[1] + unit - 1) / unit;
  unsigned long long units_total, buckets_total;
  const unsigned long long u0 = cta1024_exclusive_scan(ua + ub, s_warp, units_total);
  const unsigned long long sa = (unsigned long long)rt[0] * cap[0];
  const unsigned long long sb = (unsigned long long)rt[1] * cap[1];
  const unsigned long long b0 = cta1024_exclusive_scan(sa + sb, s_warp, buckets_total);
  for (int i = 0; i < 2; ++i) {
    const int p = 2 * tid + i;
    if (p < parts) {
      aux.unit_base[p] = u0 + (i ? ua : 0ull);
      aux.region_base[p] = b0 + (i ? sa : 0ull);
      aux.tile_cap[p] = cap[i];
    }
  }
  if (tid == 0) {
    aux.unit_base[parts] = units_total;
    aux.region_base[parts] = buckets_total;
    *aux.overflow = 0ull;
    *aux.deferred = 0ull;
  }
  for (int i = 0; i < 2; ++i) {
    const int p = 2 * tid + i;
    if (p < parts) aux.deferred_n[p] = 0ull;
  }
}

// Region of unit u (the last p with unit_base[p] <= u) and its event range.
__device__ __forceinline__ int unit_region(const unsigned long long *unit_base, int parts,
                                           uint64_t u) {
  int lo = 0, hi = parts - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (unit_base[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// Tile of an event inside its region: its home slot in the region's table
// (n_slots slots), relative to the region's first tile.
__device__ __forceinline__ uint32_t tile_in_region(uint64_t ev, uint64_t n_slots,
                                                   uint64_t first_tile) {
  const uint64_t home = home_slot(ev >> 3, n_slots);
  return (uint32_t)((home >> kTileLog2) - first_tile);
}

// kBatch events of [base, b) strided by BLOCK, kEmpty past b (never an event:
// events hold keys of at most 60 bits).
template <int BLOCK>
__device__ __forceinline__ void load_batch(const uint64_t *__restrict__ ev, uint64_t base,
                                           uint64_t b, uint64_t (&e)[kBatch]) {
#pragma unroll
  for (int r = 0; r < kBatch; ++r) {
    const uint64_t i = base + (uint64_t)r * BLOCK + threadIdx.x;
    e[r] = i < b ? __ldcs(ev + i) : kEmpty;
  }
}

// Per unit: every event appended to its tile's bucket in the second buffer.
// Each chunk of BLOCK * kBatch events is counting-sorted by tile in shared
// memory first, so that every tile's run of the chunk is written by
// consecutive threads to consecutive addresses (coalesced stores instead of
// one scattered 8-byte store per event) and takes its place in the bucket
// with one atomic.  STAGED: a bulk copy brings the CTA's next chunk into
// shared memory while the current one is sorted and written (the events'
// load latency leaves the critical path); the 1024-thread form for large
// regions has no room for the stage and loads to registers.
constexpr int kMaxBinsPerThread = 4;  // tiles per region / tile scatter threads, at most

template <int BLOCK, bool STAGED>
constexpr size_t tile_scatter_smem(int tpr) {
  return (size_t)BLOCK * kBatch * (8 + 4) + (STAGED ? ((size_t)BLOCK * kBatch + 2) * 8 : 0) +
         (size_t)tpr * 20;
}

// A CTA's chunks, in order: its units blockIdx.x, + gridDim.x, ..., each cut
// into chunks [x, y) of at most C events of the unit's range [., b).
struct TileChunk {
  uint64_t u, x, y, b;
  int p;  // region of unit u
};

// The first chunk of unit u (false past the last unit).  Units are never
// empty; p_hint is a region at or before u's (the regions only grow along a
// CTA's units, so the walk forward is short).
__device__ __forceinline__ bool tile_chunk_first(uint64_t u, int p_hint, uint64_t C,
                                                 const unsigned long long *begin,
                                                 const unsigned long long *counts,
                                                 const TileAux &aux, int parts, uint64_t unit,
                                                 TileChunk &c) {
  if (u >= aux.unit_base[parts]) return false;
  int p = p_hint;
  while (p + 1 < parts && aux.unit_base[p + 1] <= u) ++p;
  c.u = u;
  c.p = p;
  c.x = begin[p] + (u - aux.unit_base[p]) * unit;
  c.b = min(c.x + unit, (uint64_t)(begin[p] + counts[p]));
  c.y = min(c.x + C, c.b);
  return true;
}

// Bulk copy of events [x & ~1, y & ~1) (16-byte aligned ends) into the stage;
// an odd last event is read from global memory by its thread.
__device__ __forceinline__ void stage_chunk(uint64_t *stage, const uint64_t *ev, uint64_t x,
                                            uint64_t y, uint64_t *bar) {
  const uint64_t x0 = x & ~1ull, y1 = y & ~1ull;
  const uint32_t bytes = y1 > x0 ? (uint32_t)((y1 - x0) * sizeof(uint64_t)) : 0u;
  mbar_expect_tx(bar, bytes);  // (0 bytes: the phase completes with this arrival)
  if (bytes) bulk_load(stage, ev + x0, bytes, bar);
}

template <int BLOCK, bool STAGED>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)  // two CTAs of 512 threads per SM
    k_tile_scatter(const uint64_t *__restrict__ ev, uint64_t *__restrict__ ev2, uint64_t ev2_cap,
                   const unsigned long long *begin, const unsigned long long *counts, TileAux aux,
                   int parts, uint64_t unit, int tpr, uint32_t *status, uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  constexpr int C = BLOCK * kBatch;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *s_ev = reinterpret_cast<uint64_t *>(smem);  // C, in tile order
  uint64_t *s_stage = s_ev + C;                          // C + 2 (STAGED): the next chunk
  uint32_t *s_tile = reinterpret_cast<uint32_t *>(s_stage + (STAGED ? C + 2 : 0));  // C
  uint32_t *s_hist = s_tile + C;   // tpr: chunk counts
  uint32_t *s_off = s_hist + tpr;  // tpr: chunk prefix
  uint32_t *s_fit = s_off + tpr;   // tpr: events of the run that fit the bucket
  uint32_t *s_at = s_fit + tpr;    // tpr: their place, relative to the region's first bucket
  uint32_t *s_ovf = s_at + tpr;    // tpr: the rest's place in the overflow area (~0: none)
  __shared__ uint32_t s_warp[BLOCK / 32];
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_failed;
  const int tid = threadIdx.x;
  const int per = (tpr + BLOCK - 1) / BLOCK;  // bins per thread in the prefix
  const int j0 = min(tpr, tid * per), j1 = min(tpr, j0 + per);
  // the overflow area holds (event, region) pairs
  const uint64_t over_base = aux.region_base[parts];
  const uint64_t over_cap = ev2_cap > over_base ? (ev2_cap - over_base) / 2 : 0ull;
  uint64_t *over = ev2 + over_base;
  if (STAGED && tid == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_failed = 0u;
  }
  TileChunk c;
  bool have = tile_chunk_first(blockIdx.x, unit_region(aux.unit_base, parts, blockIdx.x), C,
                               begin, counts, aux, parts, unit, c);
  __syncthreads();
  if (STAGED && have && tid == 0) stage_chunk(s_stage, ev, c.x, c.y, &s_bar);
  uint32_t parity = 0;
  while (have) {
    const uint32_t cap = aux.tile_cap[c.p];
    uint32_t *fill = aux.fill + aux.region_tile0[c.p];
    uint64_t *out = ev2 + aux.region_base[c.p];
    const uint64_t ns = aux.region_nslots[c.p];
    const uint64_t first_tile = aux.region_first[c.p] >> kTileLog2;
    // (the previous chunk's write-out reads no s_hist: no barrier before this)
    for (int j = tid; j < tpr; j += BLOCK) s_hist[j] = 0u;
    __syncthreads();
    uint64_t e[kBatch];
    if constexpr (STAGED) {
      const bool ok = mbar_wait(&s_bar, parity);
      parity ^= 1u;
      if (!ok) s_failed = 1u;
      const uint64_t x0 = c.x & ~1ull, y1 = c.y & ~1ull;
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        const uint64_t i = c.x + (uint64_t)r * BLOCK + tid;
        e[r] = ok && i < c.y ? (i < y1 ? s_stage[i - x0] : __ldcs(ev + i)) : kEmpty;
      }
    } else {
      load_batch<BLOCK>(ev, c.x, c.y, e);
    }
    uint32_t where[kBatch];  // tile << 16 | rank (rank < C <= 65536)
#pragma unroll
    for (int r = 0; r < kBatch; ++r) {
      if (e[r] != kEmpty) {
        const uint32_t t = tile_in_region(e[r], ns, first_tile);
        where[r] = (t << 16) | atomicAdd(&s_hist[t], 1u);
      }
    }
    __syncthreads();  // (the stage is read: it may take the next chunk)
    TileChunk nx = c;
    bool have_next;
    if (c.y < c.b) {
      nx.x = c.y;
      nx.y = min(nx.x + (uint64_t)C, c.b);
      have_next = true;
    } else {
      have_next = tile_chunk_first(c.u + gridDim.x, c.p, C, begin, counts, aux, parts, unit, nx);
    }
    if constexpr (STAGED) {
      if (s_failed) {  // a copy never landed: report it, let the direct insert do the call
        if (tid == 0) {
          set_sticky(status, DBG_ERR_TIMEOUT);
          atomicExch(use_binned, 0u);
          mbar_wait(&s_bar, parity ^ 1u);  // one more bounded chance for the copy to land
        }
        return;
      }
      if (have_next && tid == 0) stage_chunk(s_stage, ev, nx.x, nx.y, &s_bar);
    }
    // each run takes its place in its bucket; the atomics are issued first,
    // so that their round trips overlap the prefix below
    uint32_t got[kMaxBinsPerThread];
#pragma unroll
    for (int q = 0; q < kMaxBinsPerThread; ++q) {
      const int j = j0 + q;
      const uint32_t h = j < j1 ? s_hist[j] : 0u;
      got[q] = h ? atomicAdd(&fill[j], h) : 0u;
    }
    // exclusive prefix of the chunk's tile counts
    uint32_t local = 0;
    for (int j = j0; j < j1; ++j) local += s_hist[j];
    uint32_t chunk_total;
    uint32_t run = cta_exclusive_prefix<BLOCK>(local, s_warp, chunk_total);
#pragma unroll
    for (int q = 0; q < kMaxBinsPerThread; ++q) {
      const int j = j0 + q;
      if (j >= j1) break;
      const uint32_t h = s_hist[j];
      s_off[j] = run;
      run += h;
      if (h) {
        const uint32_t at = got[q];
        const uint32_t fit = at >= cap ? 0u : min(h, cap - at);
        s_fit[j] = fit;
        s_at[j] = (uint32_t)((uint64_t)j * cap + at);
        if (fit < h) {
          const unsigned long long o = atomicAdd(aux.overflow, (unsigned long long)(h - fit));
          if (o + (h - fit) > over_cap) {  // the area is full: the direct insert takes over
            atomicExch(use_binned, 0u);
            s_ovf[j] = ~0u;
          } else {
            s_ovf[j] = (uint32_t)o;
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kBatch; ++r) {
      if (e[r] != kEmpty) {
        const uint32_t t = where[r] >> 16;
        const uint32_t i = s_off[t] + (where[r] & 0xFFFFu);
        s_ev[i] = e[r];
        s_tile[i] = t;
      }
    }
    __syncthreads();
    const uint32_t n = (uint32_t)(c.y - c.x);
    for (uint32_t i = tid; i < n; i += BLOCK) {
      const uint32_t t = s_tile[i];
      const uint32_t r = i - s_off[t];
      const uint32_t fit = s_fit[t];
      if (r < fit) {
        out[(uint64_t)s_at[t] + r] = s_ev[i];
      } else {
        const uint32_t o = s_ovf[t];
        if (o != ~0u) {
          uint64_t *rec = over + 2 * ((uint64_t)o + (r - fit));
          rec[0] = s_ev[i];
          rec[1] = (uint64_t)c.p;
        }
      }
    }
    c = nx;
    have = have_next;
  }
}

// Slot fingerprints of the tile in shared memory: one byte per slot, 0 for an
// empty slot, else the low byte of the key's hash (1..255; the home slot
// comes from the high bits).  A probe step reads four slots' bytes at once
// and looks for the event's byte or 0 with two zero-byte tests; only such a
// candidate's key is read.  A warp then runs as long as its longest probe in
// steps of four slots instead of one.
constexpr int kFpBytes = kTileSlots + 16;  // (the last step reads one word past the tile)

__device__ __forceinline__ uint32_t slot_fp(uint64_t h) {
  const uint32_t f = (uint32_t)h & 0xFFu;
  return f ? f : 1u;
}

// 0x80 in every byte of x that is zero, and possibly in bytes above a zero
// byte (a borrow), never below the lowest zero byte.
__device__ __forceinline__ uint32_t zero_bytes(uint32_t x) {
  return (x - 0x01010101u) & ~x & 0x80808080u;
}

// The tile in shared memory.  AosTile: the table's own 32-byte slots (a tile
// brought in from the table by a bulk copy).  SoaTile (fresh tables, built
// from EMPTY): the keys in one array and the counters label-major.  With
// 32-byte slots every slot's key falls on one of four bank pairs, so a warp's
// random slots conflict (41 % of the apply's shared-memory wavefronts were
// conflicts); in the SoA tile the keys spread over 16 bank pairs and each
// label's counters over all 32 banks.  The copy-out writes 32-byte slots.
struct AosTile {
  Slot *st;
  __device__ unsigned long long *key(int sl) const { return &st[sl].key; }
  __device__ uint32_t *counter(int sl, uint32_t label) const { return &st[sl].cnt[label]; }
};
struct SoaTile {
  unsigned long long *keys;  // [kTileSlots]
  uint32_t *counts;          // [4][kTileSlots]
  __device__ unsigned long long *key(int sl) const { return &keys[sl]; }
  __device__ uint32_t *counter(int sl, uint32_t label) const {
    return &counts[label * (uint32_t)kTileSlots + (uint32_t)sl];
  }
};
constexpr size_t kSoaTileBytes = (size_t)kTileSlots * (8 + 16);

// One event against the tile in shared memory: found or claimed and counted,
// failed (max_probes inside the tile), or deferred (the probe left the tile).
// Slots are examined in probe order exactly as one at a time would: the first
// slot from home that holds the key or is empty decides.
template <class Tile>
__device__ __forceinline__ void tile_event(uint64_t e, const Tile &tile, uint8_t *fp, uint64_t first,
                                           int len, uint64_t n_slots, uint32_t max_probes,
                                           uint32_t *status, SpillRecord *spill,
                                           uint64_t spill_cap, unsigned long long *spill_count,
                                           int p, uint64_t *ev,
                                           const unsigned long long *begin,
                                           unsigned long long *deferred_n) {
  const unsigned long long key = e >> 3;
  const uint64_t h = key_hash(key);
  const int home = (int)(__umul64hi(h, n_slots) - first);  // = home_slot(key) - first
  const uint32_t f = slot_fp(h), f4 = f * 0x01010101u;
  // the key can only sit in [home, limit): max_probes slots, or up to the tile's end
  const bool capped = max_probes <= (uint32_t)(len - home);
  const int limit = capped ? home + (int)max_probes : len;
  const uint32_t *fp32 = reinterpret_cast<const uint32_t *>(fp);
  int q = home;
  while (q < limit) {
    const uint32_t w = __funnelshift_r(fp32[q >> 2], fp32[(q >> 2) + 1], 8 * (q & 3));
    uint32_t cand = zero_bytes(w ^ f4) | zero_bytes(w);
    if (limit - q < 4) cand &= (1u << (8 * (limit - q))) - 1u;
    if (cand == 0u) {
      q += 4;
      continue;
    }
    const int i = (__ffs(cand) >> 3) - 1;  // the first candidate's byte
    const int sl = q + i;
    // one shared-memory CAS for every candidate: it claims an empty slot and
    // returns an occupied slot's key, so found, claimed and another key take
    // one path (measured faster than a load for the byte matches and a CAS
    // for the empty bytes, whose paths diverge)
    const unsigned long long prev = atomicCAS(tile.key(sl), kEmpty, key);
    if (prev == kEmpty) fp[sl] = (uint8_t)f;
    const bool found = prev == kEmpty || prev == key;
    if (found) {
      if (e & 4ull) atomicAdd(tile.counter(sl, (uint32_t)(e & 3ull)), 1u);
      return;
    }
    q = sl + 1;  // another key (claimed meanwhile, or a byte collision): on to the next
  }
  if (capped)  // max_probes slots inside the tile: as the direct insert
    spill_or_fail(spill, spill_cap, spill_count, status, key, (e & 4ull) != 0,
                  (uint32_t)(e & 3ull));
  else
    ev[begin[p] + atomicAdd(&deferred_n[p], 1ull)] = e;  // left the tile: later, globally
}

// tile_region[t] = the region of every tile t (one CTA per region).
__global__ void k_tile_map(TileAux aux, int parts, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  const int p = blockIdx.x;
  if (p >= parts) return;
  const uint32_t t0 = aux.region_tile0[p], t1 = aux.region_tile0[p + 1];
  for (uint32_t t = t0 + threadIdx.x; t < t1; t += blockDim.x) aux.tile_region[t] = (uint16_t)p;
}

// Persistent CTAs take tiles: a bulk copy brings the tile into shared memory
// while the threads load their first events; the events are applied there;
// a bulk copy writes the tile back while the CTA moves to its next tile.
// Tiles are numbered compactly over the chain's regions; a tile's region
// gives its table (the item's descriptor), its first slot and its bucket.
// An event whose probe leaves its tile is listed in its region's part of the
// first event buffer (which the split has consumed, and which holds at least
// as many places as the region has events) for the global pass.
//
// FRESH: the tables are being rebuilt from empty (dbg_build_reads,
// dbg_build_batch), so their contents are not read at all: every tile starts
// in shared memory as EMPTY slots with zero counters and fingerprints, and
// every tile -- with events or without -- is written back.  That one write
// is the tables' reset: the separate emptying pass (a full write of every
// table) disappears.  Each thread copies out and then re-initialises the
// same 16-byte words of the tile, so the next tile needs no extra barrier.
__device__ __forceinline__ void empty_soa_tile(const SoaTile &tile, uint32_t *fp32) {
  for (int i = threadIdx.x; i < kTileSlots; i += blockDim.x) tile.keys[i] = kEmpty;
  for (int i = threadIdx.x; i < 4 * kTileSlots; i += blockDim.x) tile.counts[i] = 0u;
  for (int i = threadIdx.x; i < kFpBytes / 4; i += blockDim.x) fp32[i] = 0u;
}

template <int BLOCK, bool FRESH, int N>
__global__ void __launch_bounds__(BLOCK, 1536 / BLOCK)  // three CTAs of 512 threads per SM
    k_tile_apply(const __grid_constant__ ItemPack<N> pk, const uint64_t *__restrict__ ev2,
                 uint64_t *ev, const unsigned long long *begin, TileAux aux, int parts,
                 int tpr_log2, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  extern __shared__ __align__(16) unsigned char smem[];  // (bulk copies need 16 bytes)
  // !FRESH: kTileSlots slots (AoS); FRESH: keys and label-major counters (SoA)
  Slot *st = reinterpret_cast<Slot *>(smem);
  const AosTile aos{st};
  const SoaTile soa{reinterpret_cast<unsigned long long *>(smem),
                    reinterpret_cast<uint32_t *>(smem + (size_t)kTileSlots * 8)};
  uint8_t *fp = smem + (FRESH ? kSoaTileBytes : (size_t)kTileSlots * sizeof(Slot));  // kFpBytes
  uint32_t *fp32 = reinterpret_cast<uint32_t *>(fp);
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_stop, s_failed;
  // a rebuild counts its vertices: every slot of a fresh tile that holds a key
  // (a non-zero fingerprint) was claimed in that tile (the deferred pass
  // counts the rest); the count goes to the item's built counts whenever the
  // item changes, and at the end
  uint32_t *cur_status = N == 1 ? pk.d[0].status : nullptr;
  uint32_t claimed = 0;
  auto flush_claims = [&]() {
    const uint32_t w = __reduce_add_sync(kFull, claimed);
    if ((threadIdx.x & 31) == 0 && w && cur_status != nullptr)
      atomicAdd(small_built(cur_status), (unsigned long long)w);
    claimed = 0;
  };
  if constexpr (FRESH) {
    empty_soa_tile(soa, fp32);
  } else if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_failed = 0u;
  }
  __syncthreads();
  uint32_t parity = 0;
  const uint64_t n_tiles = aux.region_tile0[parts];
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // the tile's region, table and bucket: its events up to the bucket's
    // size (the rest overflowed).  One table's regions all hold 2^tpr_log2
    // tiles but the last; a chain of many tables looks its tiles up.
    const int p = N == 1 ? (int)(t >> tpr_log2) : (int)aux.tile_region[t];
    const uint64_t j = t - aux.region_tile0[p];
    // (one table: its fields stay kernel parameters, not registers)
    const ItemDesc &it = pk.d[N == 1 ? 0 : aux.region_item[p]];
    const uint32_t cap = aux.tile_cap[p];
    const uint64_t a = aux.region_base[p] + j * cap;
    const uint64_t b = a + min(aux.fill[t], cap);
    const uint64_t first = aux.region_first[p] + (j << kTileLog2);
    const uint64_t n_slots = it.n_slots;
    Slot *table = it.table;
    uint32_t *status = it.status;
    const int len = (int)min((uint64_t)kTileSlots, n_slots - first);
    uint64_t e[kBatch];
    if constexpr (FRESH) {
      if (N > 1 && status != cur_status) {  // (the same for the whole CTA)
        flush_claims();
        cur_status = status;
      }
      uint4 *dst = reinterpret_cast<uint4 *>(table + first);
      if (a == b) {  // no event: the tile is written as it starts, EMPTY
        const uint4 head = make_uint4(0xffffffffu, 0xffffffffu, 0u, 0u);
        const uint4 tail = make_uint4(0u, 0u, 0u, 0u);
        for (int i = threadIdx.x; i < 2 * len; i += BLOCK) __stcs(dst + i, (i & 1) ? tail : head);
        continue;  // (shared memory untouched: still the EMPTY tile)
      }
      if (threadIdx.x == 0) s_stop = ld_volatile_u32(status);
      load_batch<BLOCK>(ev2, a, b, e);
      __syncthreads();  // s_stop; the tile's EMPTY words (the previous copy-out re-made them)
    } else {
      // no event: the tile stays as it is (the same decision for the whole CTA)
      if (a == b) continue;
      const uint32_t bytes = (uint32_t)len * (uint32_t)sizeof(Slot);
      if (threadIdx.x == 0) {
        s_stop = ld_volatile_u32(status);
        bulk_wait_read_all();  // the previous tile's write-back has left `st`
        mbar_expect_tx(&s_bar, bytes);
        bulk_load(st, table + first, bytes, &s_bar);
      }
      load_batch<BLOCK>(ev2, a, b, e);  // overlaps the tile's arrival
      const bool landed = mbar_wait(&s_bar, parity);
      if (!landed) atomicExch(&s_failed, 1u);
      parity ^= 1u;
      if (landed) {  // the tile's fingerprints, four slots per word
        for (int wi = threadIdx.x; wi < kFpBytes / 4; wi += BLOCK) {
          uint32_t v = 0u;
#pragma unroll
          for (int jj = 0; jj < 4; ++jj) {
            const int sl = 4 * wi + jj;
            const unsigned long long k = sl < len ? st[sl].key : kEmpty;
            if (k != kEmpty) v |= slot_fp(key_hash(k)) << (8 * jj);
          }
          fp32[wi] = v;
        }
      }
      __syncthreads();
      if (s_failed) {
        // The copy did not land within the bound.  Before the CTA leaves, the
        // copy must no longer target its shared memory: wait for the same
        // phase again with the same bound (a bulk copy from valid memory
        // lands, so a second bound is only a guard), and for the write-backs
        // this thread issued.
        if (threadIdx.x == 0) {
          set_sticky(status, DBG_ERR_TIMEOUT);
          mbar_wait(&s_bar, parity ^ 1u);
          bulk_wait_all();
        }
        __syncthreads();
        return;
      }
    }
    if (s_stop == 0u) {  // an earlier error stops the insert, as in the direct kernel
      for (uint64_t base = a;;) {
#pragma unroll
        for (int r = 0; r < kBatch; ++r) {
          if (e[r] == kEmpty) continue;
          if constexpr (FRESH)
            tile_event(e[r], soa, fp, first, len, n_slots, it.max_probes, status, it.spill,
                       it.spill_cap, it.spill_count, p, ev, begin, aux.deferred_n);
          else
            tile_event(e[r], aos, fp, first, len, n_slots, it.max_probes, status, it.spill,
                       it.spill_cap, it.spill_count, p, ev, begin, aux.deferred_n);
        }
        base += (uint64_t)BLOCK * kBatch;
        if (base >= b) break;
        load_batch<BLOCK>(ev2, base, b, e);
      }
    }
    __syncthreads();
    if constexpr (FRESH) {
      // copy the tile out as 32-byte slots (written even after an earlier
      // error: the table is at least empty there), 16 bytes a thread: an even
      // word is (key, cnt[0], cnt[1]), an odd one (cnt[2], cnt[3], pad).  Each
      // thread re-makes the EMPTY words it has just read.  (Slots past `len`
      // take no event: they stay EMPTY.)
      uint4 *dst = reinterpret_cast<uint4 *>(table + first);
      const uint32_t K = (uint32_t)kTileSlots;
      for (int i = threadIdx.x; i < 2 * len; i += BLOCK) {
        const uint32_t sl = (uint32_t)i >> 1;
        uint4 v;
        if ((i & 1) == 0) {
          const unsigned long long k = soa.keys[sl];
          v = make_uint4((uint32_t)k, (uint32_t)(k >> 32), soa.counts[sl], soa.counts[K + sl]);
          soa.keys[sl] = kEmpty;
          soa.counts[sl] = 0u;
          soa.counts[K + sl] = 0u;
        } else {
          v = make_uint4(soa.counts[2 * K + sl], soa.counts[3 * K + sl], 0u, 0u);
          soa.counts[2 * K + sl] = 0u;
          soa.counts[3 * K + sl] = 0u;
        }
        __stcs(dst + i, v);
      }
      for (int i = threadIdx.x; i < kFpBytes / 4; i += BLOCK) {
        const uint32_t w = fp32[i];  // four fingerprints: non-zero for a key
        claimed += (uint32_t)__popc((((w & 0x7F7F7F7Fu) + 0x7F7F7F7Fu) | w) & 0x80808080u);
        fp32[i] = 0u;
      }
      // (the next tile's barrier orders these writes before its events)
    } else if (threadIdx.x == 0 && s_stop == 0u) {
      fence_proxy_async_smem();  // the CTA's shared-memory updates, before the bulk read
      bulk_store(table + first, st, (uint32_t)len * (uint32_t)sizeof(Slot));
      bulk_commit();
    }
  }
  if constexpr (FRESH) flush_claims();
  if (!FRESH && threadIdx.x == 0) bulk_wait_all();
}

// One event, from its home slot, with the global find-or-claim (its tile is
// final by now).
// Returns 1 when the event claimed a new slot (a new vertex), else 0.
__device__ __forceinline__ uint32_t global_event(uint64_t e, const ItemDesc &it) {
  const unsigned long long key = e >> 3;
  uint64_t s;
  bool claimed = false;
  if (find_or_claim(it.table, it.n_slots, it.max_probes, key, s, &claimed)) {
    if (e & 4ull) atomicAdd(&it.table[s].cnt[e & 3ull], 1u);
  } else {
    spill_or_fail(it.spill, it.spill_cap, it.spill_count, it.status, key, (e & 4ull) != 0,
                  (uint32_t)(e & 3ull));
  }
  return claimed ? 1u : 0u;
}

// The events that left their tile (each region's list), then those of the
// overflow area ((event, region) pairs), from their home slots.  New
// vertices are added to their graph's built counts (meaningful only on a
// rebuild, which zeroed them): one atomic per warp and region, and for the
// overflow area one per warp of a single table, else one per new vertex.
template <int N>
__global__ void k_tile_deferred(const __grid_constant__ ItemPack<N> pk,
                                const uint64_t *__restrict__ ev,
                                const uint64_t *__restrict__ ev2, const unsigned long long *begin,
                                TileAux aux, int parts, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  for (int p = blockIdx.x; p < parts; p += gridDim.x) {
    const uint64_t n = aux.deferred_n[p];
    if (n == 0) continue;
    if (threadIdx.x == 0) atomicAdd(aux.deferred, (unsigned long long)n);
    const ItemDesc &it = pk.d[aux.region_item[p]];
    const uint64_t *list = ev + begin[p];
    uint32_t claimed = 0;
    for (uint64_t i = threadIdx.x; i < n; i += blockDim.x) claimed += global_event(list[i], it);
    claimed = __reduce_add_sync(kFull, claimed);
    if ((threadIdx.x & 31) == 0 && claimed)
      atomicAdd(small_built(it.status), (unsigned long long)claimed);
  }
  const uint64_t no = *aux.overflow;  // (all of it written: the flag is still set)
  const uint64_t *over = ev2 + aux.region_base[parts];
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint32_t claimed = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < no; i += stride) {
    const ItemDesc &it = pk.d[aux.region_item[over[2 * i + 1]]];
    const uint32_t c = global_event(over[2 * i], it);
    if (N == 1)
      claimed += c;
    else if (c)
      atomicAdd(small_built(it.status), 1ull);
  }
  if (N == 1) {
    claimed = __reduce_add_sync(kFull, claimed);
    if ((threadIdx.x & 31) == 0 && claimed)
      atomicAdd(small_built(pk.d[0].status), (unsigned long long)claimed);
  }
}

// Empty every item's table (grid: x strides over the slots, y = item); with
// a gate, nothing happens when *gate != 0 (the binned kernels did the work: a
// rebuild's tiled apply has emptied the tables itself); without one, the
// items' sticky statuses and spill counts are cleared too.
template <int N>
__global__ void k_tables_init(const __grid_constant__ ItemPack<N> pk, const uint32_t *gate) {
  if (gate != nullptr && ld_volatile_u32(gate) != 0u) return;
  const int i = blockIdx.y;
  if (i >= pk.n_items) return;
  if (gate == nullptr && blockIdx.x == 0 && threadIdx.x == 0) {
    *pk.d[i].status = 0u;
    *pk.d[i].spill_count = 0ull;
  }
  // (the gated form runs when a binned chain gave its call to the direct
  // insert, which counts nothing)
  if (gate != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *small_counted(pk.d[i].status) = 0u;
  uint4 *t = reinterpret_cast<uint4 *>(pk.d[i].table);
  const uint64_t n_vec = 2 * pk.d[i].n_slots;
  const uint4 head = make_uint4(0xffffffffu, 0xffffffffu, 0u, 0u);
  const uint4 tail = make_uint4(0u, 0u, 0u, 0u);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n_vec; v += stride)
    t[v] = (v & 1) ? tail : head;
}

int ceil_log2(uint64_t x) {
  int r = 0;
  while ((1ull << r) < x) ++r;
  return r;
}

}  // namespace

BinGeometry bin_geometry(uint64_t n_slots, int region_log2) {
  BinGeometry g;
  g.shift = std::max(region_log2 > 0 ? region_log2 : kBinMinShift,
                     ceil_log2((n_slots + kMaxParts - 1) / kMaxParts));
  g.parts = (int)((n_slots + (1ull << g.shift) - 1) >> g.shift);
  return g;
}

// meta area layout (see dbg_binned.cuh)
struct MetaView {
  unsigned long long *begin;   // kBinMaxParts + 1
  unsigned long long *counts;  // kBinMaxParts
  unsigned long long *cursor;  // kBinMaxParts
  unsigned long long *ctr;     // 4 counters; ctr[3] holds the use-binned flag
  uint32_t *flag;
  unsigned long long *apply_ctr;  // kBinApplyCounters
  unsigned long long *totals;  // kBatchItems: vertex positions per item
  unsigned long long *edges;   // kBatchItems: edges (k-mers) per item
  uint32_t *hist;              // kBinSlices * kBinMaxParts
};

MetaView meta_view(const BinScratch &sc) {
  MetaView v;
  unsigned long long *b = sc.meta;
  v.begin = b;
  v.counts = v.begin + kBinMaxParts + 1;
  v.cursor = v.counts + kBinMaxParts;
  v.ctr = v.cursor + kBinMaxParts;
  v.flag = reinterpret_cast<uint32_t *>(v.ctr + 3);
  v.apply_ctr = v.ctr + 4;
  v.totals = v.apply_ctr + (size_t)kBinMaxParts * kBinApplyCounters;
  v.edges = v.totals + kBatchItems;
  v.hist = reinterpret_cast<uint32_t *>(v.edges + kBatchItems);
  return v;
}

void free_bin_scratch(BinScratch &sc) {
  cudaFree(sc.ev);
  cudaFree(sc.ev2);
  cudaFree(sc.aux);
  cudaFree(sc.meta);
  if (sc.done) cudaEventDestroy(sc.done);
  sc = BinScratch{};
}

namespace {

uint64_t default_events(uint64_t n_slots) {
  return std::max(kBinMinEvents, kBinEventsPerSlot * n_slots + n_slots / 4);
}

// The meta area, the ordering event and an event buffer of exactly `events`
// events (a buffer of another size is replaced, after the device is idle:
// earlier calls may still read it).
int ensure_events(BinScratch &sc, uint64_t events) {
  if (!sc.meta) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, kBinMetaBytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binned meta)");
    sc.meta = static_cast<unsigned long long *>(p);
  }
  if (!sc.done) DBG_CK(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming));
  if (sc.cap != events) {
    DBG_CK(cudaDeviceSynchronize());
    cudaFree(sc.ev);
    cudaFree(sc.ev2);  // the tiled apply's buffer follows the event capacity
    sc.ev = sc.ev2 = nullptr;
    sc.cap = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, events * sizeof(uint64_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binned events)");
    sc.ev = static_cast<uint64_t *>(p);
    sc.cap = events;
  }
  return DBG_OK;
}

}  // namespace

uint64_t bin_events_wanted(dbg_handle h) {
  return h->bin_want ? h->bin_want : default_events(h->n_slots);
}

int ensure_bin_scratch(dbg_handle h, uint64_t events) {
  return ensure_events(h->bin, events ? events : bin_events_wanted(h));
}

namespace {

uint64_t tile_unit(int tpr) { return std::max<uint64_t>(16384, 64ull * (uint64_t)tpr); }

// Events the second buffer holds: the first buffer's capacity plus room for
// the tile buckets' margins (the first buffer's regions have their own);
// bucket positions are 32-bit.
uint64_t ev2_capacity(uint64_t bin_cap) {
  return std::min<uint64_t>(bin_cap + bin_cap / 8 + (1ull << 20), 0xFFFFFFFFull);
}
// The largest first buffer whose second one stays within 32-bit positions.
constexpr uint64_t kMaxChainEvents = 3800000000ull;

// Layout of the tiled apply's aux buffer for `parts` regions and `tiles`
// tiles (compact numbering).
struct TileAuxLayout {
  size_t unit_base, region_base, tile_cap, fill, item, first, nslots, tile0, map, deferred_n,
      counters, total;
};

TileAuxLayout tile_aux_layout(int parts, uint64_t tiles) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t P = (size_t)parts;
  TileAuxLayout l;
  l.unit_base = 0;
  l.region_base = al(l.unit_base + (P + 1) * 8);
  l.tile_cap = al(l.region_base + (P + 1) * 8);
  l.fill = al(l.tile_cap + P * 4);
  l.item = al(l.fill + (size_t)tiles * 4);
  l.first = al(l.item + P * 4);
  l.nslots = al(l.first + P * 8);
  l.tile0 = al(l.nslots + P * 8);
  l.map = al(l.tile0 + (P + 1) * 4);
  l.deferred_n = al(l.map + (size_t)tiles * 2);
  l.counters = al(l.deferred_n + P * 8);
  l.total = al(l.counters + 16);
  return l;
}

TileAux tile_aux(const BinScratch &sc, int parts, uint64_t tiles) {
  const TileAuxLayout l = tile_aux_layout(parts, tiles);
  char *b = static_cast<char *>(sc.aux);
  TileAux a;
  a.unit_base = reinterpret_cast<unsigned long long *>(b + l.unit_base);
  a.region_base = reinterpret_cast<unsigned long long *>(b + l.region_base);
  a.tile_cap = reinterpret_cast<uint32_t *>(b + l.tile_cap);
  a.fill = reinterpret_cast<uint32_t *>(b + l.fill);
  a.region_item = reinterpret_cast<uint32_t *>(b + l.item);
  a.region_first = reinterpret_cast<unsigned long long *>(b + l.first);
  a.region_nslots = reinterpret_cast<unsigned long long *>(b + l.nslots);
  a.region_tile0 = reinterpret_cast<uint32_t *>(b + l.tile0);
  a.tile_region = reinterpret_cast<uint16_t *>(b + l.map);
  a.deferred_n = reinterpret_cast<unsigned long long *>(b + l.deferred_n);
  a.overflow = reinterpret_cast<unsigned long long *>(b + l.counters);
  a.deferred = a.overflow + 1;
  return a;
}

// The second event buffer and the aux buffer of the tiled apply; false if
// they cannot be had -- out of memory, or inside a stream capture that began
// before they existed.
bool ensure_tile_scratch(BinScratch &sc, int parts, uint64_t tiles, bool capturing) {
  const size_t need = tile_aux_layout(parts, tiles).total;
  if (sc.ev2 && sc.aux && sc.aux_bytes >= need) return true;
  if (capturing) return false;
  if (cudaDeviceSynchronize() != cudaSuccess) return false;  // earlier calls may use them
  if (!sc.ev2) {
    void *p = nullptr;
    if (cudaMalloc(&p, ev2_capacity(sc.cap) * sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();  // clear the allocation failure
      return false;
    }
    sc.ev2 = static_cast<uint64_t *>(p);
  }
  if (sc.aux_bytes < need) {
    cudaFree(sc.aux);
    sc.aux = nullptr;
    sc.aux_bytes = 0;
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    sc.aux = p;
    sc.aux_bytes = need;
  }
  return true;
}

// Tiles (compact numbering) of a table of n_slots slots cut into regions of
// 2^shift slots.
uint64_t table_tiles(uint64_t n_slots, int shift) {
  const uint64_t R = 1ull << shift;
  const uint64_t full = n_slots >> shift, rest = n_slots & (R - 1);
  return full * (R >> kTileLog2) + ((rest + kTileSlots - 1) >> kTileLog2);
}

int regions_of(uint64_t n_slots, int shift) {
  return (int)((n_slots + (1ull << shift) - 1) >> shift);
}

}  // namespace

template <int B, int U, int M>
int launch_apply(dbg_handle h, const MetaView &mv, const BinGeometry &geo, int sms,
                 const dbg_tuning &t, cudaStream_t s) {
  int per_sm = 0;
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_apply<B, U, M>, B, 0));
  if (t.apply_ctas > 0) per_sm = std::min(per_sm, t.apply_ctas);
  const int grid = std::max(1, per_sm) * sms;
  // regions per launch (default: all of them in one launch)
  const int group = t.apply_group > 0 ? std::min(t.apply_group, geo.parts) : geo.parts;
  const int n_groups = (geo.parts + group - 1) / group;
  DBG_CK(cudaMemsetAsync(mv.apply_ctr, 0,
                         (size_t)n_groups * t.apply_counters * sizeof(unsigned long long), s));
  for (int gi = 0; gi < n_groups; ++gi) {
    const int p0 = gi * group, p1 = std::min(geo.parts, p0 + group);
    k_bin_apply<B, U, M><<<grid, B, 0, s>>>(
        h->bin.ev, mv.begin, p0, p1, mv.flag, h->table, h->n_slots, h->max_probes, h->d_status,
        mv.apply_ctr + (size_t)gi * t.apply_counters, t.apply_counters, h->d_spill, h->spill_cap,
        h->d_spill_count);
  }
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

template <int B, int U>
int launch_apply_m(dbg_handle h, const MetaView &mv, const BinGeometry &geo, int sms,
                   const dbg_tuning &t, cudaStream_t s) {
  switch (t.apply_chunk) {
    case 4: return launch_apply<B, U, 4>(h, mv, geo, sms, t, s);
    case 16: return launch_apply<B, U, 16>(h, mv, geo, sms, t, s);
    default: return launch_apply<B, U, 8>(h, mv, geo, sms, t, s);
  }
}

template <int BT, bool STAGED>
int launch_tile_scatter(const BinScratch &sc, const MetaView &mv, const TileAux &aux, int parts,
                        uint64_t unit, int tpr, int sms, cudaStream_t s, uint32_t *status) {
  if (tpr > kMaxBinsPerThread * BT) return DBG_ERR_INVALID_ARG;  // (the launch sizes BT by tpr)
  const size_t smem = tile_scatter_smem<BT, STAGED>(tpr);
  // (set even below 48 KB: the kernel's static shared memory counts too)
  DBG_CK(cudaFuncSetAttribute(k_tile_scatter<BT, STAGED>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_scatter<BT, STAGED>, BT,
                                                       smem));
  k_tile_scatter<BT, STAGED><<<std::max(1, per_sm) * sms, BT, smem, s>>>(
      sc.ev, sc.ev2, ev2_capacity(sc.cap), mv.begin, mv.counts, aux, parts, unit, tpr, status,
      mv.flag);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

namespace {

// Records the kernel timer's marks of a single-table call (no-op for batches).
struct Marks {
  dbg_handle h = nullptr;
  int call = -1;
  void operator()(int m, cudaStream_t s) const {
    if (h) timer_mark(h, call, m, s);
  }
};

// One tiled chain over items[0..n) (N >= n): their tables are cut into
// regions of 2^shift slots (`parts` of them, `tiles` tiles), item i's first
// region is items[i].region0, and items[i].tile_begin numbers the walk's
// tiles of kScatterTileReads reads.  `direct` holds the same items numbered
// for the direct kernel (`direct_tiles` tiles), which does the call instead
// when the events do not fit the scratch.  The scratch's event buffer, second
// buffer and aux area must exist.  `status` receives a timeout of the split.
template <int N>
int tiled_chain(BinScratch &sc, const ItemDesc *items, int n, int shift, int parts,
                uint64_t tiles, uint64_t walk_tiles, const ItemDesc *direct,
                uint64_t direct_tiles, const dbg_tuning &tuning, int sms, cudaStream_t s,
                bool fresh, const Marks &mark, const InputParts *input = nullptr) {
  const int scatter_reads = scatter_tile_reads(tuning);
  const MetaView mv = meta_view(sc);
  const int tpr = 1 << (shift - kTileLog2);
  const TileAux aux = tile_aux(sc, parts, tiles);
  ItemPack<N> pk{};
  pk.n_items = n;
  pk.total_tiles = walk_tiles;
  for (int i = 0; i < n; ++i) pk.d[i] = items[i];
  const uint64_t slices = std::min<uint64_t>(walk_tiles, kBinSlices);
  DBG_CK(cudaMemsetAsync(mv.ctr, 0, 4 * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.counts, 0, parts * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.totals, 0, n * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.edges, 0, n * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(aux.fill, 0, tiles * sizeof(uint32_t), s));
  sc.counters = aux.overflow;
  mark(1, s);
  // bucket sizing: positions per item, then buckets and the region table
  {
    // four CTAs per SM over the items, and more when the largest read set
    // would take over 32 reads a thread (items of very uneven size: the
    // largest one sets the time; the others' extra CTAs return at once), at
    // most 16384 CTAs in all
    uint64_t max_reads = 0;
    for (int i = 0; i < n; ++i) max_reads = std::max<uint64_t>(max_reads, items[i].n_reads);
    const uint64_t want = std::min<uint64_t>((max_reads + 256 * 32 - 1) / (256 * 32),
                                             (uint64_t)std::max(1, 16384 / n));
    const int gx = (int)std::max<uint64_t>(want, (uint64_t)std::max(1, (sms * 4 + n - 1) / n));
    k_bin_totals<N><<<dim3(gx, n), 256, 0, s>>>(pk, mv.totals, mv.edges, fresh ? 1 : 0);
    DBG_CK(cudaGetLastError());
    k_bin_buckets<N><<<1, 1024, 0, s>>>(pk, mv.totals, mv.edges, fresh ? 1 : 0, shift, parts,
                                        mv.begin, mv.cursor, sc.cap, mv.ctr, mv.flag, aux);
    DBG_CK(cudaGetLastError());
    if (N > 1) {
      k_tile_map<<<parts, 256, 0, s>>>(aux, parts, mv.flag);
      DBG_CK(cudaGetLastError());
    }
  }
  mark(3, s);
  {
    // 512 threads: flushes of 4096 events, so that a region's run in a flush
    // is long enough to fill whole sectors (shorter runs cost the L2 a
    // read-modify-write of partly written sectors)
    constexpr int BS = 512;
    const size_t smem = scatter_smem<BS>(scatter_reads, parts);
    DBG_CK(cudaFuncSetAttribute(k_bin_scatter<BS, N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<BS, N>, BS, smem));
    // one launch over every read tile, or (input arriving in parts) one per
    // part, each after its part's copy: tiles [cut[c], cut[c + 1]) hold reads
    // that have all arrived (a tile split by a cut goes to the later part)
    const int n_parts = (N == 1 && input != nullptr && input->n > 1) ? input->n : 1;
    for (int c = 0; c < n_parts; ++c) {
      uint64_t a = 0, b = walk_tiles;
      if (n_parts > 1) {
        a = c == 0 ? 0 : std::min<uint64_t>(walk_tiles, input->read_cut[c] / (uint64_t)scatter_reads);
        b = c + 1 == n_parts
                ? walk_tiles
                : std::min<uint64_t>(walk_tiles, input->read_cut[c + 1] / (uint64_t)scatter_reads);
        DBG_CK(cudaStreamWaitEvent(s, input->ready[c], 0));
        if (b <= a) continue;
        if (c > 0) DBG_CK(cudaMemsetAsync(mv.ctr + 1, 0, sizeof(unsigned long long), s));
      }
      const uint64_t sl = std::min<uint64_t>(b - a, kBinSlices);
      const int grid = (int)std::max<uint64_t>(
          1, std::min<uint64_t>(sl, (uint64_t)std::max(1, per_sm) * sms));
      k_bin_scatter<BS, N><<<grid, BS, smem, s>>>(pk, scatter_reads, shift, parts, a, b, sl,
                                                  mv.hist, mv.cursor, sc.ev, sc.cap, mv.ctr,
                                                  mv.flag, mv.begin + 1);
      DBG_CK(cudaGetLastError());
    }
  }
  const uint64_t unit = tile_unit(tpr);
  mark(4, s);
  k_tile_units<<<1, 1024, 0, s>>>(mv.counts, mv.begin, mv.cursor, parts, unit,
                                  ev2_capacity(sc.cap), aux, mv.flag);
  DBG_CK(cudaGetLastError());
  // chunks of 8 events per thread: larger blocks for more tiles per region,
  // so that each tile's run in a chunk stays several events long (a timeout of
  // the staged copies is recorded in the first item's status)
  // (tuning.split_threads overrides the choice when it has at most four bins
  // a thread)
  int bt = tpr <= 256 ? 256 : tpr <= 1024 ? 512 : 1024;
  if (tuning.split_threads > 0 && tpr <= kMaxBinsPerThread * tuning.split_threads)
    bt = tuning.split_threads;
  if (bt == 256) {
    DBG_TRY((launch_tile_scatter<256, true>(sc, mv, aux, parts, unit, tpr, sms, s,
                                            items[0].status)));
  } else if (bt == 512) {  // (1024 tiles: two bins per thread; measured faster than 1024 threads)
    DBG_TRY((launch_tile_scatter<512, true>(sc, mv, aux, parts, unit, tpr, sms, s,
                                            items[0].status)));
  } else {
    DBG_TRY((launch_tile_scatter<1024, false>(sc, mv, aux, parts, unit, tpr, sms, s,
                                              items[0].status)));
  }
  mark(5, s);
  {
    // 512 threads: three such CTAs (66 KB of shared memory each, or 50 KB
    // for a rebuild's split tile, with the fingerprints; registers allow
    // three) fill an SM with 48 warps, enough to hide the dependent hash and
    // probe latencies
    constexpr int BA = 512;
    const size_t smem = (fresh ? kSoaTileBytes : (size_t)kTileSlots * sizeof(Slot)) + kFpBytes;
    auto kern = fresh ? k_tile_apply<BA, true, N> : k_tile_apply<BA, false, N>;
    DBG_CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BA, smem));
    const uint64_t grid = std::max<uint64_t>(
        1, std::min<uint64_t>(tiles, (uint64_t)std::max(1, per_sm) * sms));
    kern<<<(int)grid, BA, smem, s>>>(pk, sc.ev2, sc.ev, mv.begin, aux, parts, shift - kTileLog2,
                                     mv.flag);
    DBG_CK(cudaGetLastError());
  }
  mark(6, s);
  k_tile_deferred<N><<<sms * 4, 256, 0, s>>>(pk, sc.ev, sc.ev2, mv.begin, aux, parts, mv.flag);
  DBG_CK(cudaGetLastError());
  // the direct insert runs only if the events did not fit the buffer (then no
  // binned kernel touched the tables: a rebuild from empty empties them first)
  mark(7, s);
  if (fresh) {
    ItemPack<N> ip{};
    ip.n_items = n;
    for (int i = 0; i < n; ++i) ip.d[i] = items[i];
    k_tables_init<N><<<dim3(std::max(1, sms * 8 / n), n), 256, 0, s>>>(ip, mv.flag);
    DBG_CK(cudaGetLastError());
  }
  const int st = launch_insert(direct, n, direct_tiles, tuning, sms, s, mv.flag);
  if (st != DBG_OK) return st;
  mark(8, s);
  return DBG_OK;
}

}  // namespace

int wait_input(const InputParts *input, cudaStream_t s) {
  if (input != nullptr)
    for (int c = 0; c < input->n; ++c) DBG_CK(cudaStreamWaitEvent(s, input->ready[c], 0));
  return DBG_OK;
}

int launch_binned(dbg_handle h, const ItemDesc &it, uint64_t tiles, const dbg_tuning &tuning,
                  cudaStream_t s, int call, bool fresh, const InputParts *input) {
  constexpr int B = 256;
  const dbg_tuning t = resolve_tuning(tuning);
  // the tiled apply re-partitions each region by tile, so its first pass can
  // use coarser regions (fewer of them: a cheaper scatter); measured best at
  // 1024 tiles per region on the 100 Mbp workload (2^20-slot regions:
  // 47.6 ms a build, 2^21: 46.9 ms, 2^22: 51.3 ms)
  const bool want_tiled = t.apply_mode != 1 && h->bin.cap < kMaxChainEvents;
  const BinGeometry geo =
      bin_geometry(h->n_slots, t.region_log2 > 0 ? t.region_log2 : (want_tiled ? kTiledShift : 0));
  const int sms = std::max(1, h->sm_count);
  const Marks mark{h, call};

  // binned calls on one handle share its scratch: order them.  Inside a
  // stream capture the captured calls are ordered by the stream itself, and
  // an event recorded outside the capture may not be waited on.
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  DBG_CK(cudaStreamIsCapturing(s, &capture));
  const bool capturing = capture != cudaStreamCaptureStatusNone;
  if (!capturing) DBG_CK(cudaStreamWaitEvent(s, h->bin.done, 0));
  const int tpr = 1 << std::max(0, geo.shift - kTileLog2);
  const uint64_t n_tiles = table_tiles(h->n_slots, std::max(geo.shift, kTileLog2));
  // (bucket positions are kept in 32 bits: the event buffer must stay below
  // 2^32 events)
  const bool tiled = want_tiled && geo.shift >= kTileLog2 && tpr <= kMaxTilesPerRegion &&
                     ensure_tile_scratch(h->bin, geo.parts, n_tiles, capturing);
  h->bin.counters = nullptr;
  if (tiled) {
    ItemDesc walk = it;  // the scatter's read tiles (larger than the direct kernel's)
    walk.tile_begin = 0;
    walk.region0 = 0;
    const uint64_t sr = (uint64_t)scatter_tile_reads(tuning);
    const uint64_t walk_tiles = (it.n_reads + sr - 1) / sr;
    ItemDesc direct = it;
    direct.tile_begin = 0;
    DBG_TRY(tiled_chain<1>(h->bin, &walk, 1, geo.shift, geo.parts, n_tiles, walk_tiles, &direct,
                           tiles, tuning, sms, s, fresh, mark, input));
    h->built_counts = fresh;  // a rebuild counted its vertices and edges (unless it fell back)
    if (!capturing) DBG_CK(cudaEventRecord(h->bin.done, s));
    return DBG_OK;
  }

  // the streaming apply: an exact count pass and its scan, the scatter into
  // gap-free region ranges, then the apply (a rebuild empties the table
  // first: this apply reads it)
  DBG_TRY(wait_input(input, s));
  if (fresh) DBG_TRY(launch_table_init(h->table, h->n_slots, s));
  const MetaView mv = meta_view(h->bin);
  const int tile_reads = std::min(t.tile_reads, B);
  const uint64_t walk_tiles = (it.n_reads + (uint64_t)tile_reads - 1) / (uint64_t)tile_reads;
  const uint64_t slices = std::min<uint64_t>(walk_tiles, kBinSlices);
  ItemPack<1> pk{};
  pk.n_items = 1;
  pk.total_tiles = walk_tiles;
  pk.d[0] = it;
  pk.d[0].region0 = 0;
  DBG_CK(cudaMemsetAsync(mv.ctr, 0, 4 * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.counts, 0, geo.parts * sizeof(unsigned long long), s));
  mark(1, s);
  {
    const size_t smem = tile_smem_bytes(tile_reads) + (size_t)geo.parts * 4;
    if (smem > 48 * 1024)
      DBG_CK(cudaFuncSetAttribute(k_bin_count<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_count<B>, B, smem));
    const int grid = (int)std::min<uint64_t>(slices, (uint64_t)std::max(1, per_sm) * sms);
    k_bin_count<B><<<grid, B, smem, s>>>(pk, tile_reads, geo.shift, geo.parts, slices, mv.hist,
                                         mv.counts, mv.ctr);
    DBG_CK(cudaGetLastError());
    mark(2, s);
    k_bin_scan<<<1, 1024, 0, s>>>(mv.counts, geo.parts, mv.begin, mv.cursor, h->bin.cap, mv.ctr,
                                  mv.flag);
    DBG_CK(cudaGetLastError());
  }
  mark(3, s);
  {
    constexpr int BS = 512;
    const size_t smem = scatter_smem<BS>(tile_reads, geo.parts);
    DBG_CK(cudaFuncSetAttribute(k_bin_scatter<BS, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<BS, 1>, BS, smem));
    const int grid = (int)std::min<uint64_t>(slices, (uint64_t)std::max(1, per_sm) * sms);
    k_bin_scatter<BS, 1><<<grid, BS, smem, s>>>(pk, tile_reads, geo.shift, geo.parts, 0,
                                                walk_tiles, slices, mv.hist, mv.cursor, h->bin.ev,
                                                h->bin.cap, mv.ctr, mv.flag, nullptr);
    DBG_CK(cudaGetLastError());
  }
  mark(5, s);
  switch (t.apply_unroll) {
    case 2: DBG_TRY((launch_apply_m<B, 2>(h, mv, geo, sms, t, s))); break;
    case 8: DBG_TRY((launch_apply_m<B, 8>(h, mv, geo, sms, t, s))); break;
    default: DBG_TRY((launch_apply_m<B, 4>(h, mv, geo, sms, t, s))); break;
  }
  // the direct insert runs only if the events did not fit the buffer
  mark(7, s);
  const int st = launch_insert(&it, 1, tiles, tuning, h->sm_count, s, mv.flag);
  if (st != DBG_OK) return st;
  mark(8, s);
  if (!capturing) DBG_CK(cudaEventRecord(h->bin.done, s));
  return DBG_OK;
}

// ---------------------------------------------------------------------------
// batches: chains of many tables, with the library's own scratch
// ---------------------------------------------------------------------------

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_batch_mu;
BinScratch g_batch[kMaxDevices];

}  // namespace

int launch_tables_init(const ItemDesc *items, int n, int sm_count, cudaStream_t s) {
  if (n <= 0) return DBG_OK;
  if (n > kBatchItems) return DBG_ERR_INVALID_ARG;
  ItemPack<kBatchItems> ip{};
  ip.n_items = n;
  for (int i = 0; i < n; ++i) ip.d[i] = items[i];
  k_tables_init<kBatchItems><<<dim3(std::max(1, std::max(1, sm_count) * 8 / n), n), 256, 0, s>>>(
      ip, nullptr);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

int launch_binned_batch(const ItemDesc *items, const uint64_t *want, int n,
                        const dbg_tuning &tuning, int sm_count, cudaStream_t s, bool fresh) {
  if (n <= 0) return DBG_OK;
  const dbg_tuning t = resolve_tuning(tuning);
  const int shift = t.region_log2 > 0 ? std::max(t.region_log2, kTileLog2) : kTiledShift;
  const int sms = std::max(1, sm_count);
  int dev = 0;
  DBG_CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return DBG_ERR_INVALID_ARG;
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  DBG_CK(cudaStreamIsCapturing(s, &capture));
  const bool capturing = capture != cudaStreamCaptureStatusNone;

  // cut the items into chains: at most kBatchItems items, kBinMaxParts
  // regions and kMaxChainEvents events each
  struct Chain {
    int i0, i1, parts;
    uint64_t tiles, events;
  };
  std::vector<Chain> chains;
  for (int i = 0; i < n;) {
    Chain c{i, i, 0, 0, 0};
    while (c.i1 < n) {
      const int r = regions_of(items[c.i1].n_slots, shift);
      const uint64_t ev = want[c.i1];
      if (c.i1 > c.i0 && (c.i1 - c.i0 == kBatchItems || c.parts + r > kBinMaxParts ||
                          c.events + ev > kMaxChainEvents))
        break;
      c.parts += r;
      c.tiles += table_tiles(items[c.i1].n_slots, shift);
      c.events += ev;
      ++c.i1;
    }
    if (c.parts > kBinMaxParts) return DBG_ERR_INVALID_ARG;  // one table of too many regions
    chains.push_back(c);
    i = c.i1;
  }
  uint64_t need_events = 0, need_tiles = 0;
  int need_parts = 0;
  for (const Chain &c : chains) {
    need_events = std::max(need_events, std::min(c.events, kMaxChainEvents));
    need_tiles = std::max(need_tiles, c.tiles);
    need_parts = std::max(need_parts, c.parts);
  }

  std::lock_guard<std::mutex> lock(g_batch_mu);
  BinScratch &sc = g_batch[dev];
  bool ready = sc.meta && sc.done && sc.cap >= need_events &&
               ensure_tile_scratch(sc, need_parts, need_tiles, true);
  if (!ready && !capturing) {
    DBG_TRY(ensure_events(sc, std::max(need_events, sc.cap)));
    ready = ensure_tile_scratch(sc, need_parts, need_tiles, false);
  }
  if (!capturing) DBG_CK(cudaStreamWaitEvent(s, sc.done, 0));
  const uint64_t sr = (uint64_t)scatter_tile_reads(tuning);
  for (const Chain &c : chains) {
    const int m = c.i1 - c.i0;
    std::vector<ItemDesc> walk(items + c.i0, items + c.i1), direct(items + c.i0, items + c.i1);
    uint64_t walk_tiles = 0, direct_tiles = 0;
    int region0 = 0;
    for (int i = 0; i < m; ++i) {
      walk[i].tile_begin = walk_tiles;
      walk[i].region0 = region0;
      walk_tiles += (walk[i].n_reads + sr - 1) / sr;
      region0 += regions_of(walk[i].n_slots, shift);
      direct[i].tile_begin = direct_tiles;
      direct_tiles += (direct[i].n_reads + (uint64_t)t.tile_reads - 1) / (uint64_t)t.tile_reads;
    }
    if (!ready) {  // no scratch inside this capture: the direct insert does it
      if (fresh) DBG_TRY(launch_tables_init(direct.data(), m, sms, s));
      DBG_TRY(launch_insert(direct.data(), m, direct_tiles, tuning, sms, s));
      continue;
    }
    DBG_TRY(tiled_chain<kBatchItems>(sc, walk.data(), m, shift, c.parts, c.tiles, walk_tiles,
                                     direct.data(), direct_tiles, tuning, sms, s, fresh, Marks{}));
  }
  if (!capturing) DBG_CK(cudaEventRecord(sc.done, s));
  return DBG_OK;
}

uint64_t batch_scratch_bytes(int dev) {
  if (dev < 0 || dev >= kMaxDevices) return 0;
  std::lock_guard<std::mutex> lock(g_batch_mu);
  const BinScratch &sc = g_batch[dev];
  uint64_t b = sc.aux_bytes + (sc.meta ? kBinMetaBytes : 0);
  if (sc.ev) b += sc.cap * sizeof(uint64_t);
  if (sc.ev2) b += ev2_capacity(sc.cap) * sizeof(uint64_t);
  return b;
}

int release_batch_scratch() {
  std::lock_guard<std::mutex> lock(g_batch_mu);
  int prev = 0;
  DBG_CK(cudaGetDevice(&prev));
  for (int d = 0; d < kMaxDevices; ++d) {
    if (!g_batch[d].meta && !g_batch[d].ev) continue;
    DBG_CK(cudaSetDevice(d));
    DBG_CK(cudaDeviceSynchronize());
    free_bin_scratch(g_batch[d]);
  }
  DBG_CK(cudaSetDevice(prev));
  return DBG_OK;
}

int binned_counters(dbg_handle h, uint64_t *out) {
  out[0] = out[1] = out[2] = 0;
  if (!h->bin.meta) return DBG_OK;  // no binned call yet
  DBG_CK(cudaDeviceSynchronize());
  uint32_t flag = 0;
  DBG_CK(cudaMemcpy(&flag, meta_view(h->bin).flag, sizeof(flag), cudaMemcpyDeviceToHost));
  out[0] = flag != 0u;
  if (flag && h->bin.counters) {
    unsigned long long c[2] = {0ull, 0ull};  // overflow, deferred
    DBG_CK(cudaMemcpy(c, h->bin.counters, sizeof(c), cudaMemcpyDeviceToHost));
    out[1] = c[1];
    out[2] = c[0];
  }
  return DBG_OK;
}

}  // namespace dbg
