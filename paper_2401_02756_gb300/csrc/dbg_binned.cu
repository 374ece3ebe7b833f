// The binned insert: the same table updates as the direct insert kernel
// (find or claim the prefix and suffix vertices, count the label -- Alg. 2-4
// and the addRightVertex prose), issued in an order that keeps them on chip.
//
// A random 32-byte slot of a table far larger than L2 costs a DRAM round trip
// that fetches a whole line, which caps the direct insert near the
// random-sector rate of HBM.  So for a large table the insert runs as:
//   buckets -- the read set's vertex positions, and for every table region
//              (2^shift slots, at most 2048 regions) a bucket of its
//              expected events plus six standard deviations;
//   scatter -- walk the read tiles, compute every vertex's key and home
//              slot, and write one 8-byte event per vertex,
//              (key << 3) | (edge << 2) | label, into its region's bucket
//              (block-local counting sort in shared memory; each flush's
//              run appended to its bucket with one atomic);
//   split   -- per region, order the events by 2048-slot table tile
//              (units of events: histogram, offsets, counting-sorted scatter);
//   apply   -- one CTA per tile: a bulk copy brings the tile into shared
//              memory, the tile's events are applied there with
//              shared-memory CAS and add, a bulk copy writes it back;
//   deferred -- the few events whose probe left their tile, from their home
//              slot, with the global find-or-claim.
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

#include "dbg_binned.cuh"
#include "dbg_tiles.cuh"
#include "dbg_tma.cuh"

namespace dbg {
namespace {

constexpr int kMaxParts = kBinMaxParts;
constexpr int kRun = 8;             // consecutive vertex positions per thread (rolled keys)

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

// *total = vertex positions of the read set, sum of max(0, len - k + 2).
__global__ void k_bin_total(const uint64_t *offsets, uint64_t n_reads, int k,
                            unsigned long long *total) {
  unsigned long long v = 0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n_reads; r += stride) {
    const uint64_t a = offsets[r], b = offsets[r + 1];
    const uint64_t len = b > a ? b - a : 0;
    v += len >= (uint64_t)k ? len - k + 2 : 0;
  }
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(kFull, v, d);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(total, v);
}

// One CTA of 1024 threads (two regions each): bucket p starts at begin[p]
// and holds its expected events plus the margin; cursor[p] = begin[p];
// the flag says whether all buckets fit the buffer; resets the scatter's
// slice counter.
__global__ void __launch_bounds__(1024)
    k_bin_buckets(const unsigned long long *total, uint64_t n_slots, int shift, int parts,
                  unsigned long long *begin, unsigned long long *cursor, uint64_t cap,
                  unsigned long long *ctr, uint32_t *use_binned) {
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double E = (double)*total;
  auto bucket = [&](int p) -> unsigned long long {
    if (p >= parts) return 0ull;
    const uint64_t first = (uint64_t)p << shift;
    const uint64_t slots = min((uint64_t)1 << shift, n_slots - first);
    const double expected = E * (double)slots / (double)n_slots;
    return (unsigned long long)ceil(expected * 1.03 + 16.0 * sqrt(expected) + 256.0);
  };
  const int p0 = 2 * tid;
  const unsigned long long ca = bucket(p0), cb = bucket(p0 + 1);
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
    const unsigned long long all = s_warp[31];
    begin[parts] = all;
    *use_binned = all <= cap ? 1u : 0u;
    ctr[1] = 0;
  }
}

// --- K1d --------------------------------------------------------------------

// A round of the tile walk gives every thread kRun events; each keeps them in
// registers with its region and its rank in the region (a shared-memory
// atomic), then the round is flushed: an exclusive prefix of the region
// counts places the events in region order in shared memory (counting
// sort), and they are written out as runs.  A run's position = the slice's
// run start in the region (reserved at the start of the slice, as long as
// the count pass measured) + the events of the region already placed.
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
      const uint32_t p = (uint32_t)(home_slot(key, c.n_slots) >> shift);
      ev[sub] = make_event(key, edge, label);
      where[sub] = (p << 16) | atomicAdd(&hist[p], 1u);
    } else {
      where[sub] = ~0u;
    }
  }
  __device__ void round_end() {
    __shared__ unsigned long long s_w[BLOCK / 32];
    __shared__ uint32_t s_total;
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // exclusive prefix over the regions; each region's place in the output
    const int per = (parts + BLOCK - 1) / BLOCK;
    const int p0 = min(parts, tid * per), p1 = min(parts, p0 + per);
    uint32_t local = 0;
    for (int p = p0; p < p1; ++p) local += hist[p];
    uint32_t incl = local;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(kFull, incl, d);
      if (lane >= d) incl += o;
    }
    if (lane == 31) s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = lane < BLOCK / 32 ? s_w[lane] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long o = __shfl_up_sync(kFull, w, d);
        if (lane >= d) w += o;
      }
      if (lane < BLOCK / 32) s_w[lane] = w;
      if (lane == BLOCK / 32 - 1) s_total = (uint32_t)w;
    }
    __syncthreads();
    uint32_t run = incl - local + (warp > 0 ? (uint32_t)s_w[warp - 1] : 0u);
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
    const uint32_t total = s_total;
    for (uint32_t j = tid; j < total; j += BLOCK) {
      const unsigned long long g = gbase[spid[j]];
      const unsigned long long at = g + j;
      if (g != ~0ull && at < cap) __stcs(out + at, sorted[j]);
    }
    // no barrier here: the next round only touches hist (already cleared)
    // before its first barrier, and sorted / spid / gbase / s_total after it
  }
};

template <int BLOCK>
constexpr size_t scatter_smem(int tile_reads, int parts) {
  return tile_smem_bytes(tile_reads) + (size_t)BLOCK * kRun * (8 + 2) +
         (size_t)parts * (4 + 4 + 8 + 8) + 64;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 1024 / BLOCK)
    k_bin_scatter(const __grid_constant__ ItemPack<1> pk, int tile_reads, int shift, int parts,
                  uint64_t slices, const uint32_t *hist, unsigned long long *cursor, uint64_t *out,
                  uint64_t cap, unsigned long long *ctr, uint32_t *use_binned,
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
  const uint64_t T = pk.total_tiles;
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
    for_each_vertex<BLOCK, 1, kRun>(pk, tile_reads, smem, vis, sl * T / slices,
                                    (sl + 1) * T / slices, 1);
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
// partition pass (split) orders each region's events by tile:
//   units   -- each region's events are cut into units of `unit` events;
//   count   -- per unit, a histogram over the region's tiles;
//   offsets -- per region, the tiles' event ranges and each unit's place in
//              every tile's range (a prefix over the units);
//   scatter -- per unit, every event to its tile's range (second buffer).
// A probe sequence that runs off the end of its tile (keys homed near the
// end of a full stretch of slots) cannot continue there: the next tile
// belongs to another CTA.  Such events are deferred to a list (in the first
// event buffer, which the split pass has consumed) and applied afterwards,
// from their home slot, with the direct insert's global find-or-claim; the
// tile they would have spilled into is final by then.  A probe that reaches
// max_probes inside its tile fails (or spills) exactly as in the direct
// insert, so every key stays within max_probes of its home slot.

constexpr int kTileLog2 = 11;
constexpr int kTileSlots = 1 << kTileLog2;  // 2048 slots = 64 KB of shared memory
constexpr int kMaxTilesPerRegion = 4096;    // beyond this the streaming apply is used
constexpr int kTiledShift = 20;             // automatic regions of the tiled path: 512 tiles

constexpr int kBatch = 8;  // events each thread loads before it uses them (memory parallelism)

struct TileAux {
  uint32_t *unit_hist;            // [units][tpr] counts, then starts (relative to the region's)
  unsigned long long *tile_begin; // [parts * tpr + 1]
  unsigned long long *unit_base;  // [parts + 1]
  unsigned long long *deferred;   // [1] events left for the global pass
};

// unit_base[p] = units of regions < p, each region cut into ceil(count/unit) units.
// (bucketed: a region's events are those its bucket received, cursor - begin;
// they become the region counts the later passes read)
__global__ void __launch_bounds__(1024)
    k_tile_units(unsigned long long *counts, const unsigned long long *begin,
                 const unsigned long long *cursor, int bucketed, int parts, uint64_t unit,
                 unsigned long long *unit_base, unsigned long long *deferred,
                 const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  __shared__ unsigned long long s_warp[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p0 = 2 * tid;
  if (bucketed) {
    if (p0 < parts) counts[p0] = cursor[p0] - begin[p0];
    if (p0 + 1 < parts) counts[p0 + 1] = cursor[p0 + 1] - begin[p0 + 1];
  }
  const unsigned long long ua = p0 < parts ? (counts[p0] + unit - 1) / unit : 0ull;
  const unsigned long long ub = p0 + 1 < parts ? (counts[p0 + 1] + unit - 1) / unit : 0ull;
  const unsigned long long local = ua + ub;
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
  if (p0 < parts) unit_base[p0] = b;
  if (p0 + 1 < parts) unit_base[p0 + 1] = b + ua;
  if (tid == 0) {
    unit_base[parts] = s_warp[31];
    *deferred = 0ull;
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

__device__ __forceinline__ uint32_t tile_in_region(uint64_t ev, uint64_t n_slots, int shift,
                                                   int p) {
  const uint64_t home = home_slot(ev >> 3, n_slots);
  return (uint32_t)((home >> kTileLog2) - ((uint64_t)p << (shift - kTileLog2)));
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

// Per unit: histogram of its events over the region's tiles.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_tile_count(const uint64_t *__restrict__ ev, const unsigned long long *begin,
                 const unsigned long long *counts, TileAux aux, int parts, uint64_t unit,
                 int shift, int tpr, uint64_t n_slots, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  extern __shared__ uint32_t s_hist[];  // tpr
  const uint64_t n_units = aux.unit_base[parts];
  for (uint64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int p = unit_region(aux.unit_base, parts, u);
    const uint64_t a = begin[p] + (u - aux.unit_base[p]) * unit;
    const uint64_t b = min(a + unit, (uint64_t)(begin[p] + counts[p]));
    for (int j = threadIdx.x; j < tpr; j += BLOCK) s_hist[j] = 0u;
    __syncthreads();
    for (uint64_t base = a; base < b; base += (uint64_t)BLOCK * kBatch) {
      uint64_t e[kBatch];
      load_batch<BLOCK>(ev, base, b, e);
#pragma unroll
      for (int r = 0; r < kBatch; ++r)
        if (e[r] != kEmpty) atomicAdd(&s_hist[tile_in_region(e[r], n_slots, shift, p)], 1u);
    }
    __syncthreads();
    uint32_t *h = aux.unit_hist + u * (uint64_t)tpr;
    for (int j = threadIdx.x; j < tpr; j += BLOCK) h[j] = s_hist[j];
    __syncthreads();
  }
}

// Per region (one CTA each): every tile's event range (tile_begin, absolute)
// and, in unit_hist, where each unit's events of each tile start (relative
// to the region's first event).
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_tile_offsets(const unsigned long long *begin, TileAux aux, int parts, int tpr,
                   const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  __shared__ unsigned long long s_warp[BLOCK / 32];
  const int p = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t u0 = aux.unit_base[p], u1 = aux.unit_base[p + 1];
  unsigned long long *tb = aux.tile_begin + (uint64_t)p * tpr;
  // each thread owns `per` consecutive tiles: their totals (kept in tb for now)
  const int per = (tpr + BLOCK - 1) / BLOCK;
  const int j0 = min(tpr, tid * per), j1 = min(tpr, j0 + per);
  unsigned long long local = 0;
  for (int j = j0; j < j1; ++j) {
    unsigned long long total = 0;
    for (uint64_t u = u0; u < u1; ++u) total += aux.unit_hist[u * (uint64_t)tpr + j];
    tb[j] = total;
    local += total;
  }
  unsigned long long incl = local;
  for (int d = 1; d < 32; d <<= 1) {
    const unsigned long long o = __shfl_up_sync(kFull, incl, d);
    if (lane >= d) incl += o;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    unsigned long long w = lane < BLOCK / 32 ? s_warp[lane] : 0ull;
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(kFull, w, d);
      if (lane >= d) w += o;
    }
    if (lane < BLOCK / 32) s_warp[lane] = w;
  }
  __syncthreads();
  // tile j's range starts after the events of the region's tiles < j
  unsigned long long rel = incl - local + (warp > 0 ? s_warp[warp - 1] : 0ull);
  for (int j = j0; j < j1; ++j) {
    const unsigned long long total = tb[j];
    tb[j] = begin[p] + rel;
    unsigned long long at = rel;
    for (uint64_t u = u0; u < u1; ++u) {
      uint32_t *c = aux.unit_hist + u * (uint64_t)tpr + j;
      const uint32_t n = *c;
      *c = (uint32_t)at;
      at += n;
    }
    rel += total;
  }
  if (p == parts - 1 && tid == 0) aux.tile_begin[(uint64_t)parts * tpr] = begin[parts];
}

// Per unit: every event to its tile's range in the second buffer.  Each
// chunk of BLOCK * kBatch events is counting-sorted by tile in shared memory
// first, so that every tile's run of the chunk is written by consecutive
// threads to consecutive addresses (coalesced stores instead of one scattered
// 8-byte store per event).
template <int BLOCK>
constexpr size_t tile_scatter_smem(int tpr) {
  return (size_t)BLOCK * kBatch * (8 + 4) + (size_t)tpr * 12;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_tile_scatter(const uint64_t *__restrict__ ev, uint64_t *__restrict__ ev2,
                   const unsigned long long *begin, const unsigned long long *counts, TileAux aux,
                   int parts, uint64_t unit, int shift, int tpr, uint64_t n_slots,
                   const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  constexpr int C = BLOCK * kBatch;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *s_ev = reinterpret_cast<uint64_t *>(smem);       // C, in tile order
  uint32_t *s_tile = reinterpret_cast<uint32_t *>(s_ev + C);  // C: tile of s_ev[i]
  uint32_t *s_at = s_tile + C;                                // tpr: next start (unit cursor)
  uint32_t *s_hist = s_at + tpr;                              // tpr: chunk counts
  uint32_t *s_off = s_hist + tpr;                             // tpr: chunk prefix
  __shared__ uint32_t s_warp[BLOCK / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (tpr + BLOCK - 1) / BLOCK;  // bins per thread in the prefix
  const int j0 = min(tpr, tid * per), j1 = min(tpr, j0 + per);
  const uint64_t n_units = aux.unit_base[parts];
  for (uint64_t u = blockIdx.x; u < n_units; u += gridDim.x) {
    const int p = unit_region(aux.unit_base, parts, u);
    const uint64_t a = begin[p] + (u - aux.unit_base[p]) * unit;
    const uint64_t b = min(a + unit, (uint64_t)(begin[p] + counts[p]));
    const uint32_t *h = aux.unit_hist + u * (uint64_t)tpr;
    for (int j = tid; j < tpr; j += BLOCK) s_at[j] = h[j];
    uint64_t *out = ev2 + begin[p];
    for (uint64_t base = a; base < b; base += C) {
      for (int j = tid; j < tpr; j += BLOCK) s_hist[j] = 0u;
      __syncthreads();
      uint64_t e[kBatch];
      uint32_t where[kBatch];  // tile << 16 | rank (rank < C <= 65536)
      load_batch<BLOCK>(ev, base, b, e);
#pragma unroll
      for (int r = 0; r < kBatch; ++r) {
        if (e[r] != kEmpty) {
          const uint32_t t = tile_in_region(e[r], n_slots, shift, p);
          where[r] = (t << 16) | atomicAdd(&s_hist[t], 1u);
        }
      }
      __syncthreads();
      // exclusive prefix of the chunk's tile counts
      uint32_t local = 0;
      for (int j = j0; j < j1; ++j) local += s_hist[j];
      uint32_t incl = local;
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, incl, d);
        if (lane >= d) incl += o;
      }
      if (lane == 31) s_warp[warp] = incl;
      __syncthreads();
      if (warp == 0) {
        uint32_t w = lane < BLOCK / 32 ? s_warp[lane] : 0u;
        for (int d = 1; d < 32; d <<= 1) {
          const uint32_t o = __shfl_up_sync(kFull, w, d);
          if (lane >= d) w += o;
        }
        if (lane < BLOCK / 32) s_warp[lane] = w;
      }
      __syncthreads();
      uint32_t run = incl - local + (warp > 0 ? s_warp[warp - 1] : 0u);
      for (int j = j0; j < j1; ++j) {
        s_off[j] = run;
        run += s_hist[j];
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
      const uint32_t n = (uint32_t)min((uint64_t)C, b - base);
      for (uint32_t i = tid; i < n; i += BLOCK) {
        const uint32_t t = s_tile[i];
        out[s_at[t] + (i - s_off[t])] = s_ev[i];
      }
      __syncthreads();
      for (int j = tid; j < tpr; j += BLOCK) s_at[j] += s_hist[j];
      __syncthreads();
    }
  }
}

// One event against the tile in shared memory: found or claimed and counted,
// failed (max_probes inside the tile), or deferred (the probe left the tile).
__device__ __forceinline__ void tile_event(uint64_t e, Slot *st, uint64_t first, int len,
                                           uint64_t n_slots, uint32_t max_probes,
                                           uint32_t *status, SpillRecord *spill,
                                           uint64_t spill_cap, unsigned long long *spill_count,
                                           uint64_t *deferred_ev, unsigned long long *deferred) {
  const unsigned long long key = e >> 3;
  int q = (int)(home_slot(key, n_slots) - first);
  uint32_t probes = 0;
  while (q < len) {
    const unsigned long long cur = st[q].key;
    bool found = cur == key;
    if (!found && cur == kEmpty) {
      const unsigned long long prev = atomicCAS(&st[q].key, kEmpty, key);
      found = prev == kEmpty || prev == key;
    }
    if (found) {
      if (e & 4ull) atomicAdd(&st[q].cnt[e & 3ull], 1u);
      return;
    }
    if (++probes >= max_probes) {
      spill_or_fail(spill, spill_cap, spill_count, status, key, (e & 4ull) != 0,
                    (uint32_t)(e & 3ull));
      return;
    }
    ++q;
  }
  deferred_ev[atomicAdd(deferred, 1ull)] = e;  // left the tile: later, globally
}

// Persistent CTAs take tiles: a bulk copy brings the tile into shared memory
// while the threads load their first events; the events are applied there;
// a bulk copy writes the tile back while the CTA moves to its next tile.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_tile_apply(const uint64_t *__restrict__ ev2, uint64_t *deferred_ev, TileAux aux,
                 const unsigned long long *begin, const unsigned long long *counts, int tpr,
                 uint64_t n_tiles, Slot *table, uint64_t n_slots, uint32_t max_probes,
                 uint32_t *status, SpillRecord *spill, uint64_t spill_cap,
                 unsigned long long *spill_count, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  extern __shared__ __align__(128) unsigned char smem[];
  Slot *st = reinterpret_cast<Slot *>(smem);  // kTileSlots slots
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ uint32_t s_stop, s_failed;
  if (threadIdx.x == 0) {
    mbar_init(&s_bar, 1);
    fence_mbar_init();
    s_failed = 0u;
  }
  __syncthreads();
  uint32_t parity = 0;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    // a region's last tile ends with the region's events (buckets may leave gaps)
    const uint64_t p = t / (uint64_t)tpr;
    const uint64_t a = aux.tile_begin[t];
    const uint64_t b = (t + 1) % (uint64_t)tpr == 0 ? (uint64_t)(begin[p] + counts[p])
                                                      : (uint64_t)aux.tile_begin[t + 1];
    const uint64_t first = t << kTileLog2;
    // no event, or a tile past the table's end (never has one): the tile stays
    // as it is (the same decision for the whole CTA)
    if (a == b || first >= n_slots) continue;
    const int len = (int)min((uint64_t)kTileSlots, n_slots - first);
    const uint32_t bytes = (uint32_t)len * (uint32_t)sizeof(Slot);
    if (threadIdx.x == 0) {
      s_stop = ld_volatile_u32(status);
      bulk_wait_read_all();  // the previous tile's write-back has left `st`
      mbar_expect_tx(&s_bar, bytes);
      bulk_load(st, table + first, bytes, &s_bar);
    }
    uint64_t e[kBatch];
    load_batch<BLOCK>(ev2, a, b, e);  // overlaps the tile's arrival
    if (!mbar_wait(&s_bar, parity)) atomicExch(&s_failed, 1u);
    parity ^= 1u;
    __syncthreads();
    if (s_failed) {
      if (threadIdx.x == 0) {
        set_sticky(status, DBG_ERR_TIMEOUT);
        mbar_wait(&s_bar, parity ^ 1u);  // give the copy one more bounded chance to land
        bulk_wait_all();
      }
      return;
    }
    if (s_stop == 0u) {  // an earlier error stops the insert, as in the direct kernel
      for (uint64_t base = a;;) {
#pragma unroll
        for (int r = 0; r < kBatch; ++r)
          if (e[r] != kEmpty)
            tile_event(e[r], st, first, len, n_slots, max_probes, status, spill, spill_cap,
                       spill_count, deferred_ev, aux.deferred);
        base += (uint64_t)BLOCK * kBatch;
        if (base >= b) break;
        load_batch<BLOCK>(ev2, base, b, e);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_stop == 0u) {
      fence_proxy_async_smem();  // the CTA's shared-memory updates, before the bulk read
      bulk_store(table + first, st, bytes);
      bulk_commit();
    }
  }
  if (threadIdx.x == 0) bulk_wait_all();
}

// The deferred events, from their home slots, with the global find-or-claim.
__global__ void k_tile_deferred(const uint64_t *__restrict__ deferred_ev, TileAux aux,
                                Slot *table, uint64_t n_slots, uint32_t max_probes,
                                uint32_t *status, SpillRecord *spill, uint64_t spill_cap,
                                unsigned long long *spill_count, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  const uint64_t n = *aux.deferred;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint64_t e = deferred_ev[i];
    const unsigned long long key = e >> 3;
    uint64_t s;
    if (find_or_claim(table, n_slots, max_probes, key, s)) {
      if (e & 4ull) atomicAdd(&table[s].cnt[e & 3ull], 1u);
    } else {
      spill_or_fail(spill, spill_cap, spill_count, status, key, (e & 4ull) != 0,
                    (uint32_t)(e & 3ull));
    }
  }
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
  uint32_t *hist;              // kBinSlices * kBinMaxParts
};

MetaView meta_view(dbg_handle h) {
  MetaView v;
  unsigned long long *b = h->bin_meta;
  v.begin = b;
  v.counts = v.begin + kBinMaxParts + 1;
  v.cursor = v.counts + kBinMaxParts;
  v.ctr = v.cursor + kBinMaxParts;
  v.flag = reinterpret_cast<uint32_t *>(v.ctr + 3);
  v.apply_ctr = v.ctr + 4;
  v.hist = reinterpret_cast<uint32_t *>(v.apply_ctr + (size_t)kBinMaxParts * kBinApplyCounters);
  return v;
}

int ensure_bin_scratch(dbg_handle h, uint64_t events) {
  if (events == 0)
    events = std::max(kBinMinEvents, kBinEventsPerSlot * h->n_slots + h->n_slots / 4);
  if (!h->bin_meta) {
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, kBinMetaBytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binned meta)");
    h->bin_meta = static_cast<unsigned long long *>(p);
  }
  if (!h->bin_done) {
    DBG_CK(cudaEventCreateWithFlags(&h->bin_done, cudaEventDisableTiming));
  }
  if (h->bin_cap != events) {
    DBG_CK(cudaDeviceSynchronize());  // earlier binned calls may still read the old buffer
    cudaFree(h->bin_ev);
    cudaFree(h->bin_ev2);  // the tiled apply's buffer follows the event capacity
    h->bin_ev = h->bin_ev2 = nullptr;
    h->bin_cap = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, events * sizeof(uint64_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binned events)");
    h->bin_ev = static_cast<uint64_t *>(p);
    h->bin_cap = events;
  }
  return DBG_OK;
}


namespace {

uint64_t tile_unit(int tpr) { return std::max<uint64_t>(16384, 64ull * (uint64_t)tpr); }

// Layout of the tiled apply's aux buffer for a geometry.
struct TileAuxLayout {
  size_t hist, tile_begin, unit_base, deferred, total;
};

TileAuxLayout tile_aux_layout(uint64_t bin_cap, const BinGeometry &geo, int tpr) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const uint64_t max_units = bin_cap / tile_unit(tpr) + (uint64_t)geo.parts;
  TileAuxLayout l;
  l.hist = 0;
  l.tile_begin = al(l.hist + max_units * (uint64_t)tpr * 4);
  l.unit_base = al(l.tile_begin + ((uint64_t)geo.parts * tpr + 1) * 8);
  l.deferred = al(l.unit_base + ((uint64_t)geo.parts + 1) * 8);
  l.total = al(l.deferred + 8);
  return l;
}

TileAux tile_aux(dbg_handle h, const BinGeometry &geo, int tpr) {
  const TileAuxLayout l = tile_aux_layout(h->bin_cap, geo, tpr);
  char *b = static_cast<char *>(h->bin_aux);
  TileAux a;
  a.unit_hist = reinterpret_cast<uint32_t *>(b + l.hist);
  a.tile_begin = reinterpret_cast<unsigned long long *>(b + l.tile_begin);
  a.unit_base = reinterpret_cast<unsigned long long *>(b + l.unit_base);
  a.deferred = reinterpret_cast<unsigned long long *>(b + l.deferred);
  return a;
}

// The second event buffer and the aux buffer of the tiled apply; false (and
// the streaming apply is used) if they cannot be had -- out of memory, or
// inside a stream capture that began before they existed.
bool ensure_tile_scratch(dbg_handle h, const BinGeometry &geo, int tpr, bool capturing) {
  const size_t need = tile_aux_layout(h->bin_cap, geo, tpr).total;
  if (h->bin_ev2 && h->bin_aux && h->bin_aux_bytes >= need) return true;
  if (capturing) return false;
  if (cudaDeviceSynchronize() != cudaSuccess) return false;  // earlier calls may use them
  if (!h->bin_ev2) {
    void *p = nullptr;
    if (cudaMalloc(&p, h->bin_cap * sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();  // clear the allocation failure
      return false;
    }
    h->bin_ev2 = static_cast<uint64_t *>(p);
  }
  if (h->bin_aux_bytes < need) {
    cudaFree(h->bin_aux);
    h->bin_aux = nullptr;
    h->bin_aux_bytes = 0;
    void *p = nullptr;
    if (cudaMalloc(&p, need) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    h->bin_aux = p;
    h->bin_aux_bytes = need;
  }
  return true;
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
        h->bin_ev, mv.begin, p0, p1, mv.flag, h->table, h->n_slots, h->max_probes, h->d_status,
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

template <int BT>
int launch_tile_scatter(dbg_handle h, const MetaView &mv, const TileAux &aux,
                        const BinGeometry &geo, uint64_t unit, int tpr, int sms, cudaStream_t s) {
  const size_t smem = tile_scatter_smem<BT>(tpr);
  // (set even below 48 KB: the kernel's static shared memory counts too)
  DBG_CK(cudaFuncSetAttribute(k_tile_scatter<BT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)smem));
  int per_sm = 0;
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_scatter<BT>, BT, smem));
  k_tile_scatter<BT><<<std::max(1, per_sm) * sms, BT, smem, s>>>(
      h->bin_ev, h->bin_ev2, mv.begin, mv.counts, aux, geo.parts, unit, geo.shift, tpr,
      h->n_slots, mv.flag);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

int launch_binned(dbg_handle h, const ItemDesc &it, uint64_t tiles, const dbg_tuning &tuning,
                  cudaStream_t s, int call) {
  constexpr int B = 256;
  const dbg_tuning t = resolve_tuning(tuning);
  const int tile_reads = std::min(t.tile_reads, B);
  // the tiled apply re-partitions each region by tile, so its first pass can
  // use coarser regions (fewer of them: a cheaper scatter); measured best at
  // 512 tiles per region on the 100 Mbp workload
  const bool want_tiled = t.apply_mode != 1 && h->bin_cap < (1ull << 32);
  const BinGeometry geo =
      bin_geometry(h->n_slots, t.region_log2 > 0 ? t.region_log2 : (want_tiled ? kTiledShift : 0));
  const uint64_t slices = std::min<uint64_t>(tiles, kBinSlices);
  const MetaView mv = meta_view(h);

  ItemPack<1> pk{};
  pk.n_items = 1;
  pk.total_tiles = tiles;
  pk.d[0] = it;
  const int sms = std::max(1, h->sm_count);

  // binned calls on one handle share its scratch: order them.  Inside a
  // stream capture the captured calls are ordered by the stream itself, and
  // an event recorded outside the capture may not be waited on.
  cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
  DBG_CK(cudaStreamIsCapturing(s, &capture));
  const bool capturing = capture != cudaStreamCaptureStatusNone;
  if (!capturing) DBG_CK(cudaStreamWaitEvent(s, h->bin_done, 0));
  const int tpr = 1 << std::max(0, geo.shift - kTileLog2);
  // (unit starts are kept in 32 bits relative to their region: the event
  // buffer must stay below 2^32 events)
  const bool tiled = want_tiled && geo.shift >= kTileLog2 && tpr <= kMaxTilesPerRegion &&
                     ensure_tile_scratch(h, geo, tpr, capturing);
  DBG_CK(cudaMemsetAsync(mv.ctr, 0, 4 * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.counts, 0, geo.parts * sizeof(unsigned long long), s));
  timer_mark(h, call, 1, s);
  if (tiled) {  // buckets instead of the count pass and its scan
    k_bin_total<<<sms * 4, 256, 0, s>>>(it.offsets, it.n_reads, it.k, mv.ctr + 2);
    DBG_CK(cudaGetLastError());
    k_bin_buckets<<<1, 1024, 0, s>>>(mv.ctr + 2, h->n_slots, geo.shift, geo.parts, mv.begin,
                                     mv.cursor, h->bin_cap, mv.ctr, mv.flag);
    DBG_CK(cudaGetLastError());
  } else {
    const size_t smem = tile_smem_bytes(tile_reads) + (size_t)geo.parts * 4;
    if (smem > 48 * 1024)
      DBG_CK(cudaFuncSetAttribute(k_bin_count<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_count<B>, B, smem));
    const int grid = (int)std::min<uint64_t>(slices, (uint64_t)std::max(1, per_sm) * sms);
    k_bin_count<B><<<grid, B, smem, s>>>(pk, tile_reads, geo.shift, geo.parts, slices, mv.hist,
                                         mv.counts, mv.ctr);
    DBG_CK(cudaGetLastError());
    timer_mark(h, call, 2, s);
    k_bin_scan<<<1, 1024, 0, s>>>(mv.counts, geo.parts, mv.begin, mv.cursor, h->bin_cap, mv.ctr,
                                  mv.flag);
    DBG_CK(cudaGetLastError());
  }
  timer_mark(h, call, 3, s);
  {
    // 512 threads: flushes of 4096 events, so that a region's run in a flush
    // is long enough to fill whole sectors (shorter runs cost the L2 a
    // read-modify-write of partly written sectors)
    constexpr int BS = 512;
    const size_t smem = scatter_smem<BS>(tile_reads, geo.parts);
    DBG_CK(cudaFuncSetAttribute(k_bin_scatter<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<BS>, BS, smem));
    const int grid = (int)std::min<uint64_t>(slices, (uint64_t)std::max(1, per_sm) * sms);
    k_bin_scatter<BS><<<grid, BS, smem, s>>>(pk, tile_reads, geo.shift, geo.parts, slices, mv.hist,
                                             mv.cursor, h->bin_ev, h->bin_cap, mv.ctr, mv.flag,
                                             tiled ? mv.begin + 1 : nullptr);
    DBG_CK(cudaGetLastError());
  }
  if (tiled) {
    const uint64_t unit = tile_unit(tpr);
    const TileAux aux = tile_aux(h, geo, tpr);
    const uint64_t n_tiles = (uint64_t)geo.parts * tpr;
    timer_mark(h, call, 4, s);
    k_tile_units<<<1, 1024, 0, s>>>(mv.counts, mv.begin, mv.cursor, 1, geo.parts, unit,
                                    aux.unit_base, aux.deferred, mv.flag);
    DBG_CK(cudaGetLastError());
    {
      int per_sm = 0;
      DBG_CK(cudaFuncSetAttribute(k_tile_count<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  tpr * 4));
      DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_count<B>, B,
                                                           (size_t)tpr * 4));
      k_tile_count<B><<<std::max(1, per_sm) * sms, B, (size_t)tpr * 4, s>>>(
          h->bin_ev, mv.begin, mv.counts, aux, geo.parts, unit, geo.shift, tpr, h->n_slots,
          mv.flag);
      DBG_CK(cudaGetLastError());
    }
    k_tile_offsets<B><<<geo.parts, B, 0, s>>>(mv.begin, aux, geo.parts, tpr, mv.flag);
    DBG_CK(cudaGetLastError());
    // chunks of 8 events per thread: larger blocks for more tiles per region,
    // so that each tile's run in a chunk stays several events long
    if (tpr <= 256) {
      DBG_TRY(launch_tile_scatter<256>(h, mv, aux, geo, unit, tpr, sms, s));
    } else if (tpr <= 512) {
      DBG_TRY(launch_tile_scatter<512>(h, mv, aux, geo, unit, tpr, sms, s));
    } else {
      DBG_TRY(launch_tile_scatter<1024>(h, mv, aux, geo, unit, tpr, sms, s));
    }
    timer_mark(h, call, 5, s);
    {
      // 512 threads: three such CTAs (64 KB of shared memory each) fill an SM
      // with 48 warps, enough to hide the dependent hash and probe latencies
      constexpr int BA = 512;
      constexpr size_t smem = (size_t)kTileSlots * sizeof(Slot);
      DBG_CK(cudaFuncSetAttribute(k_tile_apply<BA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
      int per_sm = 0;
      DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tile_apply<BA>, BA, smem));
      const uint64_t grid = std::min<uint64_t>(n_tiles, (uint64_t)std::max(1, per_sm) * sms);
      k_tile_apply<BA><<<(int)grid, BA, smem, s>>>(
          h->bin_ev2, h->bin_ev, aux, mv.begin, mv.counts, tpr, n_tiles, h->table, h->n_slots,
          h->max_probes, h->d_status, h->d_spill, h->spill_cap, h->d_spill_count, mv.flag);
      DBG_CK(cudaGetLastError());
    }
    timer_mark(h, call, 6, s);
    k_tile_deferred<<<sms * 4, 256, 0, s>>>(h->bin_ev, aux, h->table, h->n_slots, h->max_probes,
                                            h->d_status, h->d_spill, h->spill_cap,
                                            h->d_spill_count, mv.flag);
    DBG_CK(cudaGetLastError());
  } else {
    timer_mark(h, call, 5, s);
    switch (t.apply_unroll) {
      case 2: DBG_TRY(launch_apply_m<B, 2>(h, mv, geo, sms, t, s)); break;
      case 8: DBG_TRY(launch_apply_m<B, 8>(h, mv, geo, sms, t, s)); break;
      default: DBG_TRY(launch_apply_m<B, 4>(h, mv, geo, sms, t, s)); break;
    }
  }
  // the direct insert runs only if the events did not fit the buffer
  timer_mark(h, call, 7, s);
  const int st = launch_insert(&it, 1, tiles, tuning, h->sm_count, s, mv.flag);
  if (st != DBG_OK) return st;
  timer_mark(h, call, 8, s);
  if (!capturing) DBG_CK(cudaEventRecord(h->bin_done, s));
  return DBG_OK;
}

}  // namespace dbg
