// The binned insert: the same table updates as the direct insert kernel
// (find or claim the prefix and suffix vertices, count the label -- Alg. 2-4
// and the addRightVertex prose), issued in an order that keeps the table
// region being updated resident in L2.
//
// A random 32-byte slot of a table far larger than L2 costs a DRAM round trip
// that fetches a whole 128-byte line, which caps the direct insert near the
// random-sector rate of HBM.  The same load + atomicAdd pattern on an
// L2-resident region runs about 9x faster.  So for a large table and a large
// call, the insert runs in four kernels:
//   K1b count   -- walk the read tiles, compute every vertex's key and home
//                  slot, and histogram the vertices by table region
//                  (region = 2^shift consecutive slots, at most 2048 regions);
//   K1c scan    -- exclusive prefix of the histogram: each region's event range;
//   K1d scatter -- walk the tiles again and write one 8-byte event per vertex,
//                  (key << 3) | (edge << 2) | label, into its region's range
//                  (block-local counting sort in shared memory, one global
//                  atomicAdd per non-empty region per 2048 events, coalesced
//                  stores);
//   K1e apply   -- stream the events in region order and apply them to the
//                  table with the insert's own find-or-claim and atomicAdd:
//                  all CTAs sweep the regions together, so the table lines
//                  they touch are L2 hits after their first miss.
// The result is identical to the direct insert (additions commute).  Events
// hold a key of at most 60 bits, so the binned path serves k <= 31.  K1c
// checks that the events fit the handle's event buffer; if not, K1d/K1e do
// nothing and the direct insert kernel, launched after them with the same
// flag as its gate, does the work instead.
#include <algorithm>

#include "dbg_binned.cuh"
#include "dbg_tiles.cuh"

namespace dbg {
namespace {

constexpr int kMaxParts = kBinMaxParts;
constexpr int kRun = 8;             // consecutive vertex positions per thread (rolled keys)
constexpr int kRoundEvents = 2048;  // events buffered per scatter flush (256 threads x kRun)

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
  static_assert(BLOCK * kRun == kRoundEvents, "one round is one flush");
  uint64_t *sorted;    // kRoundEvents, in region order
  uint16_t *spid;      // region of sorted[j]
  uint32_t *hist;      // parts: events per region in this round
  uint32_t *off;       // parts: exclusive prefix of hist
  unsigned long long *cur;    // parts: next global position of each region (this slice)
  unsigned long long *gbase;  // parts: cur[p] - off[p] for this round
  uint64_t *out;
  uint64_t cap;  // events the buffer holds: never store past it
  int shift, parts;
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
      gbase[p] = cur[p] - run;
      cur[p] += h;
      run += h;
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
      const unsigned long long at = gbase[spid[j]] + j;
      if (at < cap) __stcs(out + at, sorted[j]);
    }
    __syncthreads();
    for (int p = tid; p < parts; p += BLOCK) hist[p] = 0;
    __syncthreads();
  }
};

template <int BLOCK>
constexpr size_t scatter_smem(int tile_reads, int parts) {
  return tile_smem_bytes(tile_reads) + (size_t)kRoundEvents * (8 + 2) +
         (size_t)parts * (4 + 4 + 8 + 8) + 64;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK)
    k_bin_scatter(const __grid_constant__ ItemPack<1> pk, int tile_reads, int shift, int parts,
                  uint64_t slices, const uint32_t *hist, unsigned long long *cursor, uint64_t *out,
                  uint64_t cap, unsigned long long *ctr, const uint32_t *use_binned) {
  if (ld_volatile_u32(use_binned) == 0u) return;
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned char *p = smem + tile_smem_bytes(tile_reads);
  ScatterVisitor<BLOCK> vis;
  vis.sorted = reinterpret_cast<uint64_t *>(p);
  p += kRoundEvents * 8;
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
  const uint64_t T = pk.total_tiles;
  for (int q = threadIdx.x; q < parts; q += BLOCK) vis.hist[q] = 0;
  for (;;) {
    const uint64_t sl = grab(&ctr[1]);
    if (sl >= slices) break;
    // reserve this slice's run in every region it reaches (counted by K1b)
    for (int q = threadIdx.x; q < parts; q += BLOCK) {
      const uint32_t h = hist[sl * parts + q];
      vis.cur[q] = h ? atomicAdd(&cursor[q], (unsigned long long)h) : 0ull;
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
  if (events == 0) events = std::max(kBinMinEvents, kBinEventsPerSlot * h->n_slots);
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
    h->bin_ev = nullptr;
    h->bin_cap = 0;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, events * sizeof(uint64_t));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(binned events)");
    h->bin_ev = static_cast<uint64_t *>(p);
    h->bin_cap = events;
  }
  return DBG_OK;
}


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

int launch_binned(dbg_handle h, const ItemDesc &it, uint64_t tiles, const dbg_tuning &tuning,
                  cudaStream_t s, int call) {
  constexpr int B = 256;
  const dbg_tuning t = resolve_tuning(tuning);
  const int tile_reads = std::min(t.tile_reads, B);
  const BinGeometry geo = bin_geometry(h->n_slots, t.region_log2);
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
  DBG_CK(cudaMemsetAsync(mv.ctr, 0, 4 * sizeof(unsigned long long), s));
  DBG_CK(cudaMemsetAsync(mv.counts, 0, geo.parts * sizeof(unsigned long long), s));
  timer_mark(h, call, 1, s);
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
  }
  timer_mark(h, call, 2, s);
  k_bin_scan<<<1, 1024, 0, s>>>(mv.counts, geo.parts, mv.begin, mv.cursor, h->bin_cap, mv.ctr,
                                mv.flag);
  DBG_CK(cudaGetLastError());
  timer_mark(h, call, 3, s);
  {
    const size_t smem = scatter_smem<B>(tile_reads, geo.parts);
    DBG_CK(cudaFuncSetAttribute(k_bin_scatter<B>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bin_scatter<B>, B, smem));
    const int grid = (int)std::min<uint64_t>(slices, (uint64_t)std::max(1, per_sm) * sms);
    k_bin_scatter<B><<<grid, B, smem, s>>>(pk, tile_reads, geo.shift, geo.parts, slices, mv.hist,
                                           mv.cursor, h->bin_ev, h->bin_cap, mv.ctr, mv.flag);
    DBG_CK(cudaGetLastError());
  }
  timer_mark(h, call, 4, s);
  switch (t.apply_unroll) {
    case 2: DBG_TRY(launch_apply_m<B, 2>(h, mv, geo, sms, t, s)); break;
    case 8: DBG_TRY(launch_apply_m<B, 8>(h, mv, geo, sms, t, s)); break;
    default: DBG_TRY(launch_apply_m<B, 4>(h, mv, geo, sms, t, s)); break;
  }
  // the direct insert runs only if the events did not fit the buffer
  timer_mark(h, call, 5, s);
  const int st = launch_insert(&it, 1, tiles, tuning, h->sm_count, s, mv.flag);
  if (st != DBG_OK) return st;
  timer_mark(h, call, 6, s);
  if (!capturing) DBG_CK(cudaEventRecord(h->bin_done, s));
  return DBG_OK;
}

}  // namespace dbg
