// Read-tile machinery shared by the insert kernels: walk read tiles, stage
// them in shared memory, and hand every vertex position to a visitor.
//
// Work unit: a tile of `tile_reads` consecutive reads of one item.  A CTA
//   1. stages the tile's offsets in shared memory, computes each read's vertex
//      count (len - k + 2 for len >= k, else 0: the last vertex of a read is a
//      target only, Alg. 2 with the addRightVertex prose) and a block-wide
//      prefix sum of them;
//   2. stages the packed bases the tile spans in a shared-memory window with
//      coalesced 16-byte loads (a tile wider than the window is cut into
//      sub-tiles; a single read wider than the window reads its bases from
//      global memory);
//   3. maps each thread to a run of up to R consecutive vertex positions of
//      one read (R >= 4: every read is cut into ceil(positions / R) runs, so
//      a run never crosses a read boundary; inside a window with 32-bit
//      indices relative to the sub-tile and the window).  A run's first key
//      is extracted -- the k-1 bases, first base most significant -- from two
//      64-bit window words with a funnel shift and a 2-bit-group reversal;
//      the run's R labels (the label s_{k-1} of a position is the base after
//      its key, the last base of the next key) come from one more funnel
//      shift, and the next keys roll: key' = ((key << 2) | label) & mask.
//      (R < 4, the direct insert: a thread's R positions are consecutive
//      positions of the flattened sub-tile and may cross reads.)
//   4. calls vis.vertex(...) for every position, in block-uniform rounds of
//      BLOCK runs, and vis.round_end() after every round.
// A visitor whose rounds contain __syncthreads sets kUniformRounds; the
// insert visitor instead may stop a thread early (vis.stop()).  The CTA walks
// tiles t_first, t_first + t_stride, ... below t_end; every thread of the CTA
// must call for_each_vertex with the same arguments.
#pragma once

#include <type_traits>

#include "dbg_internal.cuh"

namespace dbg {

constexpr int kWinWords = 2048;  // 16 KB window of packed bases per CTA (64 Ki bases)
constexpr unsigned kFull = 0xffffffffu;

// Dynamic shared memory the tile machinery uses (the visitor's own region
// follows it, 16-byte aligned): the window, the reads' offsets and vertex
// prefix (64-bit), both again relative to the window (32-bit), and the
// reads' run prefix for the tile and relative to the sub-tile (32-bit).
__host__ __device__ constexpr size_t tile_smem_bytes(int tile_reads) {
  return (size_t)(kWinWords + 2) * 8 + (size_t)(tile_reads + 1) * 16 +
         2 * (((size_t)(tile_reads + 1) * 8 + 15) & ~(size_t)15);
}

// What a visitor learns about the item a vertex belongs to.
struct VertexCtx {
  Slot *table;
  uint64_t n_slots;
  uint32_t *status;
  uint32_t max_probes;
  int k;
  int item;
  SpillRecord *spill;
  uint64_t spill_cap;
  unsigned long long *spill_count;
  int region0;  // the item's first region (binned insert)
};

__device__ __forceinline__ uint4 ldg_stream_v4(const uint8_t *p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
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

// Base `pos` of the packed stream from global memory (0 past the end).
__device__ __forceinline__ uint32_t base_from_global(const uint8_t *packed, uint64_t nbytes,
                                                     uint64_t pos) {
  const uint64_t b = pos >> 2;
  return b < nbytes ? (uint32_t)(__ldg(packed + b) >> (2 * (pos & 3))) & 3u : 0u;
}

// Walk tiles t_first, t_first + t_stride, ... (< t_end) of the items in `pk`.
template <int BLOCK, int N, int R, class Visitor>
__device__ __forceinline__ void for_each_vertex(const ItemPack<N> &pk, int tile_reads,
                                                unsigned char *smem_raw, Visitor &vis,
                                                uint64_t t_first, uint64_t t_end,
                                                uint64_t t_stride) {
  uint64_t *s_win = reinterpret_cast<uint64_t *>(smem_raw);  // kWinWords + 2
  uint64_t *s_off = s_win + kWinWords + 2;                     // tile_reads + 1
  uint64_t *s_vpre = s_off + tile_reads + 1;                   // tile_reads + 1
  // inside a window: vertex prefix relative to the sub-tile's first vertex,
  // read starts relative to the window's first base (tile_reads + 1 each)
  uint32_t *s_vrel = reinterpret_cast<uint32_t *>(s_vpre + tile_reads + 1);
  uint32_t *s_prel = s_vrel + tile_reads + 1;
  // runs (R >= 4): first run of every read, for the tile and for the sub-tile
  // (modulo 2^32: only differences inside a window-sized sub-tile are used)
  uint32_t *s_upre = reinterpret_cast<uint32_t *>(
      reinterpret_cast<unsigned char *>(s_vrel) + (((size_t)(tile_reads + 1) * 8 + 15) & ~(size_t)15));
  uint32_t *s_urel = s_upre + tile_reads + 1;
  constexpr bool kAligned = R >= 4;
  static_assert(!kAligned || ((R & (R - 1)) == 0 && R <= 32), "aligned runs: R a power of two <= 32");
  using LabelWord = typename std::conditional<(R <= 16), uint32_t, uint64_t>::type;

  __shared__ ItemDesc s_item;
  __shared__ int s_item_idx;
  __shared__ uint32_t s_stop;
  __shared__ uint64_t s_nbytes;
  __shared__ uint64_t s_warp[BLOCK / 32];
  __shared__ uint32_t s_warpu[BLOCK / 32];
  __shared__ int s_rb, s_global;
  __shared__ uint64_t s_wb0;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) s_item_idx = -1;

  const uint64_t total_tiles = min(pk.total_tiles, t_end);
  for (uint64_t t = t_first; t < total_tiles; t += t_stride) {
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
    }
    vis.tile_begin();
    __syncthreads();
    if (s_stop == 0u) {
      const uint8_t *packed = s_item.packed;
      const uint64_t origin = s_item.origin;
      const VertexCtx ctx{s_item.table,      s_item.n_slots,   s_item.status,
                          s_item.max_probes, s_item.k,         s_item_idx,
                          s_item.spill,      s_item.spill_cap, s_item.spill_count,
                          s_item.region0};
      const int k = ctx.k, m = k - 1;
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
        // runs of the read (R >= 4), modulo 2^32
        const uint32_t nu = kAligned ? (uint32_t)((nv + (uint64_t)(R - 1)) / (uint64_t)R) : 0u;
        uint64_t incl = nv;
        uint32_t inclu = nu;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const uint64_t o = __shfl_up_sync(kFull, incl, d);
          if (lane >= d) incl += o;
          if (kAligned) {
            const uint32_t ou = __shfl_up_sync(kFull, inclu, d);
            if (lane >= d) inclu += ou;
          }
        }
        if (lane == 31) {
          s_warp[warp] = incl;
          if (kAligned) s_warpu[warp] = inclu;
        }
        __syncthreads();
        if (warp == 0) {
          uint64_t w = lane < BLOCK / 32 ? s_warp[lane] : 0;
          uint32_t wu = kAligned && lane < BLOCK / 32 ? s_warpu[lane] : 0u;
#pragma unroll
          for (int d = 1; d < 32; d <<= 1) {
            const uint64_t o = __shfl_up_sync(kFull, w, d);
            if (lane >= d) w += o;
            if (kAligned) {
              const uint32_t ou = __shfl_up_sync(kFull, wu, d);
              if (lane >= d) wu += ou;
            }
          }
          if (lane < BLOCK / 32) {
            s_warp[lane] = w;  // inclusive over warps
            if (kAligned) s_warpu[lane] = wu;
          }
        }
        __syncthreads();
        const uint64_t excl = incl - nv + (warp > 0 ? s_warp[warp - 1] : 0);
        if (tid < nr) s_vpre[tid] = excl;
        if (tid == nr - 1) s_vpre[nr] = excl + nv;
        if (kAligned) {
          const uint32_t exclu = inclu - nu + (warp > 0 ? s_warpu[warp - 1] : 0u);
          if (tid < nr) s_upre[tid] = exclu;
          if (tid == nr - 1) s_upre[nr] = exclu + nu;
        }
        __syncthreads();

        // 2-4. sub-tiles whose bases fit the window
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
            // the sub-tile's reads fit the window: 32-bit indices from here on
            for (int i = ra + tid; i <= rb; i += BLOCK) {
              s_vrel[i] = (uint32_t)(s_vpre[i] - s_vpre[ra]);
              s_prel[i] = (uint32_t)(s_off[i] - origin - (wb0 << 2));
              if (kAligned) s_urel[i] = s_upre[i] - s_upre[ra];
            }
            __syncthreads();
          }
          const uint64_t v_lo = s_vpre[ra], v_hi = s_vpre[rb];
          const uint64_t mask = (1ull << (2 * m)) - 1ull;
          int r = ra;
          if (kAligned && !gmode) {
            // runs of up to R positions of one read: run u of the sub-tile
            // belongs to the last read whose first run is at or before u
            const uint32_t n_runs = s_urel[rb];
            for (uint32_t ub = 0; ub < n_runs; ub += (uint32_t)BLOCK) {
              if (!Visitor::kUniformRounds && vis.stop(lane)) break;
              const uint32_t u = ub + (uint32_t)tid;
              uint64_t key = kEmpty;
              LabelWord labels = 0;
              uint32_t cnt = 0, cnt_edge = 0;
              if (u < n_runs) {
                int lo = ra, hi = rb - 1;
                while (lo < hi) {
                  const int mid = (lo + hi + 1) >> 1;
                  if (s_urel[mid] <= u)
                    lo = mid;
                  else
                    hi = mid - 1;
                }
                const uint32_t j0 = (u - s_urel[lo]) * (uint32_t)R;  // first position in the read
                const uint32_t nvr = s_vrel[lo + 1] - s_vrel[lo];     // > j0
                cnt = min((uint32_t)R, nvr - j0);
                cnt_edge = min((uint32_t)R, nvr - 1u - j0);  // the read's last vertex has no edge
                const uint32_t q = s_prel[lo] + j0;
                key = key_from_words(s_win[q >> 5], s_win[(q >> 5) + 1], (q & 31) * 2, m);
                const uint32_t qe = q + (uint32_t)m;  // base of the first label
                const uint32_t sh = (qe & 31) * 2;
                const uint64_t w0 = s_win[qe >> 5], w1 = s_win[(qe >> 5) + 1];
                labels = (LabelWord)(sh ? (w0 >> sh) | (w1 << (64u - sh)) : w0);
              }
#pragma unroll
              for (int sub = 0; sub < R; ++sub) {
                const uint32_t label = (uint32_t)(labels >> (2 * sub)) & 3u;
                vis.vertex((uint32_t)sub < cnt, key, (uint32_t)sub < cnt_edge, label, lane, sub,
                           ctx);
                key = ((key << 2) | label) & mask;
              }
              if (Visitor::kUniformRounds) vis.round_end();
            }
            __syncthreads();
            ra = rb;
            continue;
          }
          if (!gmode) {
            // v: vertex index relative to v_lo; q: base position relative to
            // the window; the read holding v spans vertices [., vr1) and
            // bases [., qend)
            const uint32_t nv = (uint32_t)(v_hi - v_lo);
            for (uint32_t base = 0; base < nv; base += (uint32_t)BLOCK * R) {
              if (!Visitor::kUniformRounds && vis.stop(lane)) break;
              uint32_t v = base + (uint32_t)tid * R;
              uint64_t key = kEmpty;
              uint32_t label = 0, vr1 = 0, q = 0, qend = 0;
              bool have = false;
#pragma unroll
              for (int sub = 0; sub < R; ++sub, ++v) {
                const bool valid = v < nv;
                bool edge = false;
                if (valid) {
                  bool fresh = !have;
                  if (fresh || v >= vr1) {
                    while (s_vrel[r + 1] <= v) ++r;  // the next read (or a few reads on)
                    vr1 = s_vrel[r + 1];
                    q = s_prel[r] + (v - s_vrel[r]);
                    qend = s_prel[r + 1];
                    fresh = true;
                  } else {
                    ++q;
                  }
                  edge = q + (uint32_t)k <= qend;
                  if (fresh) {
                    const uint32_t wi = q >> 5;
                    key = key_from_words(s_win[wi], s_win[wi + 1], (q & 31) * 2, m);
                  } else {
                    key = ((key << 2) | label) & mask;
                  }
                  const uint32_t qe = q + (uint32_t)m;
                  label = (uint32_t)(s_win[qe >> 5] >> ((qe & 31) * 2)) & 3u;
                  have = true;
                }
                vis.vertex(valid, key, edge, label, lane, sub, ctx);
              }
              if (Visitor::kUniformRounds) vis.round_end();
            }
            __syncthreads();
            ra = rb;
            continue;
          }
          // a read wider than the window: its bases come from global memory
          for (uint64_t base = v_lo; base < v_hi; base += (uint64_t)BLOCK * R) {
            if (!Visitor::kUniformRounds && vis.stop(lane)) break;
            uint64_t v = base + (uint64_t)tid * R;
            uint64_t key = kEmpty;
            uint32_t label = 0;
            // the read holding position v: vertex range [vr0, vr1), bases end at pend
            uint64_t vr1 = 0, p = 0, pend = 0;
            bool have = false;
#pragma unroll
            for (int sub = 0; sub < R; ++sub, ++v) {
              const bool valid = v < v_hi;
              bool edge = false;
              if (valid) {
                bool fresh = !have;
                if (fresh || v >= vr1) {
                  while (s_vpre[r + 1] <= v) ++r;
                  vr1 = s_vpre[r + 1];
                  p = s_off[r] - origin + (v - s_vpre[r]);
                  pend = s_off[r + 1] - origin;
                  fresh = true;
                } else {
                  ++p;
                }
                edge = p + (uint64_t)k <= pend;
                if (fresh) {
                  key = key_from_global(packed, nbytes, p, m, label);
                } else {
                  key = ((key << 2) | label) & mask;
                  label = base_from_global(packed, nbytes, p + (uint64_t)m);
                }
                have = true;
              }
              vis.vertex(valid, key, edge, label, lane, sub, ctx);
            }
            if (Visitor::kUniformRounds) vis.round_end();
          }
          __syncthreads();
          ra = rb;
        }
      } else if (tid == 0) {
        set_sticky(ctx.status, DBG_ERR_BAD_OFFSETS);
      }
    }
    __syncthreads();
  }
}

}  // namespace dbg
