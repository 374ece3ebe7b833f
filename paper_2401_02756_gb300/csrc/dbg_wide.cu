// Graphs with k from 33 to 64 (the paper's default is k = 51, Section "Code
// organization"): vertex keys of 32..63 bases need up to 126 bits.
//
// Slot (32 bytes, the same table as for k <= 32): word 0 = the key's high 64
// bits, word 1 = its low 64 bits, then the four 32-bit counters.  An empty
// slot has word 0 = all ones (never a key's high word: it holds at most 62
// bits) and word 1 = 0, which is what the table initialisation writes.
// Claims are one 128-bit atomicCAS (atom.cas.b128); a probe reads word 0
// first, word 1 only when word 0 matches, and settles a possibly torn pair
// (word 0 already new, word 1 not yet visible) with a 128-bit atomic read.
//
// The insert kernel takes tiles of reads: it stages the tiles' packed bytes
// in shared memory (coalesced, bounded by the stream's length), then gives
// each thread vertex positions of the tile; a key is cut from three 64-bit
// words of the staged stream and its 2-bit groups reversed so that the first
// base is most significant.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

struct WideSlot {
  unsigned long long w0;  // key bits 64..127 (kEmpty: empty slot)
  unsigned long long w1;  // key bits 0..63
  uint32_t cnt[4];
};
static_assert(sizeof(WideSlot) == 32, "one sector per slot");

constexpr int kWideTile = 128;        // reads per tile
constexpr int kWideWinBytes = 16384;  // staged bytes per tile (wider tiles read global memory)

__device__ __forceinline__ uint64_t wide_home(uint64_t hi, uint64_t lo, uint64_t n_slots) {
  return __umul64hi(fmix64(lo ^ fmix64(hi ^ 0x9E3779B97F4A7C15ull)), n_slots);
}

// Atomic 128-bit compare-and-swap of a slot's key words; returns the old pair.
__device__ __forceinline__ void cas128(WideSlot *s, uint64_t c0, uint64_t c1, uint64_t v0,
                                       uint64_t v1, uint64_t &o0, uint64_t &o1) {
  asm volatile(
      "{\n"
      ".reg .b128 c, v, d;\n"
      "mov.b128 c, {%2, %3};\n"
      "mov.b128 v, {%4, %5};\n"
      "atom.relaxed.gpu.global.cas.b128 d, [%6], c, v;\n"
      "mov.b128 {%0, %1}, d;\n"
      "}\n"
      : "=l"(o0), "=l"(o1)
      : "l"(c0), "l"(c1), "l"(v0), "l"(v1), "l"(&s->w0)
      : "memory");
}

// Slot of key (hi, lo), claimed if absent; false after max_probes slots.
__device__ __forceinline__ bool wide_find_or_claim(WideSlot *t, uint64_t n_slots,
                                                   uint32_t max_probes, uint64_t hi, uint64_t lo,
                                                   uint64_t &slot) {
  uint64_t s = wide_home(hi, lo, n_slots);
  for (uint32_t i = 0; i < max_probes; ++i) {
    const unsigned long long w0 = ld_relaxed_u64(&t[s].w0);
    uint64_t o0, o1;
    if (w0 == kEmpty) {
      cas128(&t[s], kEmpty, 0ull, hi, lo, o0, o1);
      if ((o0 == kEmpty && o1 == 0ull) || (o0 == hi && o1 == lo)) {
        slot = s;
        return true;
      }
    } else if (w0 == hi) {
      if (ld_relaxed_u64(&t[s].w1) == lo) {
        slot = s;
        return true;
      }
      cas128(&t[s], kEmpty, 0ull, kEmpty, 0ull, o0, o1);  // an atomic read of the pair
      if (o0 == hi && o1 == lo) {
        slot = s;
        return true;
      }
    }
    if (++s == n_slots) s = 0;
  }
  return false;
}

__device__ __forceinline__ uint64_t rev_pairs(uint64_t x) {
  x = __brevll(x);
  return ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
}

// Key (hi, lo) of m bases (32 <= m <= 63) whose little-endian 2-bit stream
// starts at bit `sh` (< 64) of the words w0, w1, w2.
__device__ __forceinline__ void wide_key(uint64_t w0, uint64_t w1, uint64_t w2, uint32_t sh,
                                         int m, uint64_t &hi, uint64_t &lo) {
  const uint64_t x_lo = sh ? (w0 >> sh) | (w1 << (64u - sh)) : w0;  // bases 0..31
  const uint64_t x_hi = sh ? (w1 >> sh) | (w2 << (64u - sh)) : w1;  // bases 32..63
  const uint64_t a = rev_pairs(x_lo), b = rev_pairs(x_hi);          // base 0 on top of a
  const int s = 128 - 2 * m;                                        // 2 .. 64
  if (s == 64) {
    hi = 0;
    lo = a;
  } else {
    hi = a >> s;
    lo = (b >> s) | (a << (64 - s));
  }
}

// Little-endian 64-bit word of the stream at byte `at`, bytes past nbytes as 0.
__device__ __forceinline__ uint64_t word_at(const uint8_t *packed, uint64_t nbytes, uint64_t at) {
  uint64_t w = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i)
    if (at + i < nbytes) w |= (uint64_t)__ldg(packed + at + i) << (8 * i);
  return w;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_insert_wide(ItemDesc it) {
  __shared__ uint64_t s_off[kWideTile + 1];
  __shared__ uint64_t s_pre[kWideTile + 1];
  __shared__ __align__(16) uint64_t s_win[kWideWinBytes / 8 + 4];
  __shared__ uint32_t s_stop;
  __shared__ uint64_t s_b0, s_staged;  // first staged byte (8-aligned); bytes staged (0: none)
  const int k = it.k, m = k - 1;
  const uint64_t last = it.offsets[it.n_reads];
  const uint64_t nbytes = last >= it.origin ? (last - it.origin + 3) >> 2 : 0;
  WideSlot *table = reinterpret_cast<WideSlot *>(it.table);
  const uint64_t tiles = (it.n_reads + kWideTile - 1) / kWideTile;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t r0 = t * kWideTile;
    const int nr = (int)min((uint64_t)kWideTile, it.n_reads - r0);
    if (threadIdx.x == 0) s_stop = ld_volatile_u32(it.status);
    for (int i = threadIdx.x; i <= nr; i += BLOCK) s_off[i] = it.offsets[r0 + i];
    __syncthreads();
    if (s_stop) return;  // an earlier error stops the insert (the same value for every thread)
    if (threadIdx.x == 0) {
      // vertex positions per read, prefix; bad offsets stop the tile
      uint64_t acc = 0;
      bool bad = false;
      for (int i = 0; i < nr; ++i) {
        s_pre[i] = acc;
        const uint64_t a = s_off[i], b = s_off[i + 1];
        if (b < a || a < it.origin) bad = true;
        const uint64_t len = b >= a ? b - a : 0;
        acc += len >= (uint64_t)k ? len - k + 2 : 0;
      }
      s_pre[nr] = bad ? 0 : acc;
      if (bad) set_sticky(it.status, DBG_ERR_BAD_OFFSETS);
      // the tile's bytes, staged if they fit the window
      const uint64_t lo_b = s_off[0] >= it.origin ? ((s_off[0] - it.origin) >> 2) & ~7ull : 0;
      const uint64_t hi_b = s_off[nr] >= it.origin ? ((s_off[nr] - it.origin + 3) >> 2) : 0;
      s_b0 = lo_b;
      s_staged = (!bad && hi_b > lo_b && hi_b - lo_b + 24 <= (uint64_t)kWideWinBytes)
                     ? hi_b - lo_b + 24
                     : 0;
    }
    __syncthreads();
    const uint64_t staged = s_staged, b0 = s_b0;
    if (staged) {
      unsigned char *win = reinterpret_cast<unsigned char *>(s_win);
      for (uint64_t i = threadIdx.x; i < staged; i += BLOCK)
        win[i] = b0 + i < nbytes ? it.packed[b0 + i] : (unsigned char)0;
    }
    __syncthreads();
    const uint64_t total = s_pre[nr];
    for (uint64_t v = threadIdx.x; v < total; v += BLOCK) {
      int lo_r = 0, hi_r = nr - 1;  // the read holding vertex position v
      while (lo_r < hi_r) {
        const int mid = (lo_r + hi_r + 1) >> 1;
        if (s_pre[mid] <= v)
          lo_r = mid;
        else
          hi_r = mid - 1;
      }
      const uint64_t j = v - s_pre[lo_r];
      const uint64_t len = s_off[lo_r + 1] - s_off[lo_r];
      const uint64_t p = s_off[lo_r] - it.origin + j;  // first base of the vertex
      const bool edge = j + (uint64_t)k <= len;
      uint64_t w0, w1, w2, wl;
      uint32_t sh;
      if (staged) {
        const uint64_t bit = 2 * p - 8 * b0;
        const uint64_t wi = bit >> 6;
        sh = (uint32_t)(bit & 63);
        w0 = s_win[wi];
        w1 = s_win[wi + 1];
        w2 = s_win[wi + 2];
      } else {
        const uint64_t at = (p >> 2);
        sh = (uint32_t)(2 * (p & 3));
        w0 = word_at(it.packed, nbytes, at);
        w1 = word_at(it.packed, nbytes, at + 8);
        w2 = word_at(it.packed, nbytes, at + 16);
      }
      uint64_t hi, lo;
      wide_key(w0, w1, w2, sh, m, hi, lo);
      uint32_t label = 0;
      if (edge) {
        const uint64_t q = p + (uint64_t)m;  // the k-mer's last base
        if (staged) {
          const uint64_t bit = 2 * q - 8 * b0;
          wl = s_win[bit >> 6] >> (bit & 63);
        } else {
          wl = (uint64_t)__ldg(it.packed + (q >> 2)) >> (2 * (q & 3));
        }
        label = (uint32_t)(wl & 3u);
      }
      uint64_t s;
      if (wide_find_or_claim(table, it.n_slots, it.max_probes, hi, lo, s)) {
        if (edge) atomicAdd(&table[s].cnt[label], 1u);
      } else {
        set_sticky(it.status, DBG_ERR_CAPACITY);
      }
    }
    __syncthreads();
  }
}

// --- export -------------------------------------------------------------------

__global__ void k_wide_words(const WideSlot *t, const unsigned long long *idx, uint64_t n,
                             unsigned long long *out, int word) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = word ? t[idx[i]].w1 : t[idx[i]].w0;
}

__global__ void k_wide_gather(const WideSlot *t, const unsigned long long *idx, uint64_t n,
                              ulonglong2 *keys, uint4 *counts) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const WideSlot &s = t[idx[i]];
    keys[i] = make_ulonglong2(s.w0, s.w1);
    counts[i] = make_uint4(s.cnt[0], s.cnt[1], s.cnt[2], s.cnt[3]);
  }
}

__global__ void k_wide_compact(const WideSlot *t, uint64_t n_slots, unsigned long long *idx,
                               unsigned long long *count, uint64_t cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (((uint64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (uint64_t base = w0 * 32; base < n_slots; base += warps * 32) {
    const uint64_t i = base + lane;
    const bool occ = i < n_slots && t[i].w0 != kEmpty;
    const unsigned mask = __ballot_sync(0xffffffffu, occ);
    unsigned long long pos = 0;
    if (lane == 0 && mask) pos = atomicAdd(count, (unsigned long long)__popc(mask));
    pos = __shfl_sync(0xffffffffu, pos, 0);
    const unsigned long long at = pos + __popc(mask & ((1u << lane) - 1u));
    if (occ && at < cap) idx[at] = i;
  }
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

int launch_insert_wide(const ItemDesc &it, int sm_count, cudaStream_t s) {
  if (it.n_reads == 0) return DBG_OK;
  constexpr int B = 256;
  int per_sm = 0;
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_insert_wide<B>, B, 0));
  const uint64_t tiles = (it.n_reads + kWideTile - 1) / kWideTile;
  const int grid =
      (int)std::min<uint64_t>(tiles, (uint64_t)std::max(1, per_sm) * std::max(1, sm_count));
  k_insert_wide<B><<<grid, B, 0, s>>>(it);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

// Sorted export of a wide table: compaction, then two stable radix sorts
// (low words, then high words) carrying the slot indices, then a gather.
int export_sorted_wide(dbg_handle h, uint64_t D, uint64_t *keys_out, uint32_t *counts_out,
                       cudaStream_t s) {
  const int m = h->k - 1;
  const int hi_bits = 2 * m - 64;  // bits of the high word (0 .. 62)
  const WideSlot *t = reinterpret_cast<const WideSlot *>(h->table);
  size_t temp_bytes = 0;
  DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr,
                                         (unsigned long long *)nullptr, (int64_t)D, 0, 64, s));
  const size_t kb = al256(D * sizeof(unsigned long long));
  const size_t total = 4 * kb + al256(D * 16) + al256(D * 16) + 256 + al256(temp_bytes);
  char *buf = nullptr;
  DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), total, s));
  unsigned long long *w_a = reinterpret_cast<unsigned long long *>(buf);
  unsigned long long *w_b = reinterpret_cast<unsigned long long *>(buf + kb);
  unsigned long long *idx_a = reinterpret_cast<unsigned long long *>(buf + 2 * kb);
  unsigned long long *idx_b = reinterpret_cast<unsigned long long *>(buf + 3 * kb);
  ulonglong2 *keys = reinterpret_cast<ulonglong2 *>(buf + 4 * kb);
  uint4 *counts = reinterpret_cast<uint4 *>(buf + 4 * kb + al256(D * 16));
  unsigned long long *count =
      reinterpret_cast<unsigned long long *>(buf + 4 * kb + 2 * al256(D * 16));
  void *temp = buf + 4 * kb + 2 * al256(D * 16) + 256;
  const int grid = std::max(1, h->sm_count) * 8;
  int rc = DBG_OK;
  do {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    k_wide_compact<<<grid, 256, 0, s>>>(t, h->n_slots, idx_a, count, D);
    k_wide_words<<<grid, 256, 0, s>>>(t, idx_a, D, w_a, 1);  // low words
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, w_a, w_b, idx_a, idx_b, (int64_t)D, 0,
                                        64, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "SortPairs(low words)"); break; }
    const unsigned long long *order = idx_b;
    if (hi_bits > 0) {  // stable: equal high words keep their low-word order
      k_wide_words<<<grid, 256, 0, s>>>(t, idx_b, D, w_a, 0);
      e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, w_a, w_b, idx_b, idx_a, (int64_t)D,
                                          0, hi_bits, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "SortPairs(high words)"); break; }
      order = idx_a;
    }
    k_wide_gather<<<grid, 256, 0, s>>>(t, order, D, keys, counts);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "wide export kernels"); break; }
    if (keys_out) {
      e = cudaMemcpyAsync(keys_out, keys, D * 16, cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(keys)"); break; }
    }
    if (counts_out) {
      e = cudaMemcpyAsync(counts_out, counts, D * sizeof(uint4), cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
    }
  } while (0);
  cudaError_t e = cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}

}  // namespace dbg
