// Sorted export of a graph (K3 compaction, K4 radix sort, gather): the
// (vertex, counters) table of the paper's Fig. 1 in key order, which is
// lexicographic order with A < C < G < T because keys hold the first base in
// their most significant bits.  Not on the timed insert path.
//
// The radix sort is CUB's DeviceRadixSort (open-source CCCL headers shipped
// with the CUDA toolkit); compaction and gather are this file's kernels.
//
// Memory.  The sort orders (key, slot index) pairs -- 8 + 4 bytes a vertex
// while the table has fewer than 2^32 slots -- and needs a second buffer of
// each.  When both outputs are device buffers they hold all four: keys_out
// is the first key buffer, and counts_out (16 bytes a vertex) holds the
// second key buffer and both index buffers until the gather overwrites it.
// The only temporary memory is then one index array (4 bytes a vertex: the
// gather cannot read its indices from the buffer it writes) and the sort's
// small histogram space.  Host outputs go through temporary device buffers.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr int kCompactBlock = 256;
constexpr int kCompactPer = 8;  // slots per thread per round: 2048 per CTA round

// K3: (key, slot index) of every occupied slot, at most `cap` of them (the
// vertices counted beforehand; nothing is ever written past the buffers).
// Each CTA round takes 2048 consecutive slots; every warp ranks its occupied
// slots with ballots, the warps' totals are summed in shared memory, and one
// atomicAdd per round places the CTA's run -- so a warp's writes of one
// ballot are 32 consecutive entries.  The order of the runs does not matter:
// the sort follows.
template <class I>
__global__ void __launch_bounds__(kCompactBlock)
    k_compact(const Slot *t, uint64_t n_slots, unsigned long long *keys, I *idx,
              unsigned long long *count, uint64_t cap) {
  constexpr int W = kCompactBlock / 32;
  __shared__ uint32_t s_w[W];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  constexpr uint64_t kRound = (uint64_t)kCompactBlock * kCompactPer;
  for (uint64_t base = (uint64_t)blockIdx.x * kRound; base < n_slots;
       base += (uint64_t)gridDim.x * kRound) {
    unsigned long long k[kCompactPer];
    unsigned bal[kCompactPer];
    uint32_t wcount = 0;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      const uint64_t i = base + (uint64_t)r * kCompactBlock + threadIdx.x;
      k[r] = i < n_slots ? __ldcs(&t[i].key) : kEmpty;
      bal[r] = __ballot_sync(0xffffffffu, k[r] != kEmpty);
      wcount += (uint32_t)__popc(bal[r]);
    }
    if (lane == 0) s_w[warp] = wcount;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const uint32_t v = s_w[j];
      before += j < warp ? v : 0u;
      total += v;
    }
    if (threadIdx.x == 0) s_base = total ? atomicAdd(count, (unsigned long long)total) : 0ull;
    __syncthreads();
    uint64_t pos = s_base + before;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      if (k[r] != kEmpty) {
        const uint64_t at = pos + (uint64_t)__popc(bal[r] & lt);
        if (at < cap) {
          keys[at] = k[r];
          idx[at] = (I)(base + (uint64_t)r * kCompactBlock + threadIdx.x);
        }
      }
      pos += (uint64_t)__popc(bal[r]);
    }
    __syncthreads();  // s_w and s_base are rewritten by the next round
  }
}

// Counters of the sorted vertices, in key order.
template <class I>
__global__ void k_gather(const Slot *t, const I *__restrict__ idx, uint4 *counts, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    // the counters sit at byte 8 of the slot: 8-byte aligned, not 16
    const uint2 *c = reinterpret_cast<const uint2 *>(&t[__ldcs(idx + i)].cnt[0]);
    const uint2 lo = c[0], hi = c[1];
    __stcs(counts + i, make_uint4(lo.x, lo.y, hi.x, hi.y));
  }
}

// The prefix sort.  Keys of up to 60 bits are sorted by their top 32 bits
// only (4 radix passes of 32-bit keys and 32-bit slot indices instead of 8
// of 64-bit keys: a third less traffic per pass, half the passes).  The
// gather then writes the keys and counters in that order, and the keys that
// share a prefix -- reads with an error in a k-mer's last bases give such
// "siblings" of a genomic k-mer, a few per k-mer at 30x, a hundred in a
// high-copy repeat -- form runs of the output, each put in key order in
// place: a thread sorts a short run in registers, a CTA sorts a long one in
// shared memory.  A run longer than kMaxLongRun (keys crowded into a few
// prefixes) makes the export fall back to the full-width sort.
constexpr int kShortRun = 4;      // runs up to this long: one thread, in registers
constexpr int kWarpRun = 32;      // up to this long: one warp, a register bitonic sort
constexpr int kMaxLongRun = 2048; // longer runs: the full-width sort instead
constexpr int kLongBlock = 256;

// K3 for the prefix sort: (top 32 bits of the key, slot index) of every
// occupied slot, at most `cap` of them; otherwise as k_compact.
__global__ void __launch_bounds__(kCompactBlock)
    k_compact_prefix(const Slot *t, uint64_t n_slots, int pshift, uint32_t *prefix, uint32_t *idx,
                     unsigned long long *count, uint64_t cap) {
  constexpr int W = kCompactBlock / 32;
  __shared__ uint32_t s_w[W];
  __shared__ unsigned long long s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  constexpr uint64_t kRound = (uint64_t)kCompactBlock * kCompactPer;
  for (uint64_t base = (uint64_t)blockIdx.x * kRound; base < n_slots;
       base += (uint64_t)gridDim.x * kRound) {
    unsigned long long k[kCompactPer];
    unsigned bal[kCompactPer];
    uint32_t wcount = 0;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      const uint64_t i = base + (uint64_t)r * kCompactBlock + threadIdx.x;
      k[r] = i < n_slots ? __ldcs(&t[i].key) : kEmpty;
      bal[r] = __ballot_sync(0xffffffffu, k[r] != kEmpty);
      wcount += (uint32_t)__popc(bal[r]);
    }
    if (lane == 0) s_w[warp] = wcount;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const uint32_t v = s_w[j];
      before += j < warp ? v : 0u;
      total += v;
    }
    if (threadIdx.x == 0) s_base = total ? atomicAdd(count, (unsigned long long)total) : 0ull;
    __syncthreads();
    uint64_t pos = s_base + before;
#pragma unroll
    for (int r = 0; r < kCompactPer; ++r) {
      if (k[r] != kEmpty) {
        const uint64_t at = pos + (uint64_t)__popc(bal[r] & lt);
        if (at < cap) {
          prefix[at] = (uint32_t)(k[r] >> pshift);
          idx[at] = (uint32_t)(base + (uint64_t)r * kCompactBlock + threadIdx.x);
        }
      }
      pos += (uint64_t)__popc(bal[r]);
    }
    __syncthreads();
  }
}

// The run pass works on contiguous chunks: kRunCtas CTAs at most, each
// owning the runs that start in its chunk of `chunk` positions (a multiple of
// kRunBlock).  Runs too long for a thread go to the CTA's own segments of
// two lists, counted in shared memory -- no global atomics: the first
// version appended to one list counter per warp and took 7.3 ms at 100 Mbp,
// serialised on that counter.
constexpr int kRunBlock = 256;
constexpr int kRunCtas = 1216;  // 8 CTAs of 256 threads on each of 152 SMs
constexpr int kRunGroups = 4;   // blocks of kRunBlock positions a thread takes per round

struct RunLists {
  uint64_t chunk;    // positions per CTA
  int ctas;          // CTAs of the run pass
  uint64_t mid_cap;  // list entries per CTA: runs of kShortRun + 1 .. kWarpRun keys
  uint64_t lng_cap;  // runs of more than kWarpRun keys
  uint64_t bytes() const { return (uint64_t)ctas * (mid_cap + lng_cap) * 8; }
};

// The lists for D positions over at most `ctas` CTAs (the scratch is sized
// for kRunCtas; a launch over fewer CTAs uses that layout only when its lists
// fit in those bytes).
RunLists run_lists(uint64_t D, int ctas = kRunCtas) {
  RunLists r;
  const uint64_t per = (D + ctas - 1) / ctas;
  r.chunk = std::max<uint64_t>(kRunBlock, (per + kRunBlock - 1) / kRunBlock * kRunBlock);
  r.ctas = (int)std::max<uint64_t>(1, (D + r.chunk - 1) / r.chunk);
  r.mid_cap = r.chunk / (kShortRun + 1) + 1;  // runs that start in a chunk, at most
  r.lng_cap = r.chunk / (kWarpRun + 1) + 1;
  return r;
}

// Runs of equal prefixes in the gathered output, each put in key order.  A
// warp finds the run starts among its 32 positions by comparing each prefix
// with its neighbour's, and a run's length from the next start in the warp
// (only the warp's last run reads on past it).  The thread at a run's first
// position sorts a run of at most kShortRun keys in registers (keys and
// counter rows together; a run already in order is left as it is); longer
// runs are listed: up to kWarpRun long for k_sort_warp_runs, longer for
// k_sort_long_runs.
__global__ void __launch_bounds__(kRunBlock)
    k_sort_runs(unsigned long long *keys, uint4 *counts, uint64_t n, int pshift, uint64_t chunk,
                unsigned long long *mid, uint64_t mid_cap, uint32_t *mid_n,
                unsigned long long *lng, uint64_t lng_cap, uint32_t *lng_n,
                unsigned int *fallback) {
  __shared__ uint32_t s_mid, s_lng;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  if (threadIdx.x == 0) {
    s_mid = 0u;
    s_lng = 0u;
  }
  __syncthreads();
  const uint64_t c0 = (uint64_t)blockIdx.x * chunk, c1 = min(n, c0 + chunk);
  unsigned long long *my_mid = mid + (uint64_t)blockIdx.x * mid_cap;
  unsigned long long *my_lng = lng + (uint64_t)blockIdx.x * lng_cap;
  // (the loop bound is the CTA's, so every lane takes part in the ballots)
  // kRunGroups blocks of positions a round: their keys are loaded first, so
  // that the loads' latencies overlap; a short run's sort may rewrite keys of
  // a later block of the round, but only within one run, whose keys share the
  // prefix the later block compares
  for (uint64_t round = c0; round < c1; round += (uint64_t)kRunBlock * kRunGroups) {
  unsigned long long gkey[kRunGroups];
  uint64_t gprev[kRunGroups];
#pragma unroll
  for (int g = 0; g < kRunGroups; ++g) {
    const uint64_t i = round + (uint64_t)g * kRunBlock + threadIdx.x;
    gkey[g] = i < n ? keys[i] : 0ull;
    gprev[g] = (lane == 0 && i < n && i > 0) ? keys[i - 1] : 0ull;
  }
#pragma unroll
  for (int g = 0; g < kRunGroups; ++g) {
    const uint64_t base = round + (uint64_t)g * kRunBlock;
    const uint64_t i = base + threadIdx.x;
    const bool in = i < n;
    const unsigned long long key = gkey[g];
    const uint64_t p = key >> pshift;
    uint64_t pp = __shfl_up_sync(0xffffffffu, p, 1);
    if (lane == 0) pp = (in && i > 0) ? (gprev[g] >> pshift) : ~p;
    const bool bnd = in && (i == 0 || pp != p);  // a run starts here
    const unsigned bmask = __ballot_sync(0xffffffffu, bnd);
    uint32_t L = 0;
    if (bnd && i < c1) {  // a run of this chunk
      const unsigned above = bmask & ~((2u << lane) - 1u);
      if (above) {
        L = (uint32_t)(__ffs((int)above) - 1 - lane);
      } else {  // the warp's last run: it may go on past the warp
        L = (uint32_t)min((uint64_t)(32 - lane), n - i);
        while (i + L < n && L <= (uint32_t)kWarpRun && (keys[i + L] >> pshift) == p) ++L;
      }
    }
    const bool want_mid = L > (uint32_t)kShortRun && L <= (uint32_t)kWarpRun;
    const bool want_lng = L > (uint32_t)kWarpRun;
    const unsigned mm = __ballot_sync(0xffffffffu, want_mid);
    const unsigned lm = __ballot_sync(0xffffffffu, want_lng);
    uint32_t mb = 0, lb = 0;
    if (lane == 0) {
      if (mm) mb = atomicAdd(&s_mid, (uint32_t)__popc(mm));
      if (lm) lb = atomicAdd(&s_lng, (uint32_t)__popc(lm));
    }
    mb = __shfl_sync(0xffffffffu, mb, 0);
    lb = __shfl_sync(0xffffffffu, lb, 0);
    if (want_mid) {
      const uint64_t at = (uint64_t)mb + __popc(mm & lt);
      if (at < mid_cap)
        my_mid[at] = i;
      else
        atomicExch(fallback, 1u);
    }
    if (want_lng) {
      const uint64_t at = (uint64_t)lb + __popc(lm & lt);
      if (at < lng_cap)
        my_lng[at] = i;
      else
        atomicExch(fallback, 1u);
    }
    if (L < 2 || L > (uint32_t)kShortRun) continue;
    unsigned long long rk[kShortRun];
    bool ordered = true;
#pragma unroll
    for (int a = 0; a < kShortRun; ++a) {
      rk[a] = a == 0 ? key : (a < (int)L ? keys[i + a] : ~0ull);
      if (a > 0 && rk[a] < rk[a - 1]) ordered = false;  // (padding keys of all ones stay last)
    }
    if (ordered) continue;
    uint4 rc[kShortRun];
#pragma unroll
    for (int a = 0; a < kShortRun; ++a)
      rc[a] = a < (int)L ? counts[i + a] : make_uint4(0u, 0u, 0u, 0u);
    // a sorting network over the four places
#define DBG_CSWAP(x, y)                        \
  if (rk[y] < rk[x]) {                         \
    const unsigned long long tk = rk[x];       \
    rk[x] = rk[y];                             \
    rk[y] = tk;                                \
    const uint4 tc = rc[x];                    \
    rc[x] = rc[y];                             \
    rc[y] = tc;                                \
  }
    DBG_CSWAP(0, 1) DBG_CSWAP(2, 3) DBG_CSWAP(0, 2) DBG_CSWAP(1, 3) DBG_CSWAP(1, 2)
#undef DBG_CSWAP
#pragma unroll
    for (int a = 0; a < kShortRun; ++a) {
      if (a < (int)L) {
        keys[i + a] = rk[a];
        counts[i + a] = rc[a];
      }
    }
  }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mid_n[blockIdx.x] = (uint32_t)min((uint64_t)s_mid, mid_cap);
    lng_n[blockIdx.x] = (uint32_t)min((uint64_t)s_lng, lng_cap);
  }
}

// A warp per listed run of kShortRun + 1 .. kWarpRun keys (CTA b takes the
// runs of chunk b): lane a holds key a (padding lanes all ones), a bitonic
// sort over the warp's registers carries each key's lane of origin, and
// every lane then takes its counter row from that lane.
__global__ void __launch_bounds__(kRunBlock)
    k_sort_warp_runs(unsigned long long *keys, uint4 *counts, uint64_t n, int pshift,
                     const unsigned long long *mid, uint64_t mid_cap, const uint32_t *mid_n) {
  const int lane = threadIdx.x & 31;
  const uint32_t runs = mid_n[blockIdx.x];
  const unsigned long long *list = mid + (uint64_t)blockIdx.x * mid_cap;
  for (uint32_t r = threadIdx.x >> 5; r < runs; r += kRunBlock / 32) {
    const uint64_t i = list[r];
    const uint64_t p = keys[i] >> pshift;
    const bool in = i + lane < n && (keys[i + lane] >> pshift) == p;
    const unsigned L = __popc(__ballot_sync(0xffffffffu, in));  // (the run is contiguous from i)
    unsigned long long k = lane < (int)L ? keys[i + lane] : ~0ull;
    uint4 row = make_uint4(0u, 0u, 0u, 0u);
    if (lane < (int)L) row = counts[i + lane];
    int src = lane;
    for (int size = 2; size <= 32; size <<= 1) {
      for (int st = size >> 1; st > 0; st >>= 1) {
        const unsigned long long ok = __shfl_xor_sync(0xffffffffu, k, st);
        const int os = __shfl_xor_sync(0xffffffffu, src, st);
        const bool lower = (lane & st) == 0;        // this lane keeps the smaller key ...
        const bool up = (lane & size) == 0;         // ... of an ascending pair
        const bool take = lower == up ? ok < k : ok > k;
        if (take) {
          k = ok;
          src = os;
        }
      }
    }
    uint4 mine;
    mine.x = __shfl_sync(0xffffffffu, row.x, src);
    mine.y = __shfl_sync(0xffffffffu, row.y, src);
    mine.z = __shfl_sync(0xffffffffu, row.z, src);
    mine.w = __shfl_sync(0xffffffffu, row.w, src);
    if (lane < (int)L) {
      keys[i + lane] = k;
      counts[i + lane] = mine;
    }
  }
}

// A CTA per listed run of more than kWarpRun keys (CTAs take the chunks' list
// segments in turn): its keys and positions sorted in shared memory (bitonic,
// padded to a power of two with keys of all ones), then the keys and counter
// rows written back in that order.  A run longer than kMaxLongRun sets
// *fallback.
__global__ void __launch_bounds__(kLongBlock)
    k_sort_long_runs(unsigned long long *keys, uint4 *counts, uint64_t n, int pshift,
                     const unsigned long long *lng, uint64_t lng_cap, const uint32_t *lng_n,
                     int chunks, unsigned int *fallback) {
  __shared__ unsigned long long s_key[kMaxLongRun];
  __shared__ uint16_t s_pos[kMaxLongRun];
  __shared__ uint4 s_row[kMaxLongRun];
  __shared__ uint32_t s_len;
  for (int b = blockIdx.x; b < chunks; b += gridDim.x) {
    const uint32_t runs = lng_n[b];
    const unsigned long long *list = lng + (uint64_t)b * lng_cap;
    for (uint32_t r = 0; r < runs; ++r) {
      const uint64_t i = list[r];
      const uint64_t p = keys[i] >> pshift;
      if (threadIdx.x == 0) {
        uint64_t L = kWarpRun;  // (longer than that: it was listed)
        while (i + L < n && L <= kMaxLongRun && (keys[i + L] >> pshift) == p) ++L;
        s_len = (uint32_t)L;
        if (L > kMaxLongRun) atomicExch(fallback, 1u);
      }
      __syncthreads();
      const uint32_t L = s_len;
      if (L > kMaxLongRun) {
        __syncthreads();
        continue;
      }
      uint32_t P = 1;
      while (P < L) P <<= 1;
      for (uint32_t j = threadIdx.x; j < P; j += kLongBlock) {
        s_key[j] = j < L ? keys[i + j] : ~0ull;
        s_pos[j] = (uint16_t)j;
        if (j < L) s_row[j] = counts[i + j];
      }
      __syncthreads();
      for (uint32_t size = 2; size <= P; size <<= 1) {
        for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
          for (uint32_t j = threadIdx.x; j < P; j += kLongBlock) {
            const uint32_t o = j ^ stride;
            if (o > j) {
              const bool up = (j & size) == 0;
              const unsigned long long a = s_key[j], c = s_key[o];
              if ((a > c) == up) {
                s_key[j] = c;
                s_key[o] = a;
                const uint16_t t = s_pos[j];
                s_pos[j] = s_pos[o];
                s_pos[o] = t;
              }
            }
          }
          __syncthreads();
        }
      }
      for (uint32_t j = threadIdx.x; j < L; j += kLongBlock) {
        keys[i + j] = s_key[j];
        counts[i + j] = s_row[s_pos[j]];
      }
      __syncthreads();
    }
  }
}

// The sorted graph from the sorted slot indices: each slot read once (one
// sector), its key and counters written in order.
__global__ void k_gather_slots(const Slot *t, const uint32_t *__restrict__ idx,
                               unsigned long long *keys, uint4 *counts, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const uint4 *sl = reinterpret_cast<const uint4 *>(t + __ldcs(idx + i));
    const uint4 a = sl[0], b = sl[1];  // key lo, key hi, cnt0, cnt1 | cnt2, cnt3, pad
    if (keys) __stcs(keys + i, (unsigned long long)a.x | ((unsigned long long)a.y << 32));
    if (counts) __stcs(counts + i, make_uint4(a.z, a.w, b.x, b.y));
  }
}

struct Guard {
  int prev = -1;
  bool changed = false;
  cudaError_t err = cudaSuccess;
  explicit Guard(int dev) {
    err = cudaGetDevice(&prev);
    if (err == cudaSuccess && prev != dev) {
      err = cudaSetDevice(dev);
      changed = err == cudaSuccess;
    }
  }
  ~Guard() {
    if (changed) cudaSetDevice(prev);
  }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool is_device_ptr(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // (an unregistered host pointer on older runtimes)
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The sort's temporary bytes for D (key, slot index) pairs of type I.
template <class I>
int sort_temp_bytes(uint64_t D, int end_bit, size_t &temp_bytes) {
  temp_bytes = 0;
  cub::DoubleBuffer<unsigned long long> dk(nullptr, nullptr);
  cub::DoubleBuffer<I> dv(nullptr, nullptr);
  DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, dk, dv, (int64_t)D, 0, end_bit,
                                         (cudaStream_t)0));
  return DBG_OK;
}

// Scratch of an in-place export: [count][sort temp][final indices].
template <class I>
int in_place_scratch_bytes(uint64_t D, int end_bit, uint64_t &bytes) {
  size_t temp = 0;
  DBG_TRY(sort_temp_bytes<I>(D, end_bit, temp));
  bytes = 256 + align256(temp) + align256(D * sizeof(I));
  return DBG_OK;
}

// The export of D vertices with slot indices of type I (k <= 32).  `caller`
// (with `caller_bytes`): scratch the caller owns, used instead of the pool
// (in-place outputs only).
template <class I>
int export_pairs(dbg_handle h, uint64_t D, uint64_t *keys_out, uint32_t *counts_out,
                 cudaStream_t s, void *caller = nullptr, uint64_t caller_bytes = 0) {
  const int end_bit = 2 * (h->k - 1);
  // in place: both outputs on the device, 16-byte aligned (keys_out needs 8,
  // the uint4 rows of counts_out 16), and the index buffers fit beside the
  // second key buffer in counts_out
  const bool in_place = sizeof(I) == 4 && is_device_ptr(keys_out) && is_device_ptr(counts_out) &&
                        ((uintptr_t)keys_out & 15u) == 0 && ((uintptr_t)counts_out & 15u) == 0;
  if (caller && !in_place) return DBG_ERR_INVALID_ARG;
  size_t temp_bytes = 0;
  DBG_TRY(sort_temp_bytes<I>(D, end_bit, temp_bytes));
  const size_t kb = align256(D * sizeof(unsigned long long));
  const size_t ib = align256(D * sizeof(I));
  const size_t cb = align256(D * sizeof(uint4));
  // scratch: [count][sort temp], then in place [final indices], otherwise
  // [keys a][keys b][indices a][indices b][counters]
  const size_t head = 256 + align256(temp_bytes);
  const size_t total = head + (in_place ? ib : 2 * kb + 2 * ib + cb);
  char *buf = nullptr;
  if (caller) {
    if (caller_bytes < total || ((uintptr_t)caller & 255u)) return DBG_ERR_INVALID_ARG;
    buf = static_cast<char *>(caller);
  } else {
    DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), total, s));
  }
  unsigned long long *count = reinterpret_cast<unsigned long long *>(buf);
  void *temp = buf + 256;
  I *idx_final = reinterpret_cast<I *>(buf + head);  // (in place only)
  unsigned long long *keys_a, *keys_b;
  I *idx_a, *idx_b;
  uint4 *counts;
  if (in_place) {
    char *c = reinterpret_cast<char *>(counts_out);
    keys_a = reinterpret_cast<unsigned long long *>(keys_out);
    keys_b = reinterpret_cast<unsigned long long *>(c);
    idx_a = reinterpret_cast<I *>(c + D * 8);
    idx_b = reinterpret_cast<I *>(c + D * 12);
    counts = reinterpret_cast<uint4 *>(counts_out);
  } else {
    char *p = buf + head;
    keys_a = reinterpret_cast<unsigned long long *>(p);
    keys_b = reinterpret_cast<unsigned long long *>(p + kb);
    idx_a = reinterpret_cast<I *>(p + 2 * kb);
    idx_b = reinterpret_cast<I *>(p + 2 * kb + ib);
    counts = reinterpret_cast<uint4 *>(p + 2 * kb + 2 * ib);
  }

  int rc = DBG_OK;
  do {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    const int sms = std::max(1, h->sm_count);
    k_compact<I><<<sms * 8, kCompactBlock, 0, s>>>(h->table, h->n_slots, keys_a, idx_a, count, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_compact"); break; }
    cub::DoubleBuffer<unsigned long long> dk(keys_a, keys_b);
    cub::DoubleBuffer<I> dv(idx_a, idx_b);
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, dk, dv, (int64_t)D, 0, end_bit, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceRadixSort::SortPairs"); break; }
    // in place, the gather writes counts_out, which holds the sorted indices
    // (and maybe the sorted keys): move them out first
    const I *gidx = dv.Current();
    if (in_place) {
      e = cudaMemcpyAsync(idx_final, dv.Current(), D * sizeof(I), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(indices)"); break; }
      gidx = idx_final;
    }
    if (keys_out && (!in_place || dk.Current() != keys_a)) {
      e = cudaMemcpyAsync(keys_out, dk.Current(), D * sizeof(uint64_t), cudaMemcpyDefault, s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(keys)"); break; }
    }
    if (counts_out) {
      k_gather<I><<<sms * 8, 256, 0, s>>>(h->table, gidx, counts, D);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_gather"); break; }
      if (!in_place) {
        e = cudaMemcpyAsync(counts_out, counts, D * sizeof(uint4), cudaMemcpyDefault, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
      }
    }
  } while (0);
  cudaError_t e = caller ? cudaSuccess : cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}

// Scratch of the prefix-sort export: [count, flag][run list counts][sort
// temp][sorted indices][run lists], and without in-place outputs [prefix a]
// [index a][prefix b][index b][keys][counters].
struct PrefixScratch {
  size_t temp, head, wb, lists, total;
};

int prefix_scratch(int k, uint64_t D, bool in_place, PrefixScratch &ps) {
  const int bits = 2 * (k - 1);
  size_t temp = 0;
  cub::DoubleBuffer<uint32_t> dk(nullptr, nullptr), dv(nullptr, nullptr);
  DBG_CK(cub::DeviceRadixSort::SortPairs(nullptr, temp, dk, dv, (int64_t)D, 0,
                                         bits > 32 ? 32 : bits, (cudaStream_t)0));
  ps.temp = temp;
  ps.head = 256 + align256(2 * (size_t)kRunCtas * sizeof(uint32_t)) + align256(temp);
  ps.wb = align256(D * sizeof(uint32_t));
  ps.lists = align256(run_lists(D).bytes());
  ps.total = ps.head + ps.wb + ps.lists +
             (in_place ? 0 : 4 * ps.wb + align256(D * 8) + align256(D * sizeof(uint4)));
  return DBG_OK;
}

bool in_place_outputs(const uint64_t *keys_out, const uint32_t *counts_out) {
  return is_device_ptr(keys_out) && is_device_ptr(counts_out) &&
         ((uintptr_t)keys_out & 15u) == 0 && ((uintptr_t)counts_out & 15u) == 0;
}

// Compaction of the prefix export into in-place outputs of `stride` rows,
// counting the occupied slots as it goes (no separate counting pass): at most
// `stride` (prefix, index) pairs are written -- prefixes at keys_out as 32-bit
// words, indices after them -- and *D_out receives the count.  Returns the
// sticky status (or NEEDS_GROW) instead when the graph has one.
int compact_counted(dbg_handle h, uint64_t *keys_out, uint64_t stride, uint64_t *D_out,
                    cudaStream_t s) {
  const int bits = 2 * (h->k - 1);
  const int pshift = bits > 32 ? bits - 32 : 0;
  uint32_t *pa = reinterpret_cast<uint32_t *>(keys_out);
  DBG_CK(cudaMemsetAsync(h->d_acc, 0, sizeof(unsigned long long), s));
  const int sms = std::max(1, h->sm_count);
  k_compact_prefix<<<sms * 8, kCompactBlock, 0, s>>>(h->table, h->n_slots, pshift, pa, pa + stride,
                                                     h->d_acc, stride);
  DBG_CK(cudaGetLastError());
  unsigned long long D = 0, spilled = 0;
  uint32_t status = 0;
  DBG_CK(cudaMemcpyAsync(&D, h->d_acc, sizeof(D), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaMemcpyAsync(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaMemcpyAsync(&spilled, h->d_spill_count, sizeof(spilled), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaStreamSynchronize(s));
  if (status != DBG_OK) return (int)status;
  if (spilled > 0) return DBG_ERR_NEEDS_GROW;
  *D_out = D;
  return DBG_OK;
}

// The prefix-sort export of D vertices (tables of at most 2^32 slots).
// Buffers: two (prefix, index) pairs for the sort, the sorted indices, the
// sort's temporary space, a counter, the long-run flag and the run lists.  In
// place (both outputs 16-byte aligned device buffers) the pairs live in
// keys_out (8 bytes a row) and counts_out, and the gather writes the outputs
// directly; otherwise everything is temporary.  `stride` (in place): the rows
// the pair layout assumes (D when 0); `compacted`: compact_counted has
// already written the pairs with that stride.  Returns DBG_ERR_CAPACITY (not
// a graph error: the caller falls back to the full-width sort) when a run of
// equal prefixes is too long.
int export_prefix(dbg_handle h, uint64_t D, uint64_t *keys_out, uint32_t *counts_out,
                  cudaStream_t s, void *caller, uint64_t caller_bytes, uint64_t stride = 0,
                  bool compacted = false) {
  const int bits = 2 * (h->k - 1);
  const int pshift = bits > 32 ? bits - 32 : 0;
  const int pbits = bits > 32 ? 32 : bits;
  const bool in_place = in_place_outputs(keys_out, counts_out);
  if ((caller || compacted) && !in_place) return DBG_ERR_INVALID_ARG;
  if (stride == 0) stride = D;
  PrefixScratch ps{};
  DBG_TRY(prefix_scratch(h->k, D, in_place, ps));
  // one wave of the run pass: as many CTAs as fit on the device at once
  int run_per_sm = 0;
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&run_per_sm, k_sort_runs, kRunBlock, 0));
  RunLists rl =
      run_lists(D, std::max(1, std::min(kRunCtas, std::max(1, run_per_sm) * std::max(1, h->sm_count))));
  if (rl.bytes() > run_lists(D).bytes()) rl = run_lists(D);  // (chunk rounding: the sized layout)
  char *buf = nullptr;
  if (caller) {
    if (caller_bytes < ps.total || ((uintptr_t)caller & 255u)) return DBG_ERR_INVALID_ARG;
    buf = static_cast<char *>(caller);
  } else {
    DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), ps.total, s));
  }
  unsigned long long *count = reinterpret_cast<unsigned long long *>(buf);
  unsigned int *fallback = reinterpret_cast<unsigned int *>(buf + 8);
  uint32_t *mid_n = reinterpret_cast<uint32_t *>(buf + 256);
  uint32_t *lng_n = mid_n + kRunCtas;
  void *temp = buf + ps.head - align256(ps.temp);
  uint32_t *idx_final = reinterpret_cast<uint32_t *>(buf + ps.head);
  unsigned long long *mid = reinterpret_cast<unsigned long long *>(buf + ps.head + ps.wb);
  unsigned long long *lng = mid + (uint64_t)rl.ctas * rl.mid_cap;
  uint32_t *pa, *ia, *pb, *ib;
  unsigned long long *keys;
  uint4 *counts;
  if (in_place) {
    pa = reinterpret_cast<uint32_t *>(keys_out);
    ia = pa + stride;
    pb = reinterpret_cast<uint32_t *>(counts_out);
    ib = pb + stride;
    keys = reinterpret_cast<unsigned long long *>(keys_out);
    counts = reinterpret_cast<uint4 *>(counts_out);
  } else {
    char *p = buf + ps.head + ps.wb + ps.lists;
    pa = reinterpret_cast<uint32_t *>(p);
    ia = reinterpret_cast<uint32_t *>(p + ps.wb);
    pb = reinterpret_cast<uint32_t *>(p + 2 * ps.wb);
    ib = reinterpret_cast<uint32_t *>(p + 3 * ps.wb);
    keys = reinterpret_cast<unsigned long long *>(p + 4 * ps.wb);
    counts = reinterpret_cast<uint4 *>(p + 4 * ps.wb + align256(D * 8));
  }

  int rc = DBG_OK;
  unsigned int fallback_host = 0;
  do {
    cudaError_t e = cudaMemsetAsync(buf, 0, 16, s);  // count, flag
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    const int sms = std::max(1, h->sm_count);
    if (!compacted) {
      k_compact_prefix<<<sms * 8, kCompactBlock, 0, s>>>(h->table, h->n_slots, pshift, pa, ia,
                                                         count, D);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_compact_prefix"); break; }
    }
    cub::DoubleBuffer<uint32_t> dk(pa, pb), dv(ia, ib);
    size_t temp_bytes = ps.temp;
    e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, dk, dv, (int64_t)D, 0, pbits, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceRadixSort::SortPairs"); break; }
    // the gather overwrites the buffers the sorted indices sit in: move them out
    e = cudaMemcpyAsync(idx_final, dv.Current(), D * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(indices)"); break; }
    k_gather_slots<<<sms * 8, 256, 0, s>>>(h->table, idx_final, keys, counts, D);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_gather_slots"); break; }
    if (pshift > 0) {  // the runs of equal prefixes, in key order
      k_sort_runs<<<rl.ctas, kRunBlock, 0, s>>>(keys, counts, D, pshift, rl.chunk, mid, rl.mid_cap,
                                                mid_n, lng, rl.lng_cap, lng_n, fallback);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_sort_runs"); break; }
      k_sort_warp_runs<<<rl.ctas, kRunBlock, 0, s>>>(keys, counts, D, pshift, mid, rl.mid_cap,
                                                     mid_n);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_sort_warp_runs"); break; }
      k_sort_long_runs<<<std::min(rl.ctas, sms * 4), kLongBlock, 0, s>>>(
          keys, counts, D, pshift, lng, rl.lng_cap, lng_n, rl.ctas, fallback);
      e = cudaGetLastError();
      if (e != cudaSuccess) { rc = cuda_fail(e, "k_sort_long_runs"); break; }
      e = cudaMemcpyAsync(&fallback_host, fallback, sizeof(fallback_host), cudaMemcpyDeviceToHost,
                          s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) { rc = cuda_fail(e, "fall-back flag"); break; }
      if (fallback_host) { rc = DBG_ERR_CAPACITY; break; }
    }
    if (!in_place) {
      if (keys_out) {
        e = cudaMemcpyAsync(keys_out, keys, D * sizeof(uint64_t), cudaMemcpyDefault, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(keys)"); break; }
      }
      if (counts_out) {
        e = cudaMemcpyAsync(counts_out, counts, D * sizeof(uint4), cudaMemcpyDefault, s);
        if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(counts)"); break; }
      }
    }
  } while (0);
  cudaError_t e = caller ? cudaSuccess : cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  return rc;
}

// Scratch of an in-place prefix export (see export_prefix).
int prefix_scratch_bytes(int k, uint64_t D, uint64_t &bytes) {
  PrefixScratch ps{};
  DBG_TRY(prefix_scratch(k, D, true, ps));
  bytes = ps.total;
  return DBG_OK;
}

}  // namespace
}  // namespace dbg

extern "C" int dbg_export_sorted(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                                 uint64_t max_n, uint64_t *n_out, void *stream) {
  using namespace dbg;
  if (!h || !n_out) return DBG_ERR_INVALID_ARG;
  Guard g(h->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  uint64_t D = 0;
  int st;
  if (h->k <= 32 && h->n_slots <= 0xFFFFFFFFull && max_n > 0 &&
      in_place_outputs(keys_out, counts_out)) {
    // in place: the compaction into the outputs counts the vertices itself
    st = compact_counted(h, keys_out, max_n, &D, s);
    if (st != DBG_OK) return st;
    *n_out = D;
    if (D > max_n) return DBG_ERR_BUFFER_TOO_SMALL;
    if (D == 0) return DBG_OK;
    st = export_prefix(h, D, keys_out, counts_out, s, nullptr, 0, max_n, true);
    if (st != DBG_ERR_CAPACITY) return st;  // (a long run of equal prefixes: full width)
    return export_pairs<uint32_t>(h, D, keys_out, counts_out, s);
  }
  st = dbg_stats(h, &D, nullptr, stream);
  if (st != DBG_OK) return st;
  *n_out = D;
  if (D > max_n) return DBG_ERR_BUFFER_TOO_SMALL;
  if (D == 0) return DBG_OK;
  if (h->k > 32) return export_sorted_wide(h, D, keys_out, counts_out, s);
  if (h->n_slots <= 0xFFFFFFFFull) {
    st = export_prefix(h, D, keys_out, counts_out, s, nullptr, 0);
    if (st != DBG_ERR_CAPACITY) return st;  // (a long run of equal prefixes: full width)
    return export_pairs<uint32_t>(h, D, keys_out, counts_out, s);
  }
  return export_pairs<unsigned long long>(h, D, keys_out, counts_out, s);
}

extern "C" uint64_t dbg_export_scratch_bytes(int k, uint64_t n_vertices, uint64_t n_slots) {
  using namespace dbg;
  if (k < 2 || k > 32 || n_slots > 0xFFFFFFFFull) return 0;
  const uint64_t D = std::max<uint64_t>(n_vertices, 1);
  uint64_t a = 0, b = 0;  // the prefix sort's, and the full-width fall-back's
  if (prefix_scratch_bytes(k, D, a) != DBG_OK) return 0;
  if (in_place_scratch_bytes<uint32_t>(D, 2 * (k - 1), b) != DBG_OK) return 0;
  return std::max(a, b);
}

extern "C" int dbg_export_sorted_with(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                                      uint64_t max_n, uint64_t *n_out, void *scratch,
                                      uint64_t scratch_bytes, void *stream) {
  using namespace dbg;
  if (!h || !n_out || h->k > 32 || h->n_slots > 0xFFFFFFFFull) return DBG_ERR_INVALID_ARG;
  Guard g(h->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint64_t D = 0;
  const bool counted = max_n > 0 && scratch && in_place_outputs(keys_out, counts_out);
  int st = counted ? compact_counted(h, keys_out, max_n, &D, s) : dbg_stats(h, &D, nullptr, stream);
  if (st != DBG_OK) return st;
  *n_out = D;
  if (D > max_n) return DBG_ERR_BUFFER_TOO_SMALL;
  if (D == 0) return DBG_OK;
  if (!keys_out || !counts_out || !scratch) return DBG_ERR_INVALID_ARG;
  st = export_prefix(h, D, keys_out, counts_out, s, scratch, scratch_bytes, counted ? max_n : 0,
                     counted);
  if (st != DBG_ERR_CAPACITY) return st;  // (a long run of equal prefixes: full width)
  return export_pairs<uint32_t>(h, D, keys_out, counts_out, s, scratch, scratch_bytes);
}
