// Downstream of the build: normalization (Section "Normalization of graph")
// and contigs (Section "Finding contigs", Alg. 5 findContigs with makePath),
// as passes over the resident table.
//
// Normalization replaces every counter c by floor(c / divisor + 0.5) in IEEE
// double (round to nearest, halves up), capped at 2^32 - 1: the counters stay
// integers, an error k-mer seen once falls to 0 and a genomic k-mer seen
// about `divisor` times stays 1.
//
// Contigs.  An outgoing edge of a vertex is a label with a nonzero counter.
// The first flag of the paper (no edge points to the vertex) is recomputed
// from the counters as they are: every slot clears the mark word in its
// padding, then every edge marks its target.  A vertex starts contigs when
// its first flag is set or it has not exactly one outgoing edge, one contig
// per outgoing edge; a contig follows edges while the vertex it reaches has
// exactly one outgoing edge, and stops on reaching a vertex it has already
// visited (keeping the edge into it).  Contigs are listed by (start key,
// label): the start edges are emitted in any order and radix-sorted.
//
// One thread walks one contig.  The walk first measures the contig: Brent's
// cycle detection (R. P. Brent, "An improved Monte Carlo factorization
// algorithm", BIT 20, 1980) over the single-exit successor map finds the
// first repeated vertex, if any, with O(1) state; a second walk writes the
// bases at the offset an exclusive scan of the lengths gives.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include <math.h>

#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

constexpr uint64_t kNotFound = ~0ull;

struct View {
  Slot *t;
  uint64_t n;
  uint32_t max_probes;
  uint64_t mask;  // 2(k-1) low bits
  uint32_t *status;
};

// The slot of an existing key (the table is quiescent), or kNotFound.
__device__ __forceinline__ uint64_t find_key(const View &v, uint64_t key) {
  uint64_t s = home_slot(key, v.n);
  for (uint32_t p = 0; p < v.max_probes; ++p) {
    const unsigned long long cur = v.t[s].key;
    if (cur == key) return s;
    if (cur == kEmpty) return kNotFound;
    if (++s == v.n) s = 0;
  }
  return kNotFound;
}

// Out-degree of a slot's counters and its lowest label with a nonzero counter.
__device__ __forceinline__ int out_degree(const Slot &sl, uint32_t &label) {
  int d = 0;
  label = 4;
#pragma unroll
  for (int b = 3; b >= 0; --b)
    if (sl.cnt[b]) {
      ++d;
      label = (uint32_t)b;
    }
  return d;
}

// (cnt0: the first counter's 32-bit word in the slot -- 2, or 4 for k > 32)
__global__ void k_normalize(Slot *t, uint64_t n, double divisor, int cnt0) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    if (t[i].key == kEmpty) continue;
    uint32_t *cnt = reinterpret_cast<uint32_t *>(t + i) + cnt0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const uint32_t c = cnt[b];
      if (!c) continue;
      const double q = floor((double)c / divisor + 0.5);
      cnt[b] = q >= 4294967295.0 ? 0xffffffffu : (uint32_t)q;
    }
  }
}

// pad[0] of every slot := 0 (the "has an incoming edge" mark).
__global__ void k_clear_marks(Slot *t, uint64_t n) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    t[i].pad[0] = 0u;
}

// Every edge marks its target.
__global__ void k_mark_targets(View v) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < v.n; i += stride) {
    const unsigned long long key = v.t[i].key;
    if (key == kEmpty) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      if (!v.t[i].cnt[b]) continue;
      const uint64_t s = find_key(v, ((key << 2) | (uint64_t)b) & v.mask);
      if (s == kNotFound) {
        atomicCAS(v.status, 0u, (uint32_t)DBG_ERR_CAPACITY);  // a target is missing
        continue;
      }
      if (v.t[s].pad[0] == 0u) atomicOr(&v.t[s].pad[0], 1u);
    }
  }
}

// Start edges: (key << 2 | label) for every outgoing edge of every vertex
// that is first or has not exactly one outgoing edge.  With out == nullptr
// only counts them.  Warps walk 32 consecutive slots and reserve their edges
// with one atomic.
__global__ void k_start_edges(View v, unsigned long long *out, unsigned long long *count,
                              uint64_t cap) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (((uint64_t)blockIdx.x * blockDim.x) + threadIdx.x) >> 5;
  for (uint64_t base = w0 * 32; base < v.n; base += warps * 32) {
    const uint64_t i = base + lane;
    unsigned long long key = kEmpty;
    uint32_t d = 0;
    if (i < v.n) {
      key = v.t[i].key;
      if (key != kEmpty) {
        uint32_t label;
        d = (uint32_t)out_degree(v.t[i], label);
        if (d == 1 && v.t[i].pad[0] != 0u) d = 0;  // single exit, not first: no start
      }
    }
    uint32_t incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long at = 0;
    if (lane == 31 && total) at = atomicAdd(count, (unsigned long long)total);
    at = __shfl_sync(0xffffffffu, at, 31) + (incl - d);
    if (!out || !d) continue;
    for (int b = 0; b < 4; ++b)
      if (v.t[i].cnt[b] && at < cap) out[at++] = (key << 2) | (unsigned long long)b;
  }
}

// Next vertex of a single-exit vertex, or kNotFound when the vertex (slot s)
// does not have exactly one outgoing edge.  *base receives the label taken.
__device__ __forceinline__ uint64_t step(const View &v, uint64_t s, uint32_t *base) {
  uint32_t label;
  if (out_degree(v.t[s], label) != 1) return kNotFound;
  *base = label;
  const uint64_t nx = find_key(v, ((v.t[s].key << 2) | label) & v.mask);
  if (nx == kNotFound) atomicCAS(v.status, 0u, (uint32_t)DBG_ERR_CAPACITY);
  return nx;
}

// Number of edges of the contig that starts with edge e = (key << 2) | label.
__device__ uint64_t contig_edges(const View &v, unsigned long long e, uint64_t guard) {
  uint32_t b;
  const uint64_t x0 = find_key(v, e & v.mask);
  if (x0 == kNotFound) {
    atomicCAS(v.status, 0u, (uint32_t)DBG_ERR_CAPACITY);  // a target is missing
    return 1;
  }
  // Brent: the hare walks; the tortoise jumps to the hare at powers of two
  uint64_t tortoise = x0, hare = step(v, x0, &b);
  if (hare == kNotFound) return 1;  // x0 is a branch or a dead end
  uint64_t taken = 1, power = 1, lam = 1;
  while (tortoise != hare) {
    if (taken > guard) {  // cannot happen: a walk repeats within n steps
      atomicCAS(v.status, 0u, (uint32_t)DBG_ERR_CAPACITY);
      return 1;
    }
    if (power == lam) {
      tortoise = hare;
      power <<= 1;
      lam = 0;
    }
    const uint64_t nx = step(v, hare, &b);
    if (nx == kNotFound) return 1 + taken;  // ends at the hare, `taken` steps past x0
    hare = nx;
    ++taken;
    ++lam;
  }
  // a cycle of length lam; mu = index of its first vertex along x0, x1, ...
  // (every vertex up to x_{mu+lam} has one exit: the hare passed them all)
  uint64_t a = x0, c = x0;
  for (uint64_t i = 0; i < lam && c != kNotFound; ++i) c = step(v, c, &b);
  uint64_t mu = 0;
  while (a != c && a != kNotFound && c != kNotFound && mu <= guard) {
    a = step(v, a, &b);
    c = step(v, c, &b);
    ++mu;
  }
  if (a != c) {
    atomicCAS(v.status, 0u, (uint32_t)DBG_ERR_CAPACITY);
    return 1;
  }
  return 1 + mu + lam;  // the walk arrives at x_mu again after mu + lam steps
}

__global__ void k_contig_lengths(View v, const unsigned long long *starts, uint64_t n_starts,
                                 int m, uint64_t guard, unsigned long long *len) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_starts; i += stride)
    len[i] = (unsigned long long)m + contig_edges(v, starts[i], guard);
  if (blockIdx.x == 0 && threadIdx.x == 0) len[n_starts] = 0;
}

__global__ void k_contig_write(View v, const unsigned long long *starts, uint64_t n_starts, int m,
                               const unsigned long long *off, const unsigned long long *len,
                               char *out) {
  const char letter[4] = {'A', 'C', 'G', 'T'};
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_starts; i += stride) {
    const unsigned long long e = starts[i];
    const unsigned long long key = e >> 2;
    char *o = out + off[i];
    for (int j = 0; j < m; ++j) o[j] = letter[(key >> (2 * (m - 1 - j))) & 3ull];
    o[m] = letter[e & 3ull];
    const uint64_t edges = len[i] - (unsigned long long)m;
    uint64_t s = find_key(v, e & v.mask);
    for (uint64_t j = 1; j < edges && s != kNotFound; ++j) {
      uint32_t b = 0;
      s = step(v, s, &b);
      o[m + j] = letter[b];
    }
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

int read_status(dbg_handle h, cudaStream_t s) {
  uint32_t st = 0;
  DBG_CK(cudaMemcpyAsync(&st, h->d_status, sizeof(st), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaStreamSynchronize(s));
  return (int)st;
}

}  // namespace
}  // namespace dbg

extern "C" int dbg_normalize(dbg_handle h, double divisor, void *stream) {
  using namespace dbg;
  if (!h || !(divisor > 0.0) || !isfinite(divisor)) return DBG_ERR_INVALID_ARG;
  h->built_counts = false;  // the counters change
  Guard g(h->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int st = dbg_get_status(h, stream);  // complete graphs only
  if (st != DBG_OK) return st;
  k_normalize<<<std::max(1, h->sm_count) * 8, 256, 0, s>>>(h->table, h->n_slots, divisor,
                                                             h->k > 32 ? 4 : 2);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

extern "C" int dbg_find_contigs(dbg_handle h, char *bases_out, uint64_t max_bases,
                                uint64_t *offsets_out, uint64_t max_contigs, uint64_t *n_contigs,
                                uint64_t *n_bases, void *stream) {
  using namespace dbg;
  if (!h || !n_contigs || !n_bases || h->k > 32) return DBG_ERR_INVALID_ARG;
  h->built_counts = false;  // (this pass takes the stats accumulators as scratch)
  Guard g(h->device);
  if (g.err != cudaSuccess) return cuda_fail(g.err, "cudaSetDevice");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int st = dbg_get_status(h, stream);
  if (st != DBG_OK) return st;

  const int m = h->k - 1;
  const View v{h->table, h->n_slots, h->max_probes,
               m >= 32 ? ~0ull : ((1ull << (2 * m)) - 1ull), h->d_status};
  const int grid = std::max(1, h->sm_count) * 8;
  unsigned long long *count = h->d_acc;  // the handle's stats accumulator, free here
  k_clear_marks<<<grid, 256, 0, s>>>(h->table, h->n_slots);
  DBG_CK(cudaGetLastError());
  k_mark_targets<<<grid, 256, 0, s>>>(v);
  DBG_CK(cudaGetLastError());
  DBG_CK(cudaMemsetAsync(count, 0, sizeof(unsigned long long), s));
  k_start_edges<<<grid, 256, 0, s>>>(v, nullptr, count, 0);
  DBG_CK(cudaGetLastError());
  unsigned long long S = 0;
  DBG_CK(cudaMemcpyAsync(&S, count, sizeof(S), cudaMemcpyDeviceToHost, s));
  DBG_CK(cudaStreamSynchronize(s));
  st = read_status(h, s);
  if (st != DBG_OK) return st;
  *n_contigs = S;
  *n_bases = 0;
  if (S == 0) {
    if (offsets_out)
      DBG_CK(cudaMemcpyAsync(offsets_out, n_bases, sizeof(uint64_t), cudaMemcpyDefault, s));
    DBG_CK(cudaStreamSynchronize(s));
    return DBG_OK;
  }

  size_t sort_bytes = 0, scan_bytes = 0;
  DBG_CK(cub::DeviceRadixSort::SortKeys(nullptr, sort_bytes, (unsigned long long *)nullptr,
                                        (unsigned long long *)nullptr, (int64_t)S, 0, 2 * m + 2,
                                        s));
  DBG_CK(cub::DeviceScan::ExclusiveSum(nullptr, scan_bytes, (unsigned long long *)nullptr,
                                       (unsigned long long *)nullptr, (int64_t)(S + 1), s));
  const size_t eb = align256((S + 1) * sizeof(unsigned long long));
  const size_t total = 4 * eb + align256(std::max(sort_bytes, scan_bytes));
  char *buf = nullptr;
  DBG_TRY(scratch_alloc(reinterpret_cast<void **>(&buf), total, s));
  unsigned long long *starts_a = reinterpret_cast<unsigned long long *>(buf);
  unsigned long long *starts_b = reinterpret_cast<unsigned long long *>(buf + eb);
  unsigned long long *len = reinterpret_cast<unsigned long long *>(buf + 2 * eb);
  unsigned long long *off = reinterpret_cast<unsigned long long *>(buf + 3 * eb);
  void *temp = buf + 4 * eb;
  char *chars = nullptr;
  int rc = DBG_OK;
  do {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemsetAsync"); break; }
    k_start_edges<<<grid, 256, 0, s>>>(v, starts_a, count, S);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_start_edges"); break; }
    e = cub::DeviceRadixSort::SortKeys(temp, sort_bytes, starts_a, starts_b, (int64_t)S, 0,
                                       2 * m + 2, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceRadixSort::SortKeys"); break; }
    const uint64_t guard = 4 * h->n_slots + 64;
    k_contig_lengths<<<grid, 256, 0, s>>>(v, starts_b, S, m, guard, len);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_contig_lengths"); break; }
    e = cub::DeviceScan::ExclusiveSum(temp, scan_bytes, len, off, (int64_t)(S + 1), s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "DeviceScan::ExclusiveSum"); break; }
    unsigned long long B = 0;
    e = cudaMemcpyAsync(&B, off + S, sizeof(B), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "contig lengths"); break; }
    *n_bases = B;
    rc = read_status(h, s);
    if (rc != DBG_OK) break;
    if (!bases_out || !offsets_out || S > max_contigs || B > max_bases) {
      rc = DBG_ERR_BUFFER_TOO_SMALL;
      break;
    }
    rc = scratch_alloc(reinterpret_cast<void **>(&chars), std::max<uint64_t>(B, 1), s);
    if (rc != DBG_OK) break;
    k_contig_write<<<grid, 256, 0, s>>>(v, starts_b, S, m, off, len, chars);
    e = cudaGetLastError();
    if (e != cudaSuccess) { rc = cuda_fail(e, "k_contig_write"); break; }
    e = cudaMemcpyAsync(offsets_out, off, (S + 1) * sizeof(uint64_t), cudaMemcpyDefault, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(bases_out, chars, B, cudaMemcpyDefault, s);
    if (e != cudaSuccess) { rc = cuda_fail(e, "cudaMemcpyAsync(contigs)"); break; }
  } while (0);
  if (chars) cudaFreeAsync(chars, s);
  cudaError_t e = cudaFreeAsync(buf, s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaFreeAsync");
  e = cudaStreamSynchronize(s);
  if (rc == DBG_OK && e != cudaSuccess) rc = cuda_fail(e, "cudaStreamSynchronize");
  if (rc == DBG_OK) rc = read_status(h, s);
  return rc;
}
