// Grow-and-rebuild: move a graph into a larger table and replay the vertex
// positions that were spilled because the old table had no room for them.
//
// Exactness: slots never become empty again, so once a key fails to find a
// slot within max_probes every later position of that key fails too; a key
// is therefore either in the table with all its counts or not in it with
// every one of its (remaining) positions spilled.  Re-inserting every
// occupied slot with its four counters, then every spilled position, gives
// the graph a large enough table would have built.
#include <algorithm>

#include "dbg_internal.cuh"

namespace dbg {
namespace {

// Every occupied slot of `old`, with its counters, into `nt`.
__global__ void k_rehash(const Slot *old, uint64_t n_old, Slot *nt, uint64_t n_new,
                         uint32_t max_probes, uint32_t *fail) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_old; i += stride) {
    const unsigned long long key = old[i].key;
    if (key == kEmpty) continue;
    uint64_t s;
    if (!find_or_claim(nt, n_new, max_probes, key, s)) {
      atomicExch(fail, 1u);
      continue;
    }
#pragma unroll
    for (int b = 0; b < 4; ++b)
      if (old[i].cnt[b]) atomicAdd(&nt[s].cnt[b], old[i].cnt[b]);
  }
}

// Every spilled vertex position into `nt`.
__global__ void k_replay(const SpillRecord *sp, uint64_t n, Slot *nt, uint64_t n_new,
                         uint32_t max_probes, uint32_t *fail) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const unsigned long long key = sp[i].key, info = sp[i].info;
    uint64_t s;
    if (!find_or_claim(nt, n_new, max_probes, key, s)) {
      atomicExch(fail, 1u);
      continue;
    }
    if (info & 4ull) atomicAdd(&nt[s].cnt[info & 3ull], 1u);
  }
}

}  // namespace

int launch_grow(dbg_handle h, uint64_t new_capacity, cudaStream_t s) {
  DBG_CK(cudaStreamSynchronize(s));
  uint32_t status = 0;
  unsigned long long spilled = 0;
  DBG_CK(cudaMemcpy(&status, h->d_status, sizeof(status), cudaMemcpyDeviceToHost));
  DBG_CK(cudaMemcpy(&spilled, h->d_spill_count, sizeof(spilled), cudaMemcpyDeviceToHost));
  if (status != DBG_OK) return (int)status;
  if (spilled > h->spill_cap) return DBG_ERR_CAPACITY;  // (the status says so as well)
  if (new_capacity == 0) new_capacity = 2 * h->n_slots;
  if (new_capacity > (~0ull / sizeof(Slot))) return DBG_ERR_INVALID_ARG;

  Slot *nt = nullptr;
  cudaError_t e = cudaMalloc(&nt, new_capacity * sizeof(Slot));
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(grown table)");
  int st = launch_table_init(nt, new_capacity, s);
  // a failure flag of its own, so a too-small new table leaves the graph as it was
  uint32_t *fail = reinterpret_cast<uint32_t *>(h->d_acc);
  const uint32_t probes = h->max_probes_auto
                              ? (uint32_t)std::min<uint64_t>(new_capacity, kDefaultMaxProbes)
                              : h->max_probes;
  if (st == DBG_OK) {
    e = cudaMemsetAsync(fail, 0, sizeof(uint32_t), s);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMemsetAsync");
  }
  const int grid = std::max(1, h->sm_count) * 8;
  if (st == DBG_OK) {
    k_rehash<<<grid, 256, 0, s>>>(h->table, h->n_slots, nt, new_capacity, probes, fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "k_rehash");
  }
  if (st == DBG_OK && spilled > 0) {
    k_replay<<<grid, 256, 0, s>>>(h->d_spill, spilled, nt, new_capacity, probes, fail);
    e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(e, "k_replay");
  }
  uint32_t failed = 0;
  if (st == DBG_OK) {
    e = cudaMemcpyAsync(&failed, fail, sizeof(failed), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = cuda_fail(e, "grow");
  }
  if (st != DBG_OK || failed) {
    cudaStreamSynchronize(s);
    cudaFree(nt);
    return st != DBG_OK ? st : DBG_ERR_CAPACITY;
  }
  // the grown table is the handle's own even when the old one was the
  // caller's (whose memory, holding the status block, stays in use)
  if (h->owns_slots) cudaFree(h->table);
  h->owns_slots = true;
  h->table = nt;
  h->n_slots = new_capacity;
  h->max_probes = probes;
  DBG_CK(cudaMemset(h->d_spill_count, 0, sizeof(unsigned long long)));
  return DBG_OK;
}

}  // namespace dbg
