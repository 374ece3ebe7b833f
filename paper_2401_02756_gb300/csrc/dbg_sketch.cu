// K7: HyperLogLog sketch of a read set's vertex keys, the input of the
// capacity predictor (the table must be sized before the build; the number of
// distinct vertices is what sizes it).
//
// For every vertex position (the same positions the insert visits) the key is
// hashed with MurmurHash3's 64-bit finalizer after an XOR with a fixed salt
// (so the sketch hash is unrelated to the table's slot hash); the top 10 bits
// of the hash pick one of 1024 registers and the register keeps the maximum
// of rho = 1 + the number of leading zeros of the remaining 54 bits
// (Flajolet, Fusy, Gandouet, Meunier, "HyperLogLog", AofA 2007).  A maximum
// does not depend on order or repetition, so the registers are a function of
// the set of distinct keys only.
#include <math.h>

#include <algorithm>

#include "dbg_tiles.cuh"

namespace dbg {
namespace {

constexpr unsigned long long kSketchSalt = 0x9E3779B97F4A7C15ull;
constexpr int kSketchRegs = DBG_SKETCH_REGISTERS;
constexpr int kSketchRun = 16;  // positions of one read per thread and round
constexpr int kSketchCtas = 7;  // CTAs of 256 threads per SM (shared memory allows 7)
// read sets per launch: 256 descriptors (26.6 KB) still fit the kernel parameters
constexpr int kSketchItems = 2 * kBatchItems;

// Registers in shared memory (one read set per launch).  A register only
// grows, and after the first few thousand keys almost no key raises it: a key
// whose rho cannot exceed the smallest register (a lower bound the CTA
// refreshes at every tile start) is dropped after one compare, the others
// read their register first and take the atomic only to raise it.  The
// registers are the same as without the bound.
struct SketchVisitor {
  static constexpr bool kUniformRounds = false;
  uint32_t *s_reg;
  volatile uint32_t *s_floor;  // every register is at least this (any value it held stays true)
  // a key whose rest (the hash's 54 low bits, left-aligned) has its high word
  // above lim_hi has rho <= floor: rest >= 2^(64 - floor) for floor <= 32;
  // for a floor above 32, rest >= 2^32 suffices; a floor of 0 drops nothing
  uint32_t lim_hi = ~0u;
  __device__ void tile_begin() {
    const uint32_t f = *s_floor;
    lim_hi = f == 0u ? ~0u : (f <= 32u ? (1u << (32u - f)) - 1u : 0u);
    if (threadIdx.x < 32) {  // the next tile's bound
      uint32_t m = ~0u;
      for (int j = threadIdx.x; j < kSketchRegs; j += 32)
        m = min(m, *reinterpret_cast<volatile uint32_t *>(&s_reg[j]));
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) m = min(m, __shfl_xor_sync(0xffffffffu, m, d));
      if (threadIdx.x == 0) *s_floor = m;
    }
  }
  __device__ bool stop(int) { return false; }
  __device__ void round_end() {}
  __device__ void vertex(bool valid, uint64_t key, bool, uint32_t, int, int, const VertexCtx &) {
    if (!valid) return;
    const uint64_t h = fmix64(key ^ kSketchSalt);
    const uint32_t rest_hi = (uint32_t)(h >> 22);  // bits 53..22 of the hash
    if (rest_hi > lim_hi) return;  // 1 + clz(rest) <= floor: no register can rise
    const uint64_t rest = h << 10;
    const uint32_t idx = (uint32_t)(h >> 54);
    const uint32_t rho = rest ? (uint32_t)__clzll(rest) + 1u : 55u;
    if (rho > *reinterpret_cast<volatile uint32_t *>(&s_reg[idx])) atomicMax(&s_reg[idx], rho);
  }
};

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, kSketchCtas)
    k_sketch(const __grid_constant__ ItemPack<1> pk, int tile_reads, uint32_t *regs) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_reg = reinterpret_cast<uint32_t *>(smem + tile_smem_bytes(tile_reads));
  __shared__ uint32_t s_floor;
  for (int j = threadIdx.x; j < kSketchRegs; j += BLOCK) s_reg[j] = 0u;
  if (threadIdx.x == 0) s_floor = 0u;
  __syncthreads();
  SketchVisitor vis{s_reg, &s_floor};
  for_each_vertex<BLOCK, 1, kSketchRun>(pk, tile_reads, smem, vis, blockIdx.x, pk.total_tiles,
                                        gridDim.x);
  __syncthreads();
  for (int j = threadIdx.x; j < kSketchRegs; j += BLOCK)
    if (s_reg[j]) atomicMax(&regs[j], s_reg[j]);
}

// Many read sets per launch.  Each CTA takes a contiguous range of tiles, so
// it meets few item boundaries; it keeps shared-memory registers for the
// item at hand and merges them into that item's global registers (carried in
// the descriptor's table pointer) when its tiles of the item end.
template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, kSketchCtas)
    k_sketch_batch(const __grid_constant__ ItemPack<kSketchItems> pk, int tile_reads,
                   uint64_t chunk) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint32_t *s_reg = reinterpret_cast<uint32_t *>(smem + tile_smem_bytes(tile_reads));
  __shared__ uint32_t s_floor;
  for (int j = threadIdx.x; j < kSketchRegs; j += BLOCK) s_reg[j] = 0u;
  if (threadIdx.x == 0) s_floor = 0u;
  __syncthreads();
  SketchVisitor vis{s_reg, &s_floor};
  const uint64_t t1 = min(pk.total_tiles, (blockIdx.x + 1) * chunk);
  for (uint64_t t = blockIdx.x * chunk; t < t1;) {
    const int it = find_item(pk, t);
    const uint64_t end = it + 1 < pk.n_items ? pk.d[it + 1].tile_begin : pk.total_tiles;
    const uint64_t tb = min(t1, end);
    for_each_vertex<BLOCK, kSketchItems, kSketchRun>(pk, tile_reads, smem, vis, t, tb, 1);
    __syncthreads();
    uint32_t *g = reinterpret_cast<uint32_t *>(pk.d[it].table);
    for (int j = threadIdx.x; j < kSketchRegs; j += BLOCK)
      if (s_reg[j]) {
        atomicMax(&g[j], s_reg[j]);
        s_reg[j] = 0u;
      }
    if (threadIdx.x == 0) s_floor = 0u;  // the next item starts from empty registers
    __syncthreads();
    t = tb;
  }
}

// Every item's registers and status word := 0.
__global__ void k_zero_registers(const __grid_constant__ ItemPack<kSketchItems> pk) {
  const int i = blockIdx.x;
  uint32_t *r = reinterpret_cast<uint32_t *>(pk.d[i].table);
  for (int j = threadIdx.x; j <= kSketchRegs; j += blockDim.x) r[j] = 0u;
}

}  // namespace
}  // namespace dbg

extern "C" int dbg_sketch_reads(int k, const uint8_t *packed, const uint64_t *offsets,
                                uint64_t n_reads, uint32_t *registers, void *stream) {
  using namespace dbg;
  if (k < 2 || k > 32 || !registers || (n_reads > 0 && (!packed || !offsets)))
    return DBG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DBG_CK(cudaMemsetAsync(registers, 0, (kSketchRegs + 1) * sizeof(uint32_t), s));
  if (n_reads == 0) return DBG_OK;
  constexpr int B = 256;
  const int tile_reads = B;
  ItemPack<1> pk{};
  pk.n_items = 1;
  pk.total_tiles = (n_reads + tile_reads - 1) / tile_reads;
  ItemDesc &it = pk.d[0];
  it.packed = packed;
  it.offsets = offsets;
  it.n_reads = n_reads;
  it.origin = 0;
  it.table = nullptr;
  it.n_slots = 1;
  it.status = registers + kSketchRegs;  // bad offsets are reported here
  it.max_probes = 0;
  it.k = k;
  it.vec_ok = ((uintptr_t)packed & 15u) == 0 ? 1 : 0;
  const size_t smem = tile_smem_bytes(tile_reads) + kSketchRegs * sizeof(uint32_t);
  int dev = 0, sms = 0, per_sm = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sketch<B>, B, smem));
  const int grid = (int)std::min<uint64_t>(pk.total_tiles, (uint64_t)std::max(1, per_sm) * sms);
  k_sketch<B><<<grid, B, smem, s>>>(pk, tile_reads, registers);
  DBG_CK(cudaGetLastError());
  return DBG_OK;
}

extern "C" int dbg_sketch_batch(const dbg_sketch_item *items, int n_items, void *stream) {
  using namespace dbg;
  if (n_items < 0 || (n_items > 0 && !items)) return DBG_ERR_INVALID_ARG;
  for (int i = 0; i < n_items; ++i)
    if (items[i].k < 2 || items[i].k > 32 || !items[i].registers ||
        (items[i].n_reads > 0 && (!items[i].packed || !items[i].offsets)))
      return DBG_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr int B = 256;
  const int tile_reads = B;
  const size_t smem = tile_smem_bytes(tile_reads) + kSketchRegs * sizeof(uint32_t);
  int dev = 0, sms = 0, per_sm = 0;
  DBG_CK(cudaGetDevice(&dev));
  DBG_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (smem > 48 * 1024)
    DBG_CK(cudaFuncSetAttribute(k_sketch_batch<B>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  DBG_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sketch_batch<B>, B, smem));
  for (int first = 0; first < n_items; first += kSketchItems) {
    const int cnt = std::min(kSketchItems, n_items - first);
    ItemPack<kSketchItems> pk{};
    pk.n_items = cnt;
    uint64_t tiles = 0;
    for (int i = 0; i < cnt; ++i) {
      const dbg_sketch_item &src = items[first + i];
      ItemDesc &it = pk.d[i];
      it.packed = src.packed;
      it.offsets = src.offsets;
      it.n_reads = src.n_reads;
      it.origin = 0;
      it.table = reinterpret_cast<Slot *>(src.registers);  // the item's registers
      it.n_slots = 1;
      it.status = src.registers + kSketchRegs;  // bad offsets are reported here
      it.max_probes = 0;
      it.k = src.k;
      it.tile_begin = tiles;
      it.vec_ok = ((uintptr_t)src.packed & 15u) == 0 ? 1 : 0;
      tiles += (src.n_reads + tile_reads - 1) / tile_reads;
    }
    pk.total_tiles = tiles;
    k_zero_registers<<<cnt, 256, 0, s>>>(pk);
    DBG_CK(cudaGetLastError());
    if (tiles == 0) continue;
    const uint64_t slots = (uint64_t)std::max(1, per_sm) * sms;
    const uint64_t chunk = (tiles + slots - 1) / slots;
    const int grid = (int)((tiles + chunk - 1) / chunk);
    k_sketch_batch<B><<<grid, B, smem, s>>>(pk, tile_reads, chunk);
    DBG_CK(cudaGetLastError());
  }
  return DBG_OK;
}

extern "C" double dbg_sketch_estimate(const uint32_t *registers) {
  if (!registers) return -1.0;
  const double m = dbg::kSketchRegs;
  const double alpha = 0.7213 / (1.0 + 1.079 / m);
  double sum = 0.0;
  int zeros = 0;
  for (int j = 0; j < dbg::kSketchRegs; ++j) {
    sum += ldexp(1.0, -(int)registers[j]);
    zeros += registers[j] == 0u;
  }
  const double raw = alpha * m * m / sum;
  if (raw <= 2.5 * m && zeros > 0) return m * log(m / zeros);  // small-range correction
  return raw;
}
