// Binned insert (see dbg_binned.cu): geometry and the host entries.
#pragma once

#include "dbg_internal.cuh"

namespace dbg {

constexpr int kBinMaxParts = 2048;           // regions of one chain (one or many tables), at most
constexpr uint64_t kBinMinTableBytes = 256ull << 20;  // auto mode: tables at least this big
constexpr uint64_t kBinMinEvents = 16ull << 20;       // smallest event buffer
constexpr uint64_t kBinEventsPerSlot = 4;             // default event buffer: 4.25 events per slot
                                                      // (4 + 1/4, the buckets' margin included)

constexpr uint64_t kBinSlices = 4096;                // count/scatter work units, at most
constexpr int kBinMinShift = 18;                     // automatic: regions of at least 2^18 slots (8 MiB)

constexpr int kBinApplyCounters = 64;                // apply: chunk counters per launch, at most

// meta area: begin[kBinMaxParts + 1] | counts[kBinMaxParts] | cursor[kBinMaxParts] |
// counters[4] (the last holds the flag) | apply counters[kBinMaxParts][kBinApplyCounters] |
// item totals[kBatchItems] | item edges[kBatchItems] | slice histograms
// u32[kBinSlices][kBinMaxParts]
constexpr size_t kBinMetaBytes =
    ((size_t)kBinMaxParts + 1) * 8 + 2 * (size_t)kBinMaxParts * 8 + 4 * 8 +
    (size_t)kBinMaxParts * kBinApplyCounters * 8 + 2 * (size_t)kBatchItems * 8 +
    (size_t)kBinSlices * kBinMaxParts * 4;

struct BinGeometry {
  int shift;  // region = slots [p << shift, (p + 1) << shift)
  int parts;
};

// Regions of 2^region_log2 slots (0: automatic), widened until there are at
// most kBinMaxParts of them.
BinGeometry bin_geometry(uint64_t n_slots, int region_log2);

// The event capacity a handle's binned inserts use: what dbg_reserve_events
// asked for, else the default of 4.25 per table slot.
uint64_t bin_events_wanted(dbg_handle h);

// Make sure the handle holds an event buffer of at least `events` events
// (0: bin_events_wanted) and the meta area.
int ensure_bin_scratch(dbg_handle h, uint64_t events);

// A read set whose packed bases arrive in parts (host input copied part by
// part on another stream): part c holds reads [read_cut[c], read_cut[c + 1])
// and is in device memory once ready[c] has completed.  The offsets of every
// read must be there before the call's first kernel.
struct InputParts {
  int n = 0;
  const uint64_t *read_cut = nullptr;  // n + 1 read indices, from 0 to the read count
  const cudaEvent_t *ready = nullptr;  // n events
};

// Make `s` wait for every part of `input` (when it is not null).
int wait_input(const InputParts *input, cudaStream_t s);

// Insert one read set through count / scan / scatter / apply, falling back to
// the direct kernel on the device when the events do not fit the buffer.
// `call`: the kernel timer's ring slot for this call (-1: not timed).
// `fresh`: the table is rebuilt from empty (its contents are discarded); the
// tiled apply then writes every tile from an EMPTY tile in shared memory
// instead of reading it, which empties the table without a pass of its own.
// `input`: the reads arrive in parts; the tiled chain's scatter takes each
// part as it arrives, every other path waits for all of them first.
int launch_binned(dbg_handle h, const ItemDesc &it, uint64_t tiles, const dbg_tuning &tuning,
                  cudaStream_t s, int call, bool fresh = false,
                  const InputParts *input = nullptr);

// Insert many read sets, each into its own table (k <= 31), through binned
// chains: every chain is one launch of each binned kernel over all of its
// items (up to kBatchItems of them and kBinMaxParts regions).  items[i]
// carries the direct kernel's tile numbering (tile_begin over `tile_reads`
// reads per tile); `want[i]` is the event capacity item i asks for.  The
// scratch is the library's own, per device.  Items of a chain whose events
// do not fit the scratch (a call captured into a CUDA graph before the
// scratch was large enough) take the direct insert instead.
int launch_binned_batch(const ItemDesc *items, const uint64_t *want, int n,
                        const dbg_tuning &tuning, int sm_count, cudaStream_t s, bool fresh);

// Empty the tables of items[0..n) (n <= kBatchItems) with one launch.
int launch_tables_init(const ItemDesc *items, int n, int sm_count, cudaStream_t s);

// Release the library's own binned scratch on every device (synchronising it).
int release_batch_scratch();

// Device bytes of the library's own binned scratch on device `dev`.
uint64_t batch_scratch_bytes(int dev);

// The last binned call's counters (synchronizes the device): out[0] = 1 if
// the binned kernels did its work, out[1] = events whose probe left their
// tile, out[2] = events that overflowed their tile's bucket.
int binned_counters(dbg_handle h, uint64_t *out);

}  // namespace dbg
