/*
 * dbg.h -- C ABI of the GB300 A-Bruijn graph builder (libdbg.so, sm_103a).
 *
 * The operation is the graph build of "Lock-free de Bruijn graph"
 * (Gorniak & Nowak, arXiv 2401.02756): every length-k substring
 * s_0..s_{k-1} of every read is an edge from the vertex s_0..s_{k-2} to the
 * vertex s_1..s_{k-1} (Section "Background"); both vertices are put in one
 * shared hash table and the source vertex's counter for the label s_{k-1}
 * is incremented (Alg. 2 "makeGraph", Alg. 3 "addLeftVertex"; the target is
 * only made to exist, per the addRightVertex prose after Alg. 3).
 *
 * Conventions for every entry point:
 *   - Return value: a dbg_status code (DBG_OK = 0).  Argument errors are
 *     returned synchronously and nothing is launched.  Errors found by the
 *     GPU while a launch runs (table full, bad offsets) are STICKY: they are
 *     recorded in the handle's device status word and returned by the next
 *     dbg_get_status, dbg_stats or dbg_export_sorted.
 *   - Streams: `stream` is a cudaStream_t passed as void* (NULL = the legacy
 *     default stream).  Launching calls are asynchronous and stream-ordered;
 *     the caller keeps every input alive until the stream has passed the call.
 *   - Device pointers may come from any allocator (cudaMalloc, a PyTorch
 *     tensor's data_ptr(), a memory pool).
 *   - Packed reads: base i of the stream sits in bits [2*(i%4), 2*(i%4)+1] of
 *     byte i/4, codes A=0, C=1, G=2, T=3.  `offsets` holds n_reads+1
 *     non-decreasing base positions; read r is [offsets[r], offsets[r+1]).
 *     offsets[0] may be non-zero.  The packed buffer must be readable for
 *     ceil(offsets[n_reads] / 4) bytes.  A read shorter than k holds no k-mer
 *     and adds nothing.
 *   - Vertex keys: the (k-1) bases of a vertex, 2 bits each, first base in
 *     the most significant position (so key order is lexicographic order
 *     with A < C < G < T).  2 <= k <= 64.  For k <= 32 a key is one 64-bit
 *     word (at most 62 bits); for k > 32 (the paper's default is k = 51,
 *     Section "Code organization") it is a 128-bit integer of at most 126
 *     bits, exported as two words per vertex, high word first.  Graphs with
 *     k > 32 support create, insert (direct path), batch, stats, export and
 *     normalize; spill, grow, the no-alloc export and contigs take k <= 32.
 *   - Counters: 32-bit unsigned, one per label in the order A, C, G, T,
 *     wrapping modulo 2^32 (the paper's are 8-bit, Section "Graph data
 *     structure"; the wider width keeps high-coverage repeats exact).
 */
#ifndef DBG_H
#define DBG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum dbg_status {
  DBG_OK = 0,
  DBG_ERR_INVALID_ARG = 1,      /* bad argument; nothing was launched */
  DBG_ERR_OOM = 2,              /* a device or host allocation failed */
  DBG_ERR_CAPACITY = 3,         /* sticky: a vertex found no free slot within max_probes */
  DBG_ERR_CUDA = 4,             /* a CUDA runtime call failed (see dbg_last_cuda_error) */
  DBG_ERR_BUFFER_TOO_SMALL = 5, /* export: max_n < number of vertices (n_out tells how many) */
  DBG_ERR_BAD_OFFSETS = 6,      /* sticky: the GPU saw offsets[r+1] < offsets[r] */
  DBG_ERR_NOALLOC_LIMIT = 7,    /* dbg_export_sorted_noalloc: graph larger than its fixed scratch */
  DBG_ERR_NEEDS_GROW = 8,       /* vertices were spilled (see dbg_set_spill): call dbg_grow */
  DBG_ERR_TIMEOUT = 9           /* a kernel gave up a bounded wait on a copy (sticky) */
} dbg_status;

typedef struct dbg_graph *dbg_handle;

/* Launch shape of the insert kernel.  Every field may be 0 for "automatic".
 * The built graph does not depend on these values: only the speed does. */
typedef struct dbg_tuning {
  int block_threads;  /* threads per CTA, a multiple of 32 in [64, 1024] (default 256) */
  int tile_reads;     /* reads staged per tile, in [1, block_threads] (default block_threads) */
  int grid_ctas;      /* CTAs in the persistent grid (default: SMs x resident CTAs per SM) */
  int warp_aggregate; /* direct insert: 1 merges a warp's equal keys with __match_any_sync,
                         0 does not, -1: default (1) */
  int insert_path;    /* 0: automatic; 1: direct; 2: binned (k <= 31; see dbg_insert_reads) */
  int apply_unroll;   /* binned apply: probe slots per thread, 2, 4 or 8 (0: default 4) */
  int apply_chunk;    /* binned apply: events per thread per work chunk, 4, 8 or 16 (0: 8) */
  int apply_ctas;     /* binned apply: CTAs per SM (0: as many as fit) */
  int apply_counters; /* binned apply: work counters the warps draw chunks from, 1..64 (0: 16) */
  int region_log2;    /* binned: table region of 2^region_log2 slots, 16..26 (0: automatic) */
  int apply_group;    /* binned apply (streaming): regions per launch (0: all in one launch) */
  int apply_mode;     /* binned apply: 0 automatic (tiled), 1 streaming, 2 tiled */
  int scatter_reads;  /* binned scatter (tiled apply): reads per read tile, 32..512 (0: 416) */
  int split_threads;  /* binned split: threads per CTA, 256, 512 or 1024, at least a quarter
                         of the tiles per region (0: automatic) */
} dbg_tuning;

typedef struct dbg_info {
  int k;
  uint64_t n_slots;     /* table slots (32 bytes each) */
  uint64_t table_bytes; /* device bytes held by the table */
  uint32_t max_probes;  /* slots probed per vertex before DBG_ERR_CAPACITY */
  int device;           /* CUDA device the table lives on */
  uint64_t event_capacity; /* binned-insert event buffer, in events (0: not allocated) */
  uint64_t spill_capacity; /* spill records (0: no spill buffer) */
} dbg_info;

/* Create an empty graph for k-mers of length k (2..64) with room for
 * `capacity` vertices (>= 1).  The table is an open-addressing array of
 * `capacity` 32-byte slots (replacing the paper's array of N list heads,
 * Section "Graph data structure", Fig. 2), allocated on the current CUDA
 * device and emptied before return (synchronously).  *out receives the
 * handle, which owns the table until dbg_destroy.
 * Errors: INVALID_ARG (k or capacity out of range, out == NULL), OOM, CUDA. */
int dbg_create(int k, uint64_t capacity, dbg_handle *out);

/* As dbg_create, with the probe bound: a vertex that finds no matching or
 * free slot within `max_probes` consecutive slots sets DBG_ERR_CAPACITY
 * (0 = default: min(n_slots, 8192)). */
int dbg_create_ex(int k, uint64_t capacity, uint32_t max_probes, dbg_handle *out);

/* Device bytes dbg_create_on needs for `capacity` slots: the slots (32 bytes
 * each) followed by a 256-byte status block.  0 when capacity is 0 or too large. */
uint64_t dbg_table_bytes(uint64_t capacity);

/* As dbg_create_ex, but on caller-owned device memory `mem` (256-byte
 * aligned, at least dbg_table_bytes(capacity) bytes) and without any
 * allocation or synchronization: the table is initialized asynchronously on
 * `stream`, so later work on other streams must be ordered after it.  This
 * is how a request loop sizes and starts one table per request from its own
 * memory pool without stalling the device.  The caller keeps `mem` alive
 * until every stream that used the handle has passed its last call on it.
 * No counterpart in the paper (whose table is one fixed allocation).
 * Errors: INVALID_ARG (k, capacity, alignment, mem_bytes), OOM (host), CUDA. */
int dbg_create_on(int k, uint64_t capacity, uint32_t max_probes, void *mem, uint64_t mem_bytes,
                  void *stream, dbg_handle *out);

/* Release the table and every buffer the handle owns.  Synchronizes the
 * device first when the handle owns device memory (always for dbg_create;
 * for dbg_create_on only after a spill buffer, host staging, binned scratch
 * or a grow allocated some); otherwise frees host state only and does not
 * wait.  NULL is ignored. */
void dbg_destroy(dbg_handle h);

/* Empty the graph (every slot EMPTY, every counter 0) and clear the sticky
 * status, stream-ordered.  Errors: INVALID_ARG, CUDA. */
int dbg_reset(dbg_handle h, void *stream);

/* Set the insert kernel's launch shape (NULL restores the defaults).
 * Errors: INVALID_ARG for out-of-range fields. */
int dbg_set_tuning(dbg_handle h, const dbg_tuning *t);

/* Size the binned insert's event buffers for `events` vertex positions per
 * call, plus a margin for the per-region buckets (events / 16 + 589,824;
 * 0 = the default of 4.25 per table slot).  The handle's first buffer (8
 * bytes per event) is allocated by its next single-read-set binned insert,
 * the second (1.125 times as large plus 2^20 events: room for the per-tile
 * buckets) with it; a batched insert instead counts this size towards the
 * library's own buffers.  Read sets with more positions per slot than the
 * buffer allows (high coverage into a tight table) should reserve their
 * position count, sum over reads of max(0, length - k + 2); otherwise those
 * calls take the direct insert.  Synchronizes the device when it drops a
 * buffer of another size.  Errors: INVALID_ARG, CUDA. */
int dbg_reserve_events(dbg_handle h, uint64_t events);

/* Measurement aid: record CUDA events around every kernel of the next insert
 * calls on this handle (dbg_insert_reads / dbg_insert_reads_host), keeping
 * the last `calls` calls (0 turns it off).  Synchronizes the device. */
int dbg_enable_kernel_timing(dbg_handle h, int calls);

/* Kernel durations of the kept calls, oldest first: out_ms[8*c + j] for
 * kernel j = 0 direct insert, 1 bin count (with the tiled apply: the bucket
 * sizing that replaces the count), 2 bin scan, 3 bin scatter, 4 bin
 * split (the tiled apply's second partition pass, all its kernels), 5 bin
 * apply, 6 bin deferred (the tiled apply's events that left their tile), 7
 * direct insert run as the binned fall-back (it returns at once when the
 * binned kernels did the work);
 * -1 for a kernel the call did not launch.  Waits for the recorded events.
 * *n_calls receives the number of calls written (at most max_calls). */
int dbg_kernel_times(dbg_handle h, float *out_ms, int max_calls, int *n_calls);

/* Diagnostics of the last binned insert call on this handle (synchronizes
 * the device first): out[0] = 1 if the binned kernels did the call's work, 0
 * if the direct insert did it (the events did not fit the buffers, or none
 * has run); out[1] = events whose probe sequence left their 2048-slot tile;
 * out[2] = events that did not fit their tile's bucket.  Both kinds are
 * applied by a global pass after the tiles; both are 0 for the streaming
 * apply.  `out` is a HOST array of 3.  Errors: INVALID_ARG, CUDA. */
int dbg_binned_counters(dbg_handle h, uint64_t *out);

/* Fill *out with the handle's parameters. */
int dbg_get_info(dbg_handle h, dbg_info *out);

/* Insert every k-mer of n_reads reads (Alg. 2 "makeGraph" with Alg. 3 and
 * the addRightVertex prose): for each length-k substring, find or claim the
 * prefix vertex and count the label s_{k-1}, and find or claim the suffix
 * vertex.  `packed` and `offsets` are DEVICE pointers (see the conventions
 * above); the work is launched on `stream`.  Calls on one handle may be
 * issued from several streams at once: counts add, so the graph does not
 * depend on the order (one handle is not safe to use from several host
 * threads at once).  n_reads == 0 launches nothing.
 *
 * Two paths give the same graph.  The direct path is one kernel that updates
 * the table as it walks the reads.  The binned path (k <= 31) first writes
 * one 8-byte event per vertex position grouped by table region, then groups
 * each region's events by 2048-slot tile and applies every tile in shared
 * memory (one CTA per tile, the tile moved by bulk copies), so the table
 * crosses DRAM once in whole lines; events whose probe leaves their tile are
 * applied afterwards from their home slots.  It is chosen automatically for
 * tables of 256 MiB or more and needs event buffers owned by the handle
 * (default 4.25 events per slot, 17 bytes per event across its two buffers,
 * allocated by the first call that needs them, or sized with
 * dbg_reserve_events).  A call with more vertex positions than the buffer
 * holds runs the direct kernel instead (decided on the device).  Binned calls
 * on one handle run one after another.
 * Errors: INVALID_ARG (NULL handle, NULL pointer with n_reads > 0), OOM (event
 * buffer), CUDA; sticky CAPACITY / BAD_OFFSETS. */
int dbg_insert_reads(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                     uint64_t n_reads, void *stream);

/* As dbg_insert_reads, with `packed` and `offsets` in HOST memory (pinned
 * memory gives asynchronous copies; pageable memory works but copies are
 * staged by the driver).  The reads are copied to device staging buffers
 * owned by the handle: whole, when packed bytes plus offsets take at most
 * 4 GiB, and inserted with one call -- the offsets first, then the bases in
 * up to 8 parts of at least 128 MiB, the binned insert's scatter starting on
 * each part as it arrives; otherwise in chunks of at most 2^22 reads /
 * 256 MiB, each chunk's copy overlapping the previous chunk's insert.  The
 * offsets are validated on the host, while the whole input's copies run or
 * before the first chunk's; no kernel is launched when one decreases
 * (INVALID_ARG, after the call's copies have finished).  Returns after the
 * last insert has been launched; the host buffers may be reused once
 * `stream` has passed the call.
 * Errors: as dbg_insert_reads, plus OOM for the staging buffers. */
int dbg_insert_reads_host(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                          uint64_t n_reads, void *stream);

/* Build the graph of n_reads reads from scratch: the table's previous
 * contents are discarded (as dbg_reset) and every k-mer is inserted (as
 * dbg_insert_reads), in one stream-ordered call on `stream`.  The result is
 * the graph dbg_reset followed by dbg_insert_reads gives.  On the binned path
 * (see dbg_insert_reads) the emptying costs no pass of its own: the tiled
 * apply starts every table tile as EMPTY slots in shared memory instead of
 * reading it, and writes every tile -- with events or without -- exactly
 * once.  So the table is not valid until the stream has passed the call:
 * no other call may use the handle from another stream meanwhile.  The
 * sticky status and pending spill records are cleared first.  n_reads == 0
 * only empties the table.  Errors: as dbg_insert_reads. */
int dbg_build_reads(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                    uint64_t n_reads, void *stream);

/* dbg_build_reads with `packed` and `offsets` in HOST memory, staged as
 * dbg_insert_reads_host stages them (the first chunk's insert does the
 * emptying, later chunks add to it).  Errors: as dbg_insert_reads_host. */
int dbg_build_reads_host(dbg_handle h, const uint8_t *packed, const uint64_t *offsets,
                         uint64_t n_reads, void *stream);

/* One item of a batched insert: a target graph and its reads (device
 * pointers, same conventions as dbg_insert_reads). */
typedef struct dbg_batch_item {
  dbg_handle graph;
  const uint8_t *packed;
  const uint64_t *offsets;
  uint64_t n_reads;
} dbg_batch_item;

/* Insert many independent read sets, each into its own graph (graphs may
 * differ in k and size), as one dbg_insert_reads per item would (Alg. 2 per
 * read set).  Graphs with k <= 31 are inserted together in binned chains
 * (see dbg_insert_reads for the binned path), whatever their size, unless
 * their tuning asks for the direct path (insert_path = 1): every binned
 * kernel is launched once per chain and covers all of the chain's tables --
 * the scatter takes (item, read tile) work units of every read set, the
 * regions of all tables share one event buffer, the split and the tiled
 * apply take every table's regions and tiles.  A chain holds up to 128
 * graphs, 2048 table regions (2^21 slots each, by default) and 3.8e9 events;
 * its event buffer holds the sum of its graphs' dbg_reserve_events sizes (or
 * defaults), and if the events do not fit it, the direct insert does that
 * chain's work (decided on the device).  The chains' buffers belong to the
 * library, one set per device, grown as needed and kept until
 * dbg_release_scratch; batched calls on one device run one after another on
 * the GPU.  Graphs on the direct path (and k = 32) share launches: one
 * kernel for up to 128 of them, its CTAs taking (item, read tile) work units
 * from one index space.  Graphs with k > 32 take their own kernel one by
 * one.  Every graph
 * must live on the current device; all work is on `stream`.  The call may be
 * captured into a CUDA graph (cudaStreamBeginCapture on `stream`) after one
 * uncaptured call with graphs of the same sizes (which grows the buffers; a
 * captured call finding them too small gives its chains to the direct
 * insert); replays must not overlap other batched calls on the device.
 * Errors: INVALID_ARG, OOM, CUDA; sticky errors are recorded in each item's
 * own graph. */
int dbg_insert_batch(const dbg_batch_item *items, int n_items, void *stream);

/* dbg_build_reads for many read sets: every item's graph is emptied (table,
 * sticky status, spill records) and built from its reads, with the batching
 * of dbg_insert_batch.  In the binned chains the emptying is folded into the
 * tiled apply (no pass of its own); direct-path graphs are emptied by one
 * launch per group of 128.  Errors: as dbg_insert_batch. */
int dbg_build_batch(const dbg_batch_item *items, int n_items, void *stream);

/* Give back the device memory the library keeps between calls: the batched
 * inserts' buffers and the export's cached temporary memory, on every device
 * (each is synchronised first).  Later calls allocate again as needed.
 * Errors: CUDA. */
int dbg_release_scratch(void);

/* Device bytes the library holds between calls on the current device: the
 * batched inserts' buffers and the export's cached temporary memory (what
 * dbg_release_scratch gives back).  A caller that keeps a device-memory
 * budget counts them; 0 when there is no device. */
uint64_t dbg_scratch_bytes(void);

/* Grow-and-rebuild.  dbg_set_spill gives the graph a buffer of `records`
 * 16-byte spill records (0 removes it): a vertex position that finds no
 * matching or empty slot within max_probes is then kept there, with its
 * label, instead of failing with DBG_ERR_CAPACITY (which remains the outcome
 * when the buffer is full).  While records are pending the graph is
 * incomplete: dbg_get_status, dbg_stats and dbg_export_sorted return
 * DBG_ERR_NEEDS_GROW.  Synchronizes the device.  Errors: INVALID_ARG, OOM. */
int dbg_set_spill(dbg_handle h, uint64_t records);

/* Rebuild the graph in a new table of `new_capacity` slots (0: twice the
 * current size): every vertex and its counters is re-inserted, then every
 * pending spill record is replayed, so the graph is exactly the one a large
 * enough table would have built.  Waits for `stream` and runs on it; the old
 * table is released on success.  If the new table is itself too small,
 * DBG_ERR_CAPACITY is returned and the graph is left as it was (old table and
 * spill intact).  Errors: INVALID_ARG, OOM, CUDA, CAPACITY, and a sticky
 * status other than DBG_OK (a graph that already lost events is not grown). */
int dbg_grow(dbg_handle h, uint64_t new_capacity, void *stream);

/* Wait for `stream`, then return the sticky status (DBG_OK, CAPACITY or
 * BAD_OFFSETS), DBG_ERR_NEEDS_GROW when spilled vertices are pending, or CUDA
 * if a launch failed. */
int dbg_get_status(dbg_handle h, void *stream);

/* Wait for `stream`, then count the vertices and the edges (the sum of all
 * counters) of the graph.  Either output pointer may be NULL.  When the last
 * call that changed the graph was a dbg_build_reads(_host) on the tiled
 * binned path, the build counted its new vertices and its k-mers as it went
 * and those counts are returned, without a pass over the table (unless the
 * build gave its work to the direct insert).
 * Returns the sticky status when it is not DBG_OK (outputs still written). */
int dbg_stats(dbg_handle h, uint64_t *n_vertices, uint64_t *n_edges, void *stream);

/* Export the graph sorted by key (ascending, i.e. lexicographic with
 * A<C<G<T): keys_out[i] (for k > 32: keys_out[2*i] high word, keys_out[2*i+1]
 * low word) and counts_out[4*i .. 4*i+3] (labels A, C, G, T).
 * Output pointers may be host or device memory (copied with
 * cudaMemcpyDefault); either may be NULL to skip it.  Waits for `stream`.
 * *n_out receives the number of vertices D.  If D > max_n,
 * DBG_ERR_BUFFER_TOO_SMALL is returned and nothing is exported (a call with
 * max_n = 0 is therefore a size query); host outputs are then untouched, but
 * in-place device outputs (below) may have served as scratch.  Temporary
 * device memory comes from a stream-ordered pool the library keeps per
 * device (up to 4 GiB of it stays cached between calls) and is released to
 * it before return: about 6 bytes per vertex (the sorted slot indices and the
 * lists of runs of keys that share their first 16 bases) when both outputs
 * are 16-byte aligned device buffers and k <= 32 -- the sort then runs
 * inside keys_out and counts_out, whose max_n rows it uses, and the
 * compaction that fills them counts the vertices, so no separate counting
 * pass over the table is made -- otherwise about 40 bytes per vertex (80 for
 * k > 32).  Errors: INVALID_ARG, OOM, CUDA, BUFFER_TOO_SMALL, and the sticky
 * status (nothing exported when it is set). */
int dbg_export_sorted(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out, uint64_t max_n,
                      uint64_t *n_out, void *stream);

/* Device bytes of scratch dbg_export_sorted_with needs for a graph of
 * n_vertices vertices (k <= 32, a table of at most 2^32 slots): the sort's
 * histograms, one slot index per vertex and the lists of runs of keys that
 * share a prefix.  0 for arguments it does not take.  Needs a device (the
 * sort sizes its work for it). */
uint64_t dbg_export_scratch_bytes(int k, uint64_t n_vertices, uint64_t n_slots);

/* dbg_export_sorted with every byte of device memory from the caller: for a
 * caller that keeps its own budget of device memory (a request loop that
 * accounts for each request's footprint) and wants none taken from the
 * library's pool.  keys_out (uint64 [n]) and counts_out (uint32 [n][4]) are
 * 16-byte aligned DEVICE buffers -- the sort runs inside them -- and
 * `scratch` is a 256-byte aligned device buffer of at least
 * dbg_export_scratch_bytes(k, n, n_slots) bytes, all owned by the caller.
 * k <= 32 and a table of at most 2^32 slots.  Same result and ordering as
 * dbg_export_sorted (the vertices are counted by the compaction into the
 * outputs); waits for `stream`.  Errors: INVALID_ARG (including too small or
 * misaligned scratch and host outputs), CUDA, BUFFER_TOO_SMALL (a size query
 * with max_n = 0), and the sticky status.  After an error the outputs'
 * contents are unspecified. */
int dbg_export_sorted_with(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                           uint64_t max_n, uint64_t *n_out, void *scratch,
                           uint64_t scratch_bytes, void *stream);

/* Normalization (Section "Normalization of graph"): every counter c of the
 * graph becomes floor(c / divisor + 0.5), computed in IEEE double and capped
 * at 2^32 - 1.  The paper's divisor is the number of k-mer duplicates,
 * reads * (read length - k + 1) / genome size (for reads of uneven length:
 * the number of edges / genome size).  Rounding to the nearest integer is a
 * reading: the paper's counters are integers, and the rounding lets an error
 * k-mer seen once fall to 0.  In place, stream-ordered; waits for `stream`
 * first to check the sticky status.  Errors: INVALID_ARG (divisor not
 * positive and finite), the sticky status, CUDA. */
int dbg_normalize(dbg_handle h, double divisor, void *stream);

/* Contigs (Section "Finding contigs", Alg. 5 findContigs and makePath).  An
 * outgoing edge is a label with a nonzero counter; the first flag (no edge
 * points to the vertex) is taken from the counters as they are now.  Every
 * vertex that is first or has not exactly one outgoing edge starts one
 * contig per outgoing edge; a contig follows edges while the vertex it
 * reaches has exactly one outgoing edge, and stops on reaching a vertex it
 * has already visited, keeping the edge into it.  Contigs are ordered by
 * (start vertex key, first label).
 * Output: bases_out gets every contig's bases as ASCII A/C/G/T, back to
 * back; offsets_out[i] .. offsets_out[i+1] delimits contig i (n + 1 entries,
 * offsets_out[0] = 0).  Both may be host or device memory; *n_contigs and
 * *n_bases always receive the sizes, and with too small or NULL buffers
 * (max_contigs < n or max_bases < total) nothing else is written and
 * DBG_ERR_BUFFER_TOO_SMALL is returned: a two-call size query.  Uses the
 * slots' padding word as scratch and temporary device memory (freed before
 * returning); synchronizes `stream`.  Errors: INVALID_ARG, the sticky status,
 * BUFFER_TOO_SMALL, CAPACITY (a target vertex missing: an incomplete graph),
 * CUDA. */
int dbg_find_contigs(dbg_handle h, char *bases_out, uint64_t max_bases, uint64_t *offsets_out,
                     uint64_t max_contigs, uint64_t *n_contigs, uint64_t *n_bases, void *stream);

/* Fixed scratch of dbg_export_sorted_noalloc, and the largest graph it exports. */
#define DBG_NOALLOC_SCRATCH_BYTES (16u << 20)
#define DBG_NOALLOC_EXPORT_MAX_VERTICES (1u << 19)

/* dbg_export_sorted without any device allocation.  The paper has no
 * counterpart: this exists for callers that must not allocate device memory
 * while they run -- a serving loop held to a memory budget that another
 * component accounts for, a framework that owns every device allocation, or
 * code that cannot accept the device-wide synchronisation cudaMalloc/cudaFree
 * may cause.  Same result and ordering as dbg_export_sorted, but:
 *   - keys_out (uint64 [n]) and counts_out (uint32 [n][4]) are DEVICE
 *     pointers owned by the caller, both required;
 *   - its temporary memory is a fixed DBG_NOALLOC_SCRATCH_BYTES device array
 *     inside libdbg.so, held by every GPU that loads the library until the
 *     process exits, so a graph of more than DBG_NOALLOC_EXPORT_MAX_VERTICES
 *     vertices is refused with DBG_ERR_NOALLOC_LIMIT (*n_out still receives
 *     the vertex count);
 *   - the first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress with that device current); make that first call
 *     before any stream capture;
 *   - every call on a device shares the one array: calls whose GPU work
 *     overlaps (different streams, or host threads) race and must be
 *     serialised by the caller.
 *   - keys of one word only: a graph with k > 32 is refused with
 *     DBG_ERR_INVALID_ARG (dbg_export_sorted exports those);
 *   - the looked-up address is kept until the process exits: after a
 *     cudaDeviceReset of that device it is stale, and the entry point must
 *     not be used again in that process.
 * Waits for `stream`.  Errors: INVALID_ARG, CUDA, BUFFER_TOO_SMALL (max_n <
 * vertices), NOALLOC_LIMIT, and the sticky status. */
int dbg_export_sorted_noalloc(dbg_handle h, uint64_t *keys_out, uint32_t *counts_out,
                              uint64_t max_n, uint64_t *n_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Capacity prediction: a HyperLogLog sketch of the vertex keys.             */
/* ------------------------------------------------------------------------ */

#define DBG_SKETCH_REGISTERS 1024

/* Sketch the distinct vertices of a read set (device buffers, conventions as
 * dbg_insert_reads) so that a table can be sized before it is built (the
 * paper sizes its table from the genome size, Section "Code organization").
 * Every vertex position's key is hashed (MurmurHash3's finalizer after a fixed
 * salt); the top 10 bits select one of DBG_SKETCH_REGISTERS registers, which
 * keep the maximum of 1 + the leading zeros of the other 54 bits (HyperLogLog,
 * Flajolet et al. 2007).  `registers` is a device array of
 * DBG_SKETCH_REGISTERS + 1 uint32: it is zeroed, then filled; the last word
 * receives DBG_ERR_BAD_OFFSETS if an offset decreases.  Asynchronous on
 * `stream`.  The registers depend only on the set of distinct keys.
 * Errors: INVALID_ARG, CUDA. */
int dbg_sketch_reads(int k, const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads,
                     uint32_t *registers, void *stream);

/* One read set of a batched sketch: its reads (device, as for
 * dbg_insert_reads) and its DBG_SKETCH_REGISTERS + 1 device words of output
 * (the registers, then a status word). */
typedef struct dbg_sketch_item {
  int k;
  const uint8_t *packed;
  const uint64_t *offsets;
  uint64_t n_reads;
  uint32_t *registers;
} dbg_sketch_item;

/* dbg_sketch_reads for many read sets at once: one launch per up to 256
 * items, whose CTAs take (item, read tile) work units from one index space.
 * Each item's registers equal those dbg_sketch_reads gives it.  Asynchronous
 * on `stream`.  Errors: INVALID_ARG (k, NULL pointers), CUDA. */
int dbg_sketch_batch(const dbg_sketch_item *items, int n_items, void *stream);

/* Host helper: the HyperLogLog estimate of the number of distinct keys from
 * DBG_SKETCH_REGISTERS registers in host memory (raw estimate with the
 * small-range linear-counting correction); -1 for a NULL pointer. */
double dbg_sketch_estimate(const uint32_t *registers);

/* The capacity predictor's network: FP32, DBG_MLP_INPUTS -> DBG_MLP_HIDDEN ->
 * DBG_MLP_HIDDEN -> 1 with ReLU, mapping a sketch's registers (divided by 64)
 * to ln(distinct vertices).  All buffers are device memory owned by the
 * caller; nothing is allocated.  Parameters (DBG_MLP_PARAMS floats):
 * W1[64][1024] | b1[64] | W2[64][64] | b2[64] | w3[64] | b3.  `work` holds
 * dbg_mlp_work_floats(batch) floats.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
#define DBG_MLP_INPUTS 1024
#define DBG_MLP_HIDDEN 64
#define DBG_MLP_PARAMS 69825

uint64_t dbg_mlp_work_floats(int batch);

/* x[b][j] = registers[b * stride + j] / 64 for j < DBG_MLP_INPUTS. */
int dbg_mlp_features(const uint32_t *registers, int64_t stride, int batch, float *x, void *stream);

/* He-uniform weights from a counter-based hash of (seed, index); zero biases. */
int dbg_mlp_init(float *params, uint64_t seed, void *stream);

/* y[b] = network(x[b]) for b < batch (x: batch x DBG_MLP_INPUTS, row-major). */
int dbg_mlp_forward(const float *params, const float *x, int batch, float *y, float *work,
                    void *stream);

/* One Adam step (step >= 1, learning rate lr, betas 0.9 / 0.999, eps 1e-8) on
 * the mean of (y - target)^2 / 2 over the batch.  `grads`, `adam_m`, `adam_v`
 * hold DBG_MLP_PARAMS floats each (the moments start at zero); *loss_out
 * (device or host, may be NULL) receives the loss before the step. */
int dbg_mlp_train_step(float *params, float *grads, float *adam_m, float *adam_v, int step,
                       float lr, const float *x, const float *target, int batch, float *work,
                       float *loss_out, void *stream);

/* Host helper: pack n ASCII bases (A, C, G, T; upper case) into out, which
 * holds ceil(n/4) bytes, starting at base position `phase` (0..3) of out[0]
 * (bits of out[0] below the phase are preserved).  Any other symbol returns
 * INVALID_ARG and *bad_index (if not NULL) receives its position; 2-bit
 * packing cannot represent N. */
int dbg_pack_ascii(const char *ascii, uint64_t n, uint8_t *out, int phase, uint64_t *bad_index);

/* Message for a status code (static storage). */
const char *dbg_strerror(int code);

/* Text of the last CUDA error seen by this library on this thread ("" if none). */
const char *dbg_last_cuda_error(void);

/* The architecture the library's kernels were compiled for, as the CUDA
 * runtime reports it for the current device (cudaFuncGetAttributes'
 * binaryVersion: major * 10 + minor, 103 for sm_103a).  Needs a GPU.
 * Errors: INVALID_ARG (NULL), CUDA (no device, or no kernel image for it). */
int dbg_binary_version(int *out);

/* ------------------------------------------------------------------------ */
/* Measurement kernels: the random-sector ceiling the insert is rated on.   */
/* ------------------------------------------------------------------------ */

/* Random 32-byte-sector traffic over `n_slots` 32-byte slots at `buf`
 * (device, 32-byte aligned): `n_ops` operations at slots drawn by a
 * counter-based hash of (seed, op index).  mode 0: atomicAdd to one 32-bit
 * word of the slot (read-modify-write at L2, no return); mode 1: load the
 * slot's first 8 bytes, then atomicAdd to a word of the same slot (the
 * insert's found-vertex pattern); mode 2: atomicCAS on the first 8 bytes.
 * The buffer's contents change.  Errors: INVALID_ARG, CUDA. */
int dbg_probe_random_sectors(void *buf, uint64_t n_slots, uint64_t n_ops, uint64_t seed, int mode,
                             void *stream);

/* As mode 1 above (load, then atomicAdd on the same slot), on a random slot
 * of a window of `window_slots` slots that slides linearly from the start to
 * the end of the buffer as the operation index grows -- the pattern of a
 * region-ordered stream of table updates.  flags bit 0: give the accesses an
 * L2 evict_last cache policy; bit 1: loads only; bit 2: atomicAdds only.
 * Errors: INVALID_ARG, CUDA. */
int dbg_probe_window(void *buf, uint64_t n_slots, uint64_t n_ops, uint64_t window_slots,
                     uint64_t seed, int flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* DBG_H */
