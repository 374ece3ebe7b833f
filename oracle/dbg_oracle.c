/*
 * CPU oracle for the A-Bruijn graph build -- TEST INFRASTRUCTURE ONLY.
 *
 * This file is the slow, plain, obviously correct definition that the CUDA
 * library is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library never does, and the two
 * share no code, headers, tables or helpers.
 *
 * What it computes (Section "Background", Alg. 2 "makeGraph", Alg. 3
 * "addLeftVertex", the prose on addRightVertex after Alg. 3):
 *   every length-k substring s_0..s_{k-1} of every read is an edge from the
 *   vertex s_0..s_{k-2} to the vertex s_1..s_{k-1}; the source vertex's
 *   counter for the label s_{k-1} is incremented once per occurrence, and the
 *   target vertex is only made to exist (never incremented).
 *
 * The reads are first unpacked to ASCII and the whole build works on ASCII
 * (k-1)-mer strings, as the paper's Node does (Fig. 2: the node stores the
 * (k-1)-mer string).  Vertices live in a hash table of chained nodes (Fig. 2),
 * hashed with FNV-1a over the string -- deliberately unrelated to the hash
 * the GPU table uses.
 *
 * Readings of the paper taken here:
 *   - counter columns are in the figures' label order A, C, G, T (the paper's
 *     (c>>1)&3 order A, C, T, G is stated not to affect the algorithm);
 *   - counters are 32-bit unsigned and wrap modulo 2^32 (the paper's 8-bit
 *     counters leave overflow unspecified);
 *   - reads shorter than k contribute nothing (they hold no k-mer);
 *   - no canonical / reverse-complement merging, no de-duplication.
 *
 * Output: vertices sorted lexicographically by their string with A<C<G<T
 * (ASCII order), each with its encoded key (A=0, C=1, G=2, T=3, first base in
 * the most significant position) and its four counters.
 *
 * Pins (tests/test_oracle.py): the paper's Fig. 1 example, brute force over
 * every short read, the k=2 closed form (dinucleotide counts), the count-sum
 * and degree-balance invariants, and Eulerian re-spelling of single reads.
 *
 * Sharding: a build may keep only the vertices whose FNV-1a hash satisfies
 * hash % shard_mod == shard_id (exact for those vertices), so that very large
 * read sets can be checked in passes.  Threads split the kept vertices again
 * by (hash / shard_mod) % n_threads; every thread scans every read.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_OK = 0, OR_ERR_ARG = 1, OR_ERR_NOMEM = 2 };

/* ------------------------------------------------------------------------- */
/* strings                                                                    */
/* ------------------------------------------------------------------------- */

static const char LETTER[4] = {'A', 'C', 'G', 'T'};

/* base i of the packed stream: byte i/4, bits 2*(i%4) .. 2*(i%4)+1 */
static void unpack_range(const uint8_t *packed, uint64_t start, uint64_t len, char *out) {
  for (uint64_t i = 0; i < len; ++i) {
    uint64_t p = start + i;
    unsigned code = (packed[p >> 2] >> (2u * (unsigned)(p & 3u))) & 3u;
    out[i] = LETTER[code];
  }
}

/* the counter column of a label: A=0, C=1, G=2, T=3 */
static int label_column(char c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
  }
}

static uint64_t fnv1a(const char *s, int m) {
  uint64_t h = 1469598103934665603ull;
  for (int i = 0; i < m; ++i) {
    h ^= (uint8_t)s[i];
    h *= 1099511628211ull;
  }
  return h;
}

/* encoded key: first base most significant, 2 bits per base */
static uint64_t encode(const char *s, int m) {
  uint64_t key = 0;
  for (int i = 0; i < m; ++i) key = key * 4u + (uint64_t)label_column(s[i]);
  return key;
}

/* ------------------------------------------------------------------------- */
/* vertex map: buckets of chained nodes (Fig. 2)                             */
/* ------------------------------------------------------------------------- */

typedef struct {
  uint64_t next; /* index + 1 of the next node in the chain, 0 = end */
  uint32_t cnt[4];
  uint32_t first; /* Section "Finding contigs": no edge points to this vertex */
} node_t;

typedef struct {
  int m;           /* vertex string length, k - 1 */
  uint64_t nbuckets;
  uint64_t *head;  /* index + 1 of the first node, 0 = empty bucket */
  node_t *nodes;
  char *strs;      /* m chars per node */
  uint64_t n, cap;
} vmap_t;

static int vmap_init(vmap_t *v, int m) {
  memset(v, 0, sizeof(*v));
  v->m = m;
  v->nbuckets = 1024;
  v->head = (uint64_t *)calloc(v->nbuckets, sizeof(uint64_t));
  v->cap = 1024;
  v->nodes = (node_t *)malloc(v->cap * sizeof(node_t));
  v->strs = (char *)malloc(v->cap * (size_t)(m > 0 ? m : 1));
  return (v->head && v->nodes && v->strs) ? OR_OK : OR_ERR_NOMEM;
}

static void vmap_free(vmap_t *v) {
  free(v->head);
  free(v->nodes);
  free(v->strs);
  memset(v, 0, sizeof(*v));
}

static int vmap_rehash(vmap_t *v) {
  uint64_t nb = v->nbuckets * 2;
  uint64_t *h = (uint64_t *)calloc(nb, sizeof(uint64_t));
  if (!h) return OR_ERR_NOMEM;
  for (uint64_t i = 0; i < v->n; ++i) {
    uint64_t b = fnv1a(v->strs + i * (uint64_t)v->m, v->m) % nb;
    v->nodes[i].next = h[b];
    h[b] = i + 1;
  }
  free(v->head);
  v->head = h;
  v->nbuckets = nb;
  return OR_OK;
}

/* Find the vertex with string s, adding it with zero counters if absent
 * (Alg. 4 "findVertex" followed by the insertion of Alg. 3).  *created tells
 * whether it was added.  Returns the node index, or UINT64_MAX when memory
 * runs out. */
static uint64_t vmap_find_or_add(vmap_t *v, const char *s, uint64_t hash, int *created) {
  uint64_t b = hash % v->nbuckets;
  *created = 0;
  for (uint64_t i = v->head[b]; i != 0; i = v->nodes[i - 1].next)
    if (memcmp(v->strs + (i - 1) * (uint64_t)v->m, s, (size_t)v->m) == 0) return i - 1;
  *created = 1;
  if (v->n == v->cap) {
    uint64_t nc = v->cap * 2;
    node_t *nn = (node_t *)realloc(v->nodes, nc * sizeof(node_t));
    if (!nn) return UINT64_MAX;
    v->nodes = nn;
    char *ns = (char *)realloc(v->strs, nc * (size_t)(v->m > 0 ? v->m : 1));
    if (!ns) return UINT64_MAX;
    v->strs = ns;
    v->cap = nc;
  }
  uint64_t idx = v->n++;
  memcpy(v->strs + idx * (uint64_t)v->m, s, (size_t)v->m);
  memset(v->nodes[idx].cnt, 0, sizeof(v->nodes[idx].cnt));
  v->nodes[idx].first = 0;
  v->nodes[idx].next = v->head[b];
  v->head[b] = idx + 1;
  if (v->n > v->nbuckets) {
    if (vmap_rehash(v) != OR_OK) return UINT64_MAX;
  }
  return idx;
}

/* ------------------------------------------------------------------------- */
/* build                                                                      */
/* ------------------------------------------------------------------------- */

typedef struct oracle_graph {
  int k;
  int nparts;
  vmap_t *parts;
} oracle_graph;

typedef struct {
  const uint8_t *packed;
  const uint64_t *offsets;
  uint64_t n_reads;
  int k;
  uint64_t shard_mod, shard_id;
  int n_threads, t;
  vmap_t *map;
  int status;
} job_t;

static int owned(const job_t *J, uint64_t h) {
  if (h % J->shard_mod != J->shard_id) return 0;
  return (int)((h / J->shard_mod) % (uint64_t)J->n_threads) == J->t;
}

/* Alg. 2 over this thread's view of every read. */
static void *build_worker(void *arg) {
  job_t *J = (job_t *)arg;
  const int k = J->k, m = k - 1;
  uint64_t maxlen = 0;
  for (uint64_t r = 0; r < J->n_reads; ++r) {
    uint64_t len = J->offsets[r + 1] - J->offsets[r];
    if (len > maxlen) maxlen = len;
  }
  char *buf = (char *)malloc(maxlen + 1);
  if (!buf) {
    J->status = OR_ERR_NOMEM;
    return NULL;
  }
  for (uint64_t r = 0; r < J->n_reads; ++r) {
    uint64_t start = J->offsets[r], len = J->offsets[r + 1] - J->offsets[r];
    if (len < (uint64_t)k) continue; /* no k-mer in this read */
    unpack_range(J->packed, start, len, buf);
    for (uint64_t j = 0; j + (uint64_t)k <= len; ++j) {
      const char *left = buf + j;      /* s_0 .. s_{k-2} */
      const char *right = buf + j + 1; /* s_1 .. s_{k-1} */
      char label = buf[j + (uint64_t)k - 1];
      uint64_t hl = fnv1a(left, m);
      int created;
      if (owned(J, hl)) { /* addLeftVertex: find-or-add, then count the edge */
        uint64_t v = vmap_find_or_add(J->map, left, hl, &created);
        if (v == UINT64_MAX) { J->status = OR_ERR_NOMEM; free(buf); return NULL; }
        J->map->nodes[v].cnt[label_column(label)] += 1u;
        /* a vertex created as a left vertex has no edge pointing to it yet */
        if (created) J->map->nodes[v].first = 1u;
      }
      uint64_t hr = fnv1a(right, m);
      if (owned(J, hr)) { /* addRightVertex: make sure it exists; an edge now
                             points to it, so its first flag is cleared */
        uint64_t v = vmap_find_or_add(J->map, right, hr, &created);
        if (v == UINT64_MAX) { J->status = OR_ERR_NOMEM; free(buf); return NULL; }
        J->map->nodes[v].first = 0u;
      }
    }
  }
  free(buf);
  return NULL;
}

void oracle_free(oracle_graph *g) {
  if (!g) return;
  for (int i = 0; i < g->nparts; ++i) vmap_free(&g->parts[i]);
  free(g->parts);
  free(g);
}

/* Build the graph of the reads (restricted to one shard of the vertices).
 * packed/offsets: the 2-bit stream and the n_reads+1 read boundaries, in
 * bases.  2 <= k <= 32.  shard_mod >= 1, shard_id < shard_mod, n_threads >= 1. */
int oracle_build(const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads, int k,
                 uint64_t shard_mod, uint64_t shard_id, int n_threads, oracle_graph **out) {
  if (!out || k < 2 || k > 64 || shard_mod < 1 || shard_id >= shard_mod || n_threads < 1)
    return OR_ERR_ARG;
  if (!offsets) return OR_ERR_ARG;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (offsets[r + 1] < offsets[r]) return OR_ERR_ARG;
  if (offsets[n_reads] > offsets[0] && !packed) return OR_ERR_ARG;
  oracle_graph *g = (oracle_graph *)calloc(1, sizeof(oracle_graph));
  if (!g) return OR_ERR_NOMEM;
  g->k = k;
  g->nparts = n_threads;
  g->parts = (vmap_t *)calloc((size_t)n_threads, sizeof(vmap_t));
  job_t *jobs = (job_t *)calloc((size_t)n_threads, sizeof(job_t));
  pthread_t *th = (pthread_t *)calloc((size_t)n_threads, sizeof(pthread_t));
  if (!g->parts || !jobs || !th) {
    free(jobs); free(th); oracle_free(g);
    return OR_ERR_NOMEM;
  }
  int st = OR_OK;
  for (int t = 0; t < n_threads; ++t)
    if (vmap_init(&g->parts[t], k - 1) != OR_OK) st = OR_ERR_NOMEM;
  if (st == OR_OK) {
    for (int t = 0; t < n_threads; ++t) {
      job_t J = {packed, offsets, n_reads, k, shard_mod, shard_id, n_threads, t, &g->parts[t], OR_OK};
      jobs[t] = J;
    }
    if (n_threads == 1) {
      build_worker(&jobs[0]);
    } else {
      for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, build_worker, &jobs[t]);
      for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    }
    for (int t = 0; t < n_threads; ++t)
      if (jobs[t].status != OR_OK) st = jobs[t].status;
  }
  free(jobs);
  free(th);
  if (st != OR_OK) {
    oracle_free(g);
    return st;
  }
  *out = g;
  return OR_OK;
}

uint64_t oracle_num_vertices(const oracle_graph *g) {
  uint64_t n = 0;
  for (int i = 0; i < g->nparts; ++i) n += g->parts[i].n;
  return n;
}

/* ------------------------------------------------------------------------- */
/* sorted export                                                              */
/* ------------------------------------------------------------------------- */

typedef struct {
  const char *s;
  const uint32_t *cnt;
  uint32_t first;
} ref_t;

static int g_sort_m; /* string length for the comparator (export is single-threaded) */

static int cmp_ref(const void *a, const void *b) {
  return memcmp(((const ref_t *)a)->s, ((const ref_t *)b)->s, (size_t)g_sort_m);
}

static int sorted_refs(const oracle_graph *g, ref_t **out, uint64_t *n_out) {
  uint64_t n = oracle_num_vertices(g);
  ref_t *refs = (ref_t *)malloc((n ? n : 1) * sizeof(ref_t));
  if (!refs) return OR_ERR_NOMEM;
  uint64_t j = 0;
  for (int p = 0; p < g->nparts; ++p)
    for (uint64_t i = 0; i < g->parts[p].n; ++i) {
      refs[j].s = g->parts[p].strs + i * (uint64_t)(g->k - 1);
      refs[j].cnt = g->parts[p].nodes[i].cnt;
      refs[j].first = g->parts[p].nodes[i].first;
      ++j;
    }
  g_sort_m = g->k - 1;
  qsort(refs, n, sizeof(ref_t), cmp_ref);
  *out = refs;
  *n_out = n;
  return OR_OK;
}

/* Vertices in lexicographic order (A<C<G<T): encoded keys and counters
 * [n][4] in A, C, G, T order.  Buffers hold at least max_n entries.  Keys
 * of k - 1 <= 32 bases only (oracle_export_sorted_wide takes any k). */
int oracle_export_sorted(const oracle_graph *g, uint64_t *keys, uint32_t *counts, uint64_t max_n) {
  ref_t *refs;
  uint64_t n;
  if (!g || (keys && g->k - 1 > 32)) return OR_ERR_ARG;
  if (oracle_num_vertices(g) > max_n) return OR_ERR_ARG;
  int st = sorted_refs(g, &refs, &n);
  if (st != OR_OK) return st;
  for (uint64_t i = 0; i < n; ++i) {
    if (keys) keys[i] = encode(refs[i].s, g->k - 1);
    if (counts) memcpy(counts + 4 * i, refs[i].cnt, 4 * sizeof(uint32_t));
  }
  free(refs);
  return OR_OK;
}

/* The same order with keys of up to 63 bases as 128-bit integers, the first
 * base most significant: keys[2i] holds bits 64..127, keys[2i+1] bits 0..63. */
int oracle_export_sorted_wide(const oracle_graph *g, uint64_t *keys, uint32_t *counts,
                              uint64_t max_n) {
  ref_t *refs;
  uint64_t n;
  if (!g) return OR_ERR_ARG;
  if (oracle_num_vertices(g) > max_n) return OR_ERR_ARG;
  int st = sorted_refs(g, &refs, &n);
  if (st != OR_OK) return st;
  const int m = g->k - 1;
  for (uint64_t i = 0; i < n; ++i) {
    uint64_t hi = 0, lo = 0;
    for (int j = 0; j < m; ++j) { /* (hi, lo) = (hi, lo) * 4 + code */
      hi = (hi << 2) | (lo >> 62);
      lo = (lo << 2) | (uint64_t)label_column(refs[i].s[j]);
    }
    if (keys) {
      keys[2 * i] = hi;
      keys[2 * i + 1] = lo;
    }
    if (counts) memcpy(counts + 4 * i, refs[i].cnt, 4 * sizeof(uint32_t));
  }
  free(refs);
  return OR_OK;
}

/* The same order: each vertex's first flag (1 = no edge points to it). */
int oracle_export_first(const oracle_graph *g, uint8_t *out, uint64_t max_n) {
  ref_t *refs;
  uint64_t n;
  if (!g || !out) return OR_ERR_ARG;
  if (oracle_num_vertices(g) > max_n) return OR_ERR_ARG;
  int st = sorted_refs(g, &refs, &n);
  if (st != OR_OK) return st;
  for (uint64_t i = 0; i < n; ++i) out[i] = (uint8_t)refs[i].first;
  free(refs);
  return OR_OK;
}

/* The same order, as strings: n * (k-1) characters, no separators. */
int oracle_export_strings(const oracle_graph *g, char *out, uint64_t max_n) {
  ref_t *refs;
  uint64_t n;
  if (!g || !out) return OR_ERR_ARG;
  if (oracle_num_vertices(g) > max_n) return OR_ERR_ARG;
  int st = sorted_refs(g, &refs, &n);
  if (st != OR_OK) return st;
  for (uint64_t i = 0; i < n; ++i) memcpy(out + i * (uint64_t)(g->k - 1), refs[i].s, (size_t)(g->k - 1));
  free(refs);
  return OR_OK;
}

/* Shard of each encoded key under this oracle's sharding (decode to the
 * string, FNV-1a, modulo shard_mod), so that another builder's output can be
 * filtered to the vertices of one oracle shard. */
void oracle_shard_of_keys(const uint64_t *keys, uint64_t n, int k, uint64_t shard_mod, uint64_t *out) {
  int m = k - 1;
  char s[64];
  for (uint64_t i = 0; i < n; ++i) {
    for (int j = 0; j < m; ++j) s[j] = LETTER[(keys[i] >> (2 * (m - 1 - j))) & 3u];
    out[i] = fnv1a(s, m) % shard_mod;
  }
}

/* ------------------------------------------------------------------------- */
/* HyperLogLog registers of the vertex keys (for the sketch kernel's parity)  */
/* ------------------------------------------------------------------------- */

/* MurmurHash3's 64-bit finalizer, from its published definition. */
static uint64_t murmur3_fmix64(uint64_t x) {
  x ^= x >> 33;
  x *= 0xff51afd7ed558ccdULL;
  x ^= x >> 33;
  x *= 0xc4ceb9fe1a85ec53ULL;
  x ^= x >> 33;
  return x;
}

/* Registers (1024) of the HyperLogLog sketch (Flajolet et al. 2007) of the
 * distinct (k-1)-mers that the build would make vertices: for each vertex
 * position of each read of length >= k, hash = fmix64(key XOR salt), register
 * = top 10 bits, value = max(value, 1 + leading zeros of the low 54 bits),
 * 55 when those bits are all zero.  The salt is the 64-bit golden ratio
 * constant. */
int oracle_sketch(const uint8_t *packed, const uint64_t *offsets, uint64_t n_reads, int k,
                  uint32_t *regs) {
  const uint64_t salt = 0x9E3779B97F4A7C15ULL;
  if (!offsets || !regs || k < 2 || k > 32) return OR_ERR_ARG;
  for (int j = 0; j < 1024; ++j) regs[j] = 0;
  uint64_t maxlen = 0;
  for (uint64_t r = 0; r < n_reads; ++r) {
    if (offsets[r + 1] < offsets[r]) return OR_ERR_ARG;
    uint64_t len = offsets[r + 1] - offsets[r];
    if (len > maxlen) maxlen = len;
  }
  char *buf = (char *)malloc(maxlen + 1);
  if (!buf) return OR_ERR_NOMEM;
  const int m = k - 1;
  for (uint64_t r = 0; r < n_reads; ++r) {
    uint64_t len = offsets[r + 1] - offsets[r];
    if (len < (uint64_t)k) continue;
    unpack_range(packed, offsets[r], len, buf);
    for (uint64_t j = 0; j + (uint64_t)m <= len; ++j) { /* vertex positions 0 .. len-k+1 */
      uint64_t h = murmur3_fmix64(encode(buf + j, m) ^ salt);
      uint32_t idx = (uint32_t)(h >> 54);
      uint64_t rest = h << 10;
      uint32_t rho = 1;
      if (rest == 0) {
        rho = 55;
      } else {
        while (!(rest & 0x8000000000000000ULL)) {
          rest <<= 1;
          ++rho;
        }
      }
      if (rho > regs[idx]) regs[idx] = rho;
    }
  }
  free(buf);
  return OR_OK;
}
