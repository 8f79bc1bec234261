/*
 * CPU oracle for the AGILE asynchronous GPU-SSD I/O path (arXiv 2504.19365).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call this
 * file: only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * use it.  It shares no code, header or table with the CUDA library.
 *
 * Plain, slow, sequential C.  Every function restates a definition from the paper (or,
 * where the paper is silent, the reading recorded in the design notes) without any
 * blocking, fusion or reordering:
 *
 *   - page store          : a flat byte array addressed in 4 KiB pages (Sec. 2.3.3: flash
 *                           is managed in 4 KB pages and cache lines align with them).
 *   - reference cache     : a sequential set-associative software cache with the line
 *                           states of Sec. 3.4 (INVALID / READY / MODIFIED; BUSY is never
 *                           observable when requests are served one at a time) and clock
 *                           replacement (Sec. 4.4 names the clock policy of Corbato 1968).
 *   - share table         : user buffers shared by pointer with a reference count and
 *                           MOESI-inspired states; a modified buffer is propagated into
 *                           the cache by its last release (Sec. 3.4.1).
 *   - embedding bag       : sum pooling of table rows, one FP32 accumulator per output
 *                           element, indices added in increasing order (Sec. 4.4 DLRM
 *                           lookups); backward scatter-add and an SGD step.
 *   - BFS                 : textbook FIFO-queue breadth-first search over CSR (Sec. 4.5).
 *   - SpMV                : y = A x over the same CSR layout plus FP32 values (Sec. 4.5
 *                           runs SpMV on the graphs of its BFS), one FP32 accumulator per
 *                           row, entries added in increasing order, each product rounded
 *                           before it is added.
 *   - compute phase       : the FP32 multiply-add chain that follows each lookup batch
 *                           in the overlap experiment (Sec. 4.2).
 *   - ideal speedup       : Eq. 1.
 *
 * Floating point: compiled with -ffp-contract=off so that a*b+c is never fused.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PAGE 4096u

/* ------------------------------------------------------------------ page store */

/* Read page p of the store (Sec. 2.3.3: the store is addressed in 4 KiB pages). */
void orc_store_read_page(const uint8_t *store, uint64_t page, uint8_t *out) {
  memcpy(out, store + page * ORC_PAGE, ORC_PAGE);
}

void orc_store_write_page(uint8_t *store, uint64_t page, const uint8_t *in) {
  memcpy(store + page * ORC_PAGE, in, ORC_PAGE);
}

/* ------------------------------------------------------------------ reference cache */

enum { ORC_INVALID = 0, ORC_BUSY = 1, ORC_READY = 2, ORC_MODIFIED = 3 };

enum {
  ORC_HIT = 0,          /* case (a): READY or MODIFIED line holds the page           */
  ORC_MISS_FILL = 1,    /* case (b): an INVALID way is filled                         */
  ORC_MISS_EVICT = 2,   /* case (d): a READY victim is reset and refilled             */
  ORC_MISS_WRITEBACK = 3 /* case (d): a MODIFIED victim is written back, then refilled */
};

typedef struct {
  uint32_t sets, ways;
  uint64_t *page;   /* [sets*ways] page held by the way                    */
  uint8_t *state;   /* [sets*ways] ORC_INVALID / ORC_READY / ORC_MODIFIED  */
  uint8_t *ref;     /* [sets*ways] clock reference bit                     */
  uint32_t *hand;   /* [sets] clock hand                                   */
  uint8_t *data;    /* [sets*ways*4096] line contents                      */
  uint64_t hits, misses, evictions, writebacks;
  uint64_t *wb_log; /* pages written back, in order                         */
  uint64_t wb_cap, wb_len;
  int policy;       /* ORC_POLICY_CLOCK or ORC_POLICY_FIFO                 */
  uint64_t *filled; /* [sets*ways] order in which the way was last filled  */
  uint64_t fills;   /* fills so far                                        */
} orc_cache;

/* Replacement policies.  Sec. 3.4 leaves the policy to the user and Sec. 4.4 runs
 * clock; FIFO is the textbook first-in first-out rule (the way filled earliest leaves
 * first, whatever its use since). */
enum { ORC_POLICY_CLOCK = 0, ORC_POLICY_FIFO = 1 };

/* Set index of a page: the 64-bit golden-ratio multiplicative hash, whose upper 32
 * bits are reduced to [0, sets) by a multiply-shift.  Any number of sets works. */
uint32_t orc_set_of(uint64_t page, uint32_t sets) {
  uint64_t h = page * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(((h >> 32) * (uint64_t)sets) >> 32);
}

orc_cache *orc_cache_new(uint32_t sets, uint32_t ways, uint64_t wb_cap) {
  orc_cache *c = (orc_cache *)calloc(1, sizeof(orc_cache));
  uint64_t n = (uint64_t)sets * ways;
  c->sets = sets;
  c->ways = ways;
  c->page = (uint64_t *)calloc(n, sizeof(uint64_t));
  c->state = (uint8_t *)calloc(n, 1);
  c->ref = (uint8_t *)calloc(n, 1);
  c->hand = (uint32_t *)calloc(sets, sizeof(uint32_t));
  c->data = (uint8_t *)calloc(n, ORC_PAGE);
  c->wb_cap = wb_cap;
  c->wb_log = (uint64_t *)calloc(wb_cap ? wb_cap : 1, sizeof(uint64_t));
  c->filled = (uint64_t *)calloc(n, sizeof(uint64_t));
  c->policy = ORC_POLICY_CLOCK;
  return c;
}

void orc_cache_set_policy(orc_cache *c, int policy) { c->policy = policy; }

void orc_cache_free(orc_cache *c) {
  if (!c) return;
  free(c->page); free(c->state); free(c->ref); free(c->hand); free(c->data); free(c->wb_log);
  free(c->filled);
  free(c);
}

static void orc_log_wb(orc_cache *c, uint64_t page) {
  if (c->wb_len < c->wb_cap) c->wb_log[c->wb_len] = page;
  c->wb_len++;
  c->writebacks++;
}

/*
 * One request for `page`, served to completion before the next (Sec. 3.4 cases):
 *   (a) a way holds the page in READY or MODIFIED           -> hit, reference bit set;
 *   (b) otherwise the lowest INVALID way of the set is filled from the store;
 *   (d) otherwise the clock picks a victim: starting at the set's hand, a way whose
 *       reference bit is set has it cleared and the hand moves on; the first way with a
 *       clear bit is the victim and the hand moves past it (FIFO policy instead: the
 *       way filled earliest is the victim).  A MODIFIED victim is written back to the
 *       store first.  The filled line gets its reference bit set.
 * On return *way_out is the way now holding the page and the code says which case ran.
 * `store` is read on a fill and written on a write-back.
 */
int orc_cache_lookup(orc_cache *c, uint8_t *store, uint64_t page, uint32_t *way_out,
                     uint64_t *victim_page) {
  uint32_t s = orc_set_of(page, c->sets);
  uint64_t base = (uint64_t)s * c->ways;
  for (uint32_t w = 0; w < c->ways; ++w) {
    uint8_t st = c->state[base + w];
    if ((st == ORC_READY || st == ORC_MODIFIED) && c->page[base + w] == page) {
      c->ref[base + w] = 1;
      c->hits++;
      *way_out = w;
      return ORC_HIT;
    }
  }
  c->misses++;
  int code = ORC_MISS_FILL;
  uint32_t victim = c->ways;
  for (uint32_t w = 0; w < c->ways; ++w) {
    if (c->state[base + w] == ORC_INVALID) { victim = w; break; }
  }
  if (victim == c->ways && c->policy == ORC_POLICY_FIFO) {
    /* FIFO: the way filled earliest */
    victim = 0;
    for (uint32_t w = 1; w < c->ways; ++w)
      if (c->filled[base + w] < c->filled[base + victim]) victim = w;
  } else if (victim == c->ways) {
    /* clock sweep: at most one full pass clears every bit, the next step finds a 0 */
    for (uint32_t step = 0; step < 2 * c->ways + 1; ++step) {
      uint32_t w = c->hand[s];
      c->hand[s] = (w + 1) % c->ways;
      if (c->ref[base + w]) {
        c->ref[base + w] = 0;
      } else {
        victim = w;
        break;
      }
    }
  }
  if (c->state[base + victim] != ORC_INVALID) {
    uint64_t old = c->page[base + victim];
    if (victim_page) *victim_page = old;
    c->evictions++;
    if (c->state[base + victim] == ORC_MODIFIED) {
      memcpy(store + old * ORC_PAGE, c->data + (base + victim) * ORC_PAGE, ORC_PAGE);
      orc_log_wb(c, old);
      code = ORC_MISS_WRITEBACK;
    } else {
      code = ORC_MISS_EVICT;
    }
  }
  memcpy(c->data + (base + victim) * ORC_PAGE, store + page * ORC_PAGE, ORC_PAGE);
  c->page[base + victim] = page;
  c->state[base + victim] = ORC_READY;
  c->ref[base + victim] = 1;
  c->filled[base + victim] = ++c->fills;
  *way_out = victim;
  return code;
}

/* Read `len` bytes at byte offset `off` inside `page` through the cache. */
int orc_cache_read(orc_cache *c, uint8_t *store, uint64_t page, uint32_t off, uint32_t len,
                   uint8_t *out) {
  uint32_t w;
  int code = orc_cache_lookup(c, store, page, &w, NULL);
  uint64_t line = (uint64_t)orc_set_of(page, c->sets) * c->ways + w;
  memcpy(out, c->data + line * ORC_PAGE + off, len);
  return code;
}

/*
 * Write `len` bytes at byte offset `off` of `page` through the cache.
 * write_through = 0: write-back policy, the line becomes MODIFIED (Sec. 3.4 case (d)
 *                    writes it back on eviction).
 * write_through = 1: the line is updated and the page is written to the store at once,
 *                    the line stays READY (Sec. 3.5: an async write updates the cache
 *                    and issues the write command).
 * A missing page is first filled from the store (write-allocate).
 */
int orc_cache_write(orc_cache *c, uint8_t *store, uint64_t page, uint32_t off, uint32_t len,
                    const uint8_t *in, int write_through) {
  uint32_t w;
  int code = orc_cache_lookup(c, store, page, &w, NULL);
  uint64_t line = (uint64_t)orc_set_of(page, c->sets) * c->ways + w;
  memcpy(c->data + line * ORC_PAGE + off, in, len);
  if (write_through) {
    memcpy(store + page * ORC_PAGE, c->data + line * ORC_PAGE, ORC_PAGE);
    if (c->state[line] != ORC_MODIFIED) c->state[line] = ORC_READY;
  } else {
    c->state[line] = ORC_MODIFIED;
  }
  return code;
}

/* Write every MODIFIED line back, in line order, and mark it READY. */
uint64_t orc_cache_flush(orc_cache *c, uint8_t *store) {
  uint64_t n = (uint64_t)c->sets * c->ways, cnt = 0;
  for (uint64_t l = 0; l < n; ++l) {
    if (c->state[l] == ORC_MODIFIED) {
      memcpy(store + c->page[l] * ORC_PAGE, c->data + l * ORC_PAGE, ORC_PAGE);
      orc_log_wb(c, c->page[l]);
      c->state[l] = ORC_READY;
      cnt++;
    }
  }
  return cnt;
}

/* Replay a trace of page reads; outcome codes go to codes[i] (may be NULL). */
void orc_cache_replay(orc_cache *c, uint8_t *store, const uint64_t *pages, uint64_t n,
                      int32_t *codes) {
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t w;
    int code = orc_cache_lookup(c, store, pages[i], &w, NULL);
    if (codes) codes[i] = code;
  }
}

void orc_cache_counters(const orc_cache *c, uint64_t out[4]) {
  out[0] = c->hits; out[1] = c->misses; out[2] = c->evictions; out[3] = c->writebacks;
}

uint64_t orc_cache_wb_log(const orc_cache *c, uint64_t *out, uint64_t cap) {
  uint64_t n = c->wb_len < c->wb_cap ? c->wb_len : c->wb_cap;
  if (n > cap) n = cap;
  memcpy(out, c->wb_log, n * sizeof(uint64_t));
  return c->wb_len;
}

/* Export tags: page[l], state[l], ref[l] for every line l = set*ways + way. */
void orc_cache_tags(const orc_cache *c, uint64_t *page, uint8_t *state, uint8_t *ref) {
  uint64_t n = (uint64_t)c->sets * c->ways;
  memcpy(page, c->page, n * sizeof(uint64_t));
  memcpy(state, c->state, n);
  memcpy(ref, c->ref, n);
}

void orc_cache_line(const orc_cache *c, uint64_t line, uint8_t *out) {
  memcpy(out, c->data + line * ORC_PAGE, ORC_PAGE);
}

/* ------------------------------------------------------------------ share table */

/*
 * Share Table of Sec. 3.4.1 (user-specified buffers shared by pointer, MOESI-inspired),
 * served one operation at a time.  An entry maps a page to the user buffer that holds
 * it, with a reference count and a state:
 *   E  one user, buffer equal to the page         S  several users, equal to the page
 *   M  one user, buffer modified                  O  several users, buffer modified
 *   (no entry = I)
 * acquire(page, mine): if an entry holds the page, its buffer is returned and its count
 *   goes up (E -> S, M -> O: the data is shared by pointer, nothing is copied); else
 *   `mine` is registered (E, count 1) and filled with the page: from its cache line if
 *   the cache holds it (a hit, which sets the line's reference bit), else straight from
 *   the store (the cache is left as it is).
 * write(page, off, data): into the entry's buffer; E -> M, S -> O.
 * release(page): the count goes down; at zero a modified buffer (M or O) is propagated
 *   into the software cache -- the page's line gets the buffer's bytes and turns
 *   MODIFIED (case (d) writes it back later) -- and the entry goes away.  Who releases
 *   last does this on the owner's behalf (the owner may have released first).
 * Buffers are 4096-byte slots of `bufs`, named by index.
 */
enum { ORC_UB_I = 0, ORC_UB_E = 1, ORC_UB_S = 2, ORC_UB_M = 3, ORC_UB_O = 4 };

typedef struct {
  orc_cache *cache;
  uint32_t cap;
  uint64_t *page;
  int32_t *buf;
  uint32_t *ref;
  uint8_t *state;
  uint64_t store_reads, cache_copies, propagations;
} orc_share;

orc_share *orc_share_new(orc_cache *cache, uint32_t cap) {
  orc_share *t = (orc_share *)calloc(1, sizeof(orc_share));
  t->cache = cache;
  t->cap = cap;
  t->page = (uint64_t *)calloc(cap, sizeof(uint64_t));
  t->buf = (int32_t *)calloc(cap, sizeof(int32_t));
  t->ref = (uint32_t *)calloc(cap, sizeof(uint32_t));
  t->state = (uint8_t *)calloc(cap, 1);
  return t;
}

void orc_share_free(orc_share *t) {
  if (!t) return;
  free(t->page); free(t->buf); free(t->ref); free(t->state);
  free(t);
}

static int64_t orc_share_find(const orc_share *t, uint64_t page) {
  for (uint32_t i = 0; i < t->cap; ++i)
    if (t->state[i] != ORC_UB_I && t->page[i] == page) return i;
  return -1;
}

/* Returns the buffer now holding the page (-1 when the table is full). */
int32_t orc_share_acquire(orc_share *t, uint8_t *store, uint8_t *bufs, uint64_t page, int32_t mine) {
  int64_t e = orc_share_find(t, page);
  if (e >= 0) {
    t->ref[e] += 1;
    if (t->state[e] == ORC_UB_E) t->state[e] = ORC_UB_S;
    if (t->state[e] == ORC_UB_M) t->state[e] = ORC_UB_O;
    return t->buf[e];
  }
  for (uint32_t i = 0; i < t->cap; ++i) {
    if (t->state[i] != ORC_UB_I) continue;
    t->page[i] = page;
    t->buf[i] = mine;
    t->ref[i] = 1;
    t->state[i] = ORC_UB_E;
    uint8_t *dst = bufs + (uint64_t)mine * ORC_PAGE;
    orc_cache *c = t->cache;
    uint32_t s = orc_set_of(page, c->sets);
    uint64_t base = (uint64_t)s * c->ways;
    for (uint32_t w = 0; w < c->ways; ++w) {
      uint8_t st = c->state[base + w];
      if ((st == ORC_READY || st == ORC_MODIFIED) && c->page[base + w] == page) {
        memcpy(dst, c->data + (base + w) * ORC_PAGE, ORC_PAGE);
        c->ref[base + w] = 1;
        t->cache_copies++;
        return mine;
      }
    }
    memcpy(dst, store + page * ORC_PAGE, ORC_PAGE);
    t->store_reads++;
    return mine;
  }
  return -1;
}

/* Write into the buffer that holds `page` (which must be acquired). */
void orc_share_write(orc_share *t, uint8_t *bufs, uint64_t page, uint32_t off, const uint8_t *data,
                     uint32_t len) {
  int64_t e = orc_share_find(t, page);
  if (e < 0) return;
  memcpy(bufs + (uint64_t)t->buf[e] * ORC_PAGE + off, data, len);
  if (t->state[e] == ORC_UB_E) t->state[e] = ORC_UB_M;
  if (t->state[e] == ORC_UB_S) t->state[e] = ORC_UB_O;
}

/* Returns 1 when this release propagated a modified buffer into the cache. */
int orc_share_release(orc_share *t, uint8_t *store, uint8_t *bufs, uint64_t page) {
  int64_t e = orc_share_find(t, page);
  if (e < 0) return 0;
  t->ref[e] -= 1;
  if (t->ref[e] > 0) return 0;
  int prop = t->state[e] == ORC_UB_M || t->state[e] == ORC_UB_O;
  if (prop) {
    orc_cache_write(t->cache, store, page, 0, ORC_PAGE, bufs + (uint64_t)t->buf[e] * ORC_PAGE, 0);
    t->propagations++;
  }
  t->state[e] = ORC_UB_I;
  return prop;
}

/* state (ORC_UB_*) and count of the entry holding `page` (I and 0 when none) */
void orc_share_entry(const orc_share *t, uint64_t page, int32_t out[3]) {
  int64_t e = orc_share_find(t, page);
  out[0] = e >= 0 ? t->state[e] : ORC_UB_I;
  out[1] = e >= 0 ? (int32_t)t->ref[e] : 0;
  out[2] = e >= 0 ? t->buf[e] : -1;
}

void orc_share_counters(const orc_share *t, uint64_t out[3]) {
  out[0] = t->store_reads; out[1] = t->cache_copies; out[2] = t->propagations;
}

/* ------------------------------------------------------------------ embedding bag */

/*
 * Sum-pooled embedding bag: out[b, d] = sum over i in [off[b], off[b+1]) of T[idx[i], d],
 * one FP32 accumulator per (b, d) starting at +0.0, indices added in increasing i.
 */
void orc_embedding_bag(const float *table, uint64_t rows, uint32_t dim, const int64_t *idx,
                       const int64_t *off, uint64_t n_bags, float *out) {
  (void)rows;
  for (uint64_t b = 0; b < n_bags; ++b) {
    for (uint32_t d = 0; d < dim; ++d) {
      float acc = 0.0f;
      for (int64_t i = off[b]; i < off[b + 1]; ++i) acc = acc + table[(uint64_t)idx[i] * dim + d];
      out[b * dim + d] = acc;
    }
  }
}

/*
 * Backward of the sum-pooled bag: G[r, d] = sum over every (b, i) with idx[i] = r of
 * gout[b, d], added in increasing (b, i) order into one FP32 accumulator per (r, d)
 * starting at +0.0.  touched[r] = 1 for each row that occurs.
 */
void orc_embedding_bag_backward(uint64_t rows, uint32_t dim, const int64_t *idx,
                                const int64_t *off, uint64_t n_bags, const float *gout,
                                float *G, uint8_t *touched) {
  memset(G, 0, rows * dim * sizeof(float));
  memset(touched, 0, rows);
  for (uint64_t b = 0; b < n_bags; ++b) {
    for (int64_t i = off[b]; i < off[b + 1]; ++i) {
      uint64_t r = (uint64_t)idx[i];
      touched[r] = 1;
      for (uint32_t d = 0; d < dim; ++d) G[r * dim + d] = G[r * dim + d] + gout[b * dim + d];
    }
  }
}

/* SGD on the touched rows: T[r, d] = T[r, d] - (lr * G[r, d]), product rounded first. */
void orc_sgd(float *table, uint64_t rows, uint32_t dim, const float *G, const uint8_t *touched,
             float lr) {
  for (uint64_t r = 0; r < rows; ++r) {
    if (!touched[r]) continue;
    for (uint32_t d = 0; d < dim; ++d) {
      float step = lr * G[r * dim + d];
      table[r * dim + d] = table[r * dim + d] - step;
    }
  }
}

/* ------------------------------------------------------------------ compute phase */

/*
 * Synthetic FP32 compute that follows each lookup batch in the overlap experiment
 * (Sec. 4.2: computation whose length sets the computation-to-communication ratio):
 * every element goes through `iters` fused multiply-adds x = fma(x, a, b), each
 * rounded once (C99 fmaf).
 */
void orc_fma_chain(float *x, uint64_t n, uint32_t iters, float a, float b) {
  for (uint64_t i = 0; i < n; ++i) {
    float v = x[i];
    for (uint32_t k = 0; k < iters; ++k) v = fmaf(v, a, b);
    x[i] = v;
  }
}

/* ------------------------------------------------------------------ BFS */

/*
 * Textbook breadth-first search with a FIFO queue over a CSR graph.
 * level[src] = 0, level[v] = level[u] + 1 for the first u that discovers v, -1 when
 * unreachable.  Returns the number of CSR entries scanned: the sum of the degrees of
 * every reached vertex (each vertex is dequeued once and scans its whole list).
 */
uint64_t orc_bfs(uint64_t n, const int64_t *offsets, const int32_t *cols, int32_t src,
                 int32_t *level) {
  for (uint64_t v = 0; v < n; ++v) level[v] = -1;
  if (n == 0 || src < 0 || (uint64_t)src >= n) return 0;
  int32_t *queue = (int32_t *)malloc(n * sizeof(int32_t));
  uint64_t head = 0, tail = 0, scanned = 0;
  level[src] = 0;
  queue[tail++] = src;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t e = offsets[u]; e < offsets[u + 1]; ++e) {
      int32_t v = cols[e];
      scanned++;
      if (level[v] < 0) {
        level[v] = level[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return scanned;
}

/* ------------------------------------------------------------------ Eq. 1 */

/* Ideal overlap speedup of Eq. 1: 1 + CTC for 0 <= CTC <= 1, else 1 + 1/CTC. */
/* SpMV over CSR (Sec. 4.5): y[v] = sum over j in [offsets[v], offsets[v+1]) of
 * vals[j] * x[cols[j]], the sum taken in increasing j in FP32 starting from +0, each
 * product rounded to FP32 before it is added (no fused multiply-add).  Returns the
 * number of entries (the CSR size). */
uint64_t orc_spmv(uint64_t n, const int64_t *offsets, const int32_t *cols, const float *vals, const float *x,
                  float *y) {
  for (uint64_t v = 0; v < n; ++v) {
    float acc = 0.0f;
    for (int64_t j = offsets[v]; j < offsets[v + 1]; ++j) {
      float prod = vals[j] * x[cols[j]];
      acc = acc + prod;
    }
    y[v] = acc;
  }
  return n ? (uint64_t)offsets[n] : 0;
}

double orc_ideal_speedup(double ctc) {
  if (ctc < 0) return 0.0 / 0.0;
  return ctc <= 1.0 ? 1.0 + ctc : 1.0 + 1.0 / ctc;
}
