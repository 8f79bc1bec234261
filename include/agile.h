/*
 * agile.h -- C-ABI of a GB300 (sm_103a) library for asynchronous GPU-centric page I/O
 * through an HBM software cache, after "AGILE: Lightweight and Efficient Asynchronous
 * GPU-SSD Integration" (arXiv 2504.19365).
 *
 * What the library computes (paper section in brackets):
 *   - NVMe-style submission/completion queue pairs held in HBM, filled by GPU threads
 *     that also write the tail doorbells themselves [Sec. 2.1, Sec. 3.3.1, Alg. 2];
 *   - a service role that polls completion queues one 32-entry window per warp and
 *     releases queue slots and per-request completion tokens [Sec. 3.2, Alg. 1];
 *   - a set-associative software cache of 4 KiB lines in HBM with the line states
 *     INVALID / BUSY / READY / MODIFIED and clock replacement [Sec. 3.4, Sec. 4.4];
 *   - warp-level and cache-level coalescing of requests for one page [Sec. 3.3.2];
 *   - an in-flight share table (page -> request in flight) [Sec. 3.4.1];
 *   - issue / continue / wait with completion tokens: no thread waits for a completion
 *     while it holds a queue slot or a cache line [Sec. 2.3.1, Sec. 2.3.2, Sec. 3.2.1];
 *   - drivers: sum-pooled embedding-bag lookups [Sec. 4.4], a CSR breadth-first search
 *     and an SpMV over the same CSR layout [Sec. 4.5], each in a synchronous mode
 *     (issue then stall) and an asynchronous mode (issue ahead, continue, wait later)
 *     [Sec. 4.2, Sec. 4.4]; the embedding bag also has a backward pass with an SGD
 *     step written back through the queues, a lookup + compute pipeline and a
 *     continuous-batching serving loop.
 *
 * The backing store is an emulated NVMe device: its data lives in pinned host memory
 * (reached over the host link), it consumes the 64-byte submission entries from the
 * HBM rings, copies 4 KiB pages between host memory and HBM, and posts 16-byte
 * completion entries with a phase bit.  Its latency and per-queue throughput are
 * configurable.  The device is emulated by warps of the same kernel launch that runs
 * the work, so it makes progress only while a library call is executing on the GPU;
 * every call drains the commands it issued before it returns on its stream.  When the
 * cache leaves enough application warps of a launch idle, those warps poll the
 * completion queues (one queue each) instead.
 *
 * Conventions
 *   - Ownership: the library owns the cache, queues, tokens, staging buffers and the
 *     pinned store.  The caller owns every buffer whose name starts with d_ (device
 *     memory, e.g. a torch tensor's data pointer) and every stream (a cudaStream_t
 *     passed as void*; NULL = legacy default stream).
 *   - Launches are asynchronous on `stream`.  A return value of 0 means the launch
 *     was accepted; errors found on the GPU (timeouts, device errors) are reported
 *     per token by agile_wait and sticky per context by agile_check.
 *   - Errors: 0 on success, else a negative AGILE_E* code.  Pointers that must not be
 *     NULL give AGILE_EINVAL.
 *   - One context may be used by one stream at a time; calls that overlap on the GPU
 *     for the same context race on its queues and cache.
 */
#ifndef AGILE_H
#define AGILE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define AGILE_API __attribute__((visibility("default")))
#else
#define AGILE_API
#endif

#define AGILE_PAGE_SIZE 4096u

/* error codes (negative) */
#define AGILE_OK 0
#define AGILE_EIO (-5)          /* a command completed with a non-zero status         */
#define AGILE_EAGAIN (-11)      /* no line or queue slot free right now               */
#define AGILE_ENOMEM (-12)      /* allocation failed                                  */
#define AGILE_ENODEV (-19)      /* no CUDA device / requested backing device absent   */
#define AGILE_EINVAL (-22)      /* bad argument                                       */
#define AGILE_ETIMEDOUT (-110)  /* a bounded wait on the GPU ran out                  */
#define AGILE_ECUDA (-1000)     /* a CUDA runtime call failed                         */

/* modes of the application drivers */
#define AGILE_SYNC 0u   /* each page is requested when needed and waited for at once */
#define AGILE_ASYNC 1u  /* pages are requested ahead, work continues, waits come later */

/* emulator fault injection flags (host-configured; no GPU fault is ever raised) */
#define AGILE_FAULT_EIO 1u        /* complete a fraction of commands with an error    */
#define AGILE_FAULT_DROP_CQE 2u   /* never post the completion of a fraction of them  */

/* token of a request: {queue:16 | slot:16 | ticket:32}; AGILE_TOKEN_HIT = served from
 * the cache without a command of its own */
typedef uint64_t agile_token;
#define AGILE_TOKEN_HIT (~(uint64_t)0)

typedef struct agile_ctx agile_ctx;

typedef struct {
  uint64_t store_bytes;     /* backing store size, multiple of 4096                    */
  const char *nvme_path;    /* NULL: emulated device (the only backend built)         */
  uint64_t cache_bytes;     /* HBM cache size; rounded down to ways*4096 multiples    */
  uint32_t ways;            /* associativity, 1..32                                   */
  uint32_t num_queues;      /* queue pairs, 1..65535                                  */
  uint32_t queue_depth;     /* entries per queue, power of two in [64, 65536]         */
  uint32_t emu_latency_ns;  /* per-command device latency (0 = none)                  */
  double emu_queue_gbps;    /* per-queue throughput cap in GB/s (0 = uncapped)        */
  uint64_t wait_timeout_ns; /* bound on every wait inside a call (0 = 10 s)           */
  int32_t device;           /* CUDA device ordinal                                    */
  uint32_t fault_flags;     /* AGILE_FAULT_* (0 = none)                               */
  double fault_rate;        /* fraction of commands hit by the injected fault         */
  uint64_t seed;            /* seed of the fault injector                             */
  uint32_t max_ctas;        /* cap on CTAs per launch (0 = all co-resident CTAs)      */
  uint32_t prefetch_depth;  /* async lookahead in work units (0 = default 1)          */
  uint32_t app_warps;       /* cap on application warps per call (0 = sized from the
                               cache so the warps' working set fits in it)           */
  uint32_t trace_records;   /* capacity of the device's command trace (0 = off); see
                               agile_trace                                           */
  uint32_t num_devices;     /* backing devices, 0 or 1 = one (Sec. 4.3): store page p
                               lives on device p mod n as its block p / n, and queue q
                               belongs to device q mod n (num_queues must be a
                               multiple of n), so requests interleave over devices  */
  uint32_t cache_policy;    /* AGILE_POLICY_CLOCK (default) or AGILE_POLICY_FIFO      */
  double emu_device_read_gbps;   /* per-device read throughput cap, GB/s (0 = none)  */
  double emu_device_write_gbps;  /* per-device write throughput cap, GB/s (0 = none) */
  uint32_t share_slots;     /* Share Table entries for user buffers (Sec. 3.4.1); 0 = no
                               Share Table (it is an option, as in the paper)        */
  uint32_t emu_extra_engines; /* application warps a call leaves idle that also serve the
                               emulated device, at most: 0 = one per CTA of the launch,
                               AGILE_NO_EXTRA_ENGINES = none (only warp 0 of each CTA) */
  uint32_t prefetch_queues; /* queue pairs that carry requests made ahead of need (the
                               asynchronous lookahead of the drivers, agile_prefetch);
                               the device serves the other, demand queues first (NVMe
                               arbitration with an urgent class), so prefetches only use
                               device time that demand leaves idle.  0 = half of the
                               queues (rounded to a multiple of num_devices; none with
                               fewer than 2 per device), AGILE_NO_PREFETCH_QUEUES = none:
                               every request shares every queue.  A call that makes no
                               request ahead of need (every SYNC call, asyncRead, BFS,
                               SpMV, serving) uses every queue for demand.  A lookahead
                               request of an application (embedding bag, pipeline,
                               backward) is a hint: it is dropped when its first queue
                               holds more than 3/4 of its depth in flight, or when two
                               queues of its class are full                          */
} agile_config;
#define AGILE_NO_EXTRA_ENGINES 0xFFFFFFFFu
#define AGILE_NO_PREFETCH_QUEUES 0xFFFFFFFFu

/* Replacement policies of the cache (Sec. 3.4 leaves the policy to the user; Sec. 4.4
 * uses clock).  Both pick a victim within the page's set starting at the set's hand and
 * skip ways that are in flight, pinned or being written back; an INVALID way is always
 * taken first (the lowest one).
 *   CLOCK: a way whose reference bit is set (by a hit, or by its fill) has it cleared
 *          and is passed over once.
 *   FIFO : the reference bit is ignored: the way at the hand is the victim, so (with
 *          nothing pinned or in flight) lines leave in the order they were filled. */
#define AGILE_POLICY_CLOCK 0u
#define AGILE_POLICY_FIFO 1u

typedef struct {
  uint64_t hits;            /* requests served by a READY/MODIFIED line (case a)      */
  uint64_t misses;          /* requests that issued a read (cases b, d)              */
  uint64_t busy_hits;       /* requests that found their page in flight (case c)     */
  uint64_t warp_coalesced;  /* requests merged by the warp-level match              */
  uint64_t share_retries;   /* misses deferred because the page's entry was taken    */
  uint64_t evictions;       /* valid victims replaced                                */
  uint64_t writebacks;      /* MODIFIED lines written back                           */
  uint64_t eagain;          /* victim searches that found nothing evictable          */
  uint64_t sq_full;         /* reservations that found every queue full             */
  uint64_t doorbells;       /* SQ tail doorbell writes                               */
  uint64_t commands;        /* commands consumed by the device                       */
  uint64_t cqes;            /* completions consumed by the pollers                   */
  uint64_t cq_doorbells;    /* CQ head doorbell writes (one per 32-entry window)     */
  uint64_t io_errors;       /* completions with a non-zero status                    */
  uint64_t bytes_read;      /* bytes the device moved store -> HBM                   */
  uint64_t bytes_written;   /* bytes the device moved HBM -> store                   */
  uint64_t prefetches;      /* prefetch requests issued                              */
  uint64_t timeouts;        /* bounded waits that ran out                            */
} agile_stats_t;

/* Fill *cfg with defaults: 128 queue pairs x 256 entries (Sec. 4.4 default), 8 ways,
 * no latency model, 10 s wait bound, device 0. */
AGILE_API void agile_config_default(agile_config *cfg);

/* Host initialisation (Listing 1 host side, Sec. 3.1): allocates the pinned store, the
 * HBM cache, the queue rings and the service state on cfg->device.  *out receives
 * the context.  AGILE_ENODEV if cfg->nvme_path is non-NULL (no real NVMe backend). */
AGILE_API int agile_init(const agile_config *cfg, agile_ctx **out);

/* Drain, flush MODIFIED lines to the store and free everything.  NULL is a no-op. */
AGILE_API int agile_destroy(agile_ctx *ctx);

/* Copy n bytes between host memory and the backing store at byte offset off
 * (host side, synchronous; the device is idle in between calls).  Cached lines of
 * the pages touched by agile_store_write are invalidated first, MODIFIED ones are
 * written back before.  AGILE_EINVAL if [off, off+n) leaves the store. */
AGILE_API int agile_store_write(agile_ctx *ctx, uint64_t off, const void *host_src, uint64_t n);
AGILE_API int agile_store_read(agile_ctx *ctx, uint64_t off, void *host_dst, uint64_t n);

/* asyncRead (Sec. 3.1, Listing 1 Method-2): for i < n, copy store page d_pages[i]
 * through the cache into d_dst + i*4096 and write its token to d_tok[i] (may be
 * NULL).  d_pages: uint64 page numbers; d_dst: n*4096 bytes, 16-byte aligned.
 * mode AGILE_ASYNC issues all misses of a warp's pages before waiting for any. */
AGILE_API int agile_read_async(agile_ctx *ctx, const uint64_t *d_pages, uint32_t n, void *d_dst,
                     agile_token *d_tok, uint32_t mode, void *stream);

/* asyncWrite (Sec. 3.5): for i < n, write d_src + i*4096 to store page d_pages[i]:
 * the cache line is updated and a write command is issued from a staging copy.
 * Pages must be distinct within one call. */
AGILE_API int agile_write_async(agile_ctx *ctx, const uint64_t *d_pages, uint32_t n,
                      const void *d_src, agile_token *d_tok, void *stream);

/* wait (Sec. 3.2.1, the per-request transaction barrier): d_status[i] = 0 when token i completed cleanly,
 * AGILE_EIO when it completed with an error, AGILE_ETIMEDOUT when it is still
 * outstanding after cfg->wait_timeout_ns. */
AGILE_API int agile_wait(agile_ctx *ctx, const agile_token *d_tok, uint32_t n, int32_t *d_status,
               void *stream);

/* prefetch (Sec. 3.1): start filling the cache with store pages d_pages[0..n). */
AGILE_API int agile_prefetch(agile_ctx *ctx, const uint64_t *d_pages, uint32_t n, void *stream);

/* Write every MODIFIED line back to the store (Sec. 3.4 case (d) write-back). */
AGILE_API int agile_flush(agile_ctx *ctx, void *stream);

/* Drop every line (flushes MODIFIED lines first); the next requests start cold. */
AGILE_API int agile_invalidate(agile_ctx *ctx, void *stream);

/* Sum-pooled embedding bag (Sec. 4.4): the table is `rows` x `dim` FP32 stored
 * row-major at byte table_byte0 of the store (multiple of 4096; dim a multiple of 4,
 * dim*4 <= 4096).  d_out[b*dim + d] = sum over i in [d_offsets[b], d_offsets[b+1])
 * of T[d_idx[i]][d], added in increasing i in FP32 (round to nearest, no fusion).
 * d_idx, d_offsets: int64; d_out: n_bags*dim floats.  Indices outside [0, rows) make
 * the call fail with AGILE_EINVAL reported through agile_check.
 * The call first sums, in a light kernel, every bag of at most 32 indices whose pages
 * are all resident; the engine launch then handles the others (scratch for their list
 * is allocated on first use and kept by the context).  mode AGILE_ASYNC requests the
 * pages of the rows ahead of the one being summed, while a warp's share of the cache
 * lines is at least 8; below that the call runs as AGILE_SYNC, since a line requested
 * ahead would be evicted before its use. */
AGILE_API int agile_embedding_bag(agile_ctx *ctx, uint64_t table_byte0, uint32_t rows, uint32_t dim,
                        const int64_t *d_idx, const int64_t *d_offsets, uint32_t n_bags,
                        float *d_out, uint32_t mode, void *stream);

/* Backward of agile_embedding_bag with a fused SGD step (differentiable extension of
 * the Sec. 4.4 lookups).  Same table and bag arguments as the forward; n_indices =
 * d_offsets[n_bags] (the length of d_idx); d_grad_out: n_bags*dim floats.
 * G[r][d] = sum over positions i with d_idx[i] = r of d_grad_out[bag(i)][d], added in
 * increasing i in FP32.  If d_grad_table != NULL it receives G (rows*dim floats, rows
 * never indexed are 0).  If lr != 0 every touched row is updated in the cache as
 * T[r][d] - (lr * G[r][d]) (product rounded first) and its line becomes MODIFIED; the
 * store sees the new rows after eviction write-backs or agile_flush.  mode AGILE_ASYNC
 * requests the pages of upcoming rows ahead.  Uses library scratch (sorted keys). */
AGILE_API int agile_embedding_bag_backward(agile_ctx *ctx, uint64_t table_byte0, uint32_t rows,
                                           uint32_t dim, const int64_t *d_idx,
                                           const int64_t *d_offsets, uint32_t n_bags,
                                           uint32_t n_indices, const float *d_grad_out, float lr,
                                           float *d_grad_table, uint32_t mode, void *stream);

/* Lookup + compute pipeline (the overlap experiment: Sec. 4.2 computation-to-
 * communication ratio, Sec. 4.4 prefetching the next batch while computing).
 * n_tables FP32 tables of rows x dim, table k at byte table_byte0 + k*table_stride
 * (both multiples of 4096).  d_idx: int64 [n_batches][n_tables][n_bags][pooling] row
 * numbers.  For every (batch t, bag b): out[t][b][k*dim + d] = sum over p of
 * T_k[idx[t][k][b][p]][d] in increasing p (FP32), then compute_iters rounds of
 * x = fma(x, 1 - 2^-12, 2^-10) per element.  d_out: float [n_batches][n_bags][n_tables*dim].
 * AGILE_SYNC requests each row when summed; AGILE_ASYNC keeps the pages of a warp's
 * upcoming rows requested ahead of its gather and compute: as many rows as the cache
 * holds for the warps running (half of its lines), at most one unit (n_tables *
 * pooling rows) ahead. */
AGILE_API int agile_embedding_pipeline(agile_ctx *ctx, uint64_t table_byte0, uint64_t table_stride,
                                       uint32_t n_tables, uint32_t rows, uint32_t dim,
                                       const int64_t *d_idx, uint32_t pooling, uint32_t n_bags,
                                       uint32_t n_batches, uint32_t compute_iters, float *d_out,
                                       uint32_t mode, void *stream);

/* Breadth-first search over a CSR graph on the store (Sec. 4.5): int64 offsets
 * [n_vertices+1] at byte offsets_byte0, int32 columns at byte cols_byte0 (both
 * multiples of 4096); 0 < n_vertices < 2^31.  d_level[v] = BFS level of v from src,
 * -1 when unreachable.  *d_edges_scanned (uint64, device, may be NULL) = sum of the
 * degrees of every reached vertex.  Top-down, level-synchronous.  AGILE_SYNC requests
 * every page when it is needed; AGILE_ASYNC issues the reads of the work at hand before
 * it waits for any of them: the list pages of a 32-vertex unit, those of a sparse
 * chunk's units, and every page of a slice of a long adjacency list. */
AGILE_API int agile_bfs(agile_ctx *ctx, uint64_t offsets_byte0, uint64_t cols_byte0,
              uint32_t n_vertices, int32_t src, int32_t *d_level,
              uint64_t *d_edges_scanned, uint32_t mode, void *stream);

/* Sparse matrix-vector product over a CSR matrix on the store (Sec. 4.5 runs SpMV
 * over the CSR graphs of its BFS): int64 offsets [n_rows+1] at byte offsets_byte0,
 * int32 column numbers at byte cols_byte0 and FP32 values at byte vals_byte0 (all
 * three multiples of 4096; entry j of the matrix is cols[j], vals[j]), read through
 * the cache.  d_x: float [n_cols] and d_y: float [n_rows], device memory of the
 * caller (16-byte alignment not required).  d_y[v] = sum over j in
 * [offsets[v], offsets[v+1]) of vals[j] * x[cols[j]] in FP32, each product rounded
 * before it is added, added in increasing j from +0 (equal bit for bit to that order
 * in every row: a row of 1024 entries or more is cut into slices of 1024 whose products
 * are computed in parallel, and each slice continues the running sum of the one
 * before).  A column number >= n_cols contributes 0 and records AGILE_EINVAL
 * (agile_check).
 * *d_entries (uint64, device, may be NULL) = number of entries (offsets[n_rows] -
 * offsets[0]).  mode as above.  Uses the library's slice-queue scratch (shared with
 * agile_bfs; allocated on first use). */
AGILE_API int agile_spmv(agile_ctx *ctx, uint64_t offsets_byte0, uint64_t cols_byte0, uint64_t vals_byte0,
                         uint32_t n_rows, uint32_t n_cols, const float *d_x, float *d_y,
                         uint64_t *d_entries, uint32_t mode, void *stream);

/* The embedding bag of agile_embedding_bag over a table held in device memory of the
 * caller (d_table: rows x dim floats, 16-byte aligned), without the cache or the queues:
 * the hit path's ceiling (plain gathers of the same rows in the same order; the same
 * bits) and the "kernel time" step of a breakdown like Sec. 4.5's.  A warp per bag;
 * indices outside [0, rows) read row 0 and record AGILE_EINVAL (agile_check).  Uses
 * the context only for its device and error word. */
AGILE_API int agile_embedding_bag_hbm(agile_ctx *ctx, const float *d_table, uint32_t rows, uint32_t dim,
                                      const int64_t *d_idx, const int64_t *d_offsets, uint32_t n_bags,
                                      float *d_out, void *stream);

/* Step 1 of the Sec. 4.5 three-step breakdown ("kernel time": the application kernel
 * with the graph in HBM, read with plain loads): the BFS of agile_bfs, the same kernel
 * and launch, over a CSR held in device memory of the caller instead of the store --
 * d_offsets int64 [n_vertices+1], d_cols int32 [n_cols] -- without the cache or the
 * queues.  Results as agile_bfs.  With agile_bfs on a cache preloaded with the whole
 * graph (step 3, cache API time) and on a cold cache (step 2, I/O API time) it splits
 * a BFS's time into kernel, cache and I/O parts.  Uses the context's launch shape and
 * BFS scratch (allocated on first use). */
AGILE_API int agile_bfs_hbm(agile_ctx *ctx, const int64_t *d_offsets, const int32_t *d_cols, uint32_t n_vertices,
                            uint64_t n_cols, int32_t src, int32_t *d_level, uint64_t *d_edges_scanned,
                            void *stream);

/* Step 1 of the Sec. 4.5 breakdown for agile_spmv: the same kernel over a CSR held in
 * device memory (d_offsets int64 [n_rows+1], d_cols int32 and d_vals float [n_entries]),
 * without the cache or the queues; results equal agile_spmv's bit for bit. */
AGILE_API int agile_spmv_hbm(agile_ctx *ctx, const int64_t *d_offsets, const int32_t *d_cols, const float *d_vals,
                             uint32_t n_rows, uint32_t n_cols, uint64_t n_entries, const float *d_x, float *d_y,
                             uint64_t *d_entries, void *stream);

/* BFS exactly as agile_bfs, for callers that cannot allocate device memory during the
 * call: code running under stream capture (where cudaMalloc is not allowed), or a
 * latency-critical loop where the device synchronisation that an allocation implies
 * would stall other streams.  The paper has no counterpart: it is an addition of this
 * library.  agile_bfs allocates a queue of long adjacency lists and a visited bitmap on
 * first use; this entry point uses fixed device arrays compiled into the library
 * instead (8 MiB and 4 MiB, held by every GPU that loads the library until the process
 * exits) and calls no cudaMalloc/cudaFree.  n_cols: number of int32 column entries of
 * the graph; graphs with more than 33,554,176 column entries (131,072 queue slots of
 * 256 entries) or more than 33,554,432 vertices are rejected with AGILE_EINVAL and a
 * message on stderr.  The first call on a device looks up the arrays' device addresses
 * (make that first call before any stream capture); the addresses are kept for the
 * process, so a device reset (cudaDeviceReset) between calls is not supported.  All
 * calls on a device share the arrays: calls of this entry point that overlap on one GPU
 * race.  Queue records from an earlier call never need clearing: each record is
 * published with a number the device draws for every kernel execution. */
AGILE_API int agile_bfs_noalloc(agile_ctx *ctx, uint64_t offsets_byte0, uint64_t cols_byte0,
                                uint32_t n_vertices, uint64_t n_cols, int32_t src, int32_t *d_level,
                                uint64_t *d_edges_scanned, uint32_t mode, void *stream);

/* Serving loop: continuous batching of lookup requests (serving extension of the
 * Sec. 4.4 lookups).  agile_serve_start launches one long-running call on `stream`
 * that keeps the queues, the emulated device and the cache resident for up to
 * session_ns (0 = 60 s); requests submitted meanwhile are admitted, oldest first, when
 * the free cache-line budget (half of the cache's lines; a request holds one line per
 * index + 1, at most the budget) covers them, or when nothing else runs, and are
 * served alongside the requests already running.  Queue slots need no budget: each is
 * returned by its completion, and a full queue sends a request to the next queue.  A request is one sum-pooled embedding bag exactly as computed by
 * agile_embedding_bag (same result alone or in any mix); its device buffers must be
 * written before it is submitted and left alone until it completes; dim <= 128.
 * While a session runs its kernel occupies every SM: launch no other kernel on the
 * device until agile_serve_stop returns (copies on other streams are fine). */
typedef struct {
  uint64_t table_byte0;     /* table at this byte offset of the store (multiple of 4096) */
  uint32_t rows, dim;
  const int64_t *d_idx;     /* row numbers                                           */
  const int64_t *d_offsets; /* n_bags + 1 bag boundaries                             */
  uint32_t n_bags;
  float *d_out;             /* n_bags * dim floats, 16-byte aligned                   */
} agile_lookup_req;
typedef struct agile_server agile_server;
/* ring_slots: requests that may be submitted and not yet finished. */
AGILE_API int agile_serve_start(agile_ctx *ctx, uint32_t ring_slots, uint32_t mode, uint64_t session_ns,
                                void *stream, agile_server **out);
/* Non-blocking; AGILE_EAGAIN when the ring is full.  *seq_out = the request's number. */
AGILE_API int agile_serve_submit(agile_server *srv, const agile_lookup_req *req, uint64_t *seq_out);
/* 1 when request `seq` has finished, 0 when not yet. */
AGILE_API int agile_serve_poll(agile_server *srv, uint64_t seq);
/* Finish every submitted request, end the session, free the server. */
AGILE_API int agile_serve_stop(agile_server *srv);
/* Replay a trace: request i is submitted at arrival_ns[i] (nanoseconds from the start,
 * non-decreasing); latency_ns[i] receives the time from its arrival to its completion
 * seen on the host.  Starts and stops its own session. */
AGILE_API int agile_serve_replay(agile_ctx *ctx, const agile_lookup_req *reqs, uint32_t n,
                                 const uint64_t *arrival_ns, uint64_t *latency_ns, uint32_t mode,
                                 void *stream);

/* Validation entry point: serve store pages d_pages[0..n) one at a time, in order, by
 * a single GPU thread (sync mode), and write the outcome of each request to
 * d_codes[i] (0 hit, 1 fill of an INVALID way, 2 eviction of a READY line, 3
 * write-back of a MODIFIED line).  With one request in flight the cache must behave
 * exactly like the sequential reference cache of Sec. 3.4 / Sec. 4.4. */
AGILE_API int agile_cache_replay(agile_ctx *ctx, const uint64_t *d_pages, uint32_t n, int32_t *d_codes,
                       void *stream);

/* Copy the cache tags to host: tag word per line (page << 20 | pin << 4 | ref << 2 |
 * state).  out must hold agile_cache_lines(ctx) words.  Synchronises the device. */
AGILE_API int agile_cache_tags(agile_ctx *ctx, uint64_t *host_out);
AGILE_API uint64_t agile_cache_lines(agile_ctx *ctx);
AGILE_API uint32_t agile_cache_sets(agile_ctx *ctx);

/* Counters since init or the last reset (synchronises the device). */
AGILE_API int agile_stats(agile_ctx *ctx, agile_stats_t *out);
AGILE_API int agile_reset_stats(agile_ctx *ctx);

/* Change the emulated device model of a context between calls (the device must be
 * idle: synchronises it first): number of backing devices (0 = 1; num_queues must be a
 * multiple), per-command latency, per-queue cap and per-device read/write caps, with
 * the meaning of the agile_config fields of the same names.  Store contents and cached
 * lines are unaffected; where a page lives only decides which queues serve it. */
AGILE_API int agile_set_device_model(agile_ctx *ctx, uint32_t num_devices, uint32_t emu_latency_ns,
                                     double emu_queue_gbps, double emu_device_read_gbps,
                                     double emu_device_write_gbps);

/* Per-page accounting of the emulated device since init or the last agile_reset_stats
 * (synchronises the device).  For store pages page0 .. page0+n-1, any of the host arrays
 * may be NULL:
 *   reads[i]   read commands the device served for the page (store -> HBM),
 *   writes[i]  write commands it served for the page (HBM -> store),
 *   dirtied[i] dirty epochs of the page: times a clean cache line of it turned MODIFIED
 *              or a page write (agile_write_async) was started.
 * Every dirty epoch ends in exactly one write (Sec. 3.4 case (d)): after agile_flush,
 * writes[i] == dirtied[i] for every page.  AGILE_EINVAL if the range leaves the store. */
AGILE_API int agile_page_io(agile_ctx *ctx, uint64_t page0, uint64_t n, uint32_t *host_reads,
                            uint32_t *host_writes, uint32_t *host_dirtied);

/* One command as the emulated device served it; times are the GPU's global timer in ns. */
typedef struct {
  uint64_t page;     /* store page                                                      */
  uint64_t t_seen;   /* doorbell that exposed the command first read by the device (0 when
                        the device has no latency or throughput model)                  */
  uint64_t t_start;  /* an engine took the command; its data moves from here            */
  uint64_t t_done;   /* its completion entry was posted                                 */
  uint32_t q, cid, opcode, status;  /* queue, command id, 0 flush/no-op 1 write 2 read,
                                       NVMe status (bit 16: completion dropped by the
                                       fault injector)                                  */
  uint64_t t_commit; /* the command was written to its submission slot (carried in the
                        command's reserved dwords 2-3)                                  */
  uint32_t pad[2];
} agile_trace_rec;

/* Copy the device's command trace (cfg.trace_records > 0) to host: up to `cap` records
 * into host_out, in the order engines took them; *n_out = records logged since init or
 * the last agile_reset_stats (may exceed the trace's capacity; later ones are dropped).
 * Synchronises the device. */
AGILE_API int agile_trace(agile_ctx *ctx, agile_trace_rec *host_out, uint32_t cap, uint32_t *n_out);

/* Application events logged since init or the last agile_reset_stats (only with
 * cfg.trace_records > 0, up to that many): out[2i] = time (GPU global timer, ns),
 * out[2i+1] = warp | kind << 32 | arg << 40.  The BFS logs, per application warp and
 * level (arg): kind 1 its own vertices done, 2 the level's long-list slices done, 3 the
 * level's barrier passed.  *n_out = events logged.  Synchronises the device. */
AGILE_API int agile_events(agile_ctx *ctx, uint64_t *out, uint32_t cap, uint32_t *n_out);

/* Host-link read bandwidth as the emulated device's engines see it: a kernel of
 * `ctas` CTAs (0 = two per SM) streams `bytes` (a multiple of 4096) from the context's
 * pinned store into d_dst with 16-byte loads, `reps` times; *gbps_out = best rate.
 * A measurement aid, not part of the paper's method. */
AGILE_API int agile_link_probe(agile_ctx *ctx, void *d_dst, uint64_t bytes, uint32_t ctas, uint32_t reps,
                               double *gbps_out);

/* For user kernels launched by agile_device.cuh (agile::launch_user): copy the
 * context's device view (the library's agile::Dev: addresses of the cache, queues and
 * device model) into *out, which has `size` bytes; AGILE_EINVAL unless size equals the
 * library's view (a header of another version).  Makes the device current. */
AGILE_API int agile_device_view(agile_ctx *ctx, void *out, uint64_t size);

/* For agile::launch_user: zero the context's per-launch state and number the launch, on
 * `stream`, right before a user launch. */
AGILE_API int agile_run_reset(agile_ctx *ctx, void *stream);

/* Validation of the Share Table (Sec. 3.4.1; needs cfg.share_slots > 0): one GPU thread
 * runs the operations d_ops[4i .. 4i+3] = {op, page, a, b} one after the other --
 * op 0: acquire `page` into user buffer a (the buffer d_bufs + a*4096; the page is
 * copied from its cache line when cached, else read from the store into the buffer; an
 * entry of the page already there is shared instead and its buffer returned), waiting
 * for the fill; op 1: write 16 bytes of value b at byte offset a of the page's buffer
 * and mark it modified; op 2: release the page (the last release of a modified buffer
 * writes it into the page's cache line, which turns MODIFIED).  d_out[3i .. 3i+2] =
 * {op 0: index of the buffer returned, op 2: 1 if this release wrote the buffer into the
 * cache; the entry's state (0 none, 1 E, 2 S, 3 M, 4 O) and count afterwards}.  Served
 * one at a time the table must decide as the sequential Share Table does.  The device
 * side for user kernels is in agile_device.cuh. */
AGILE_API int agile_share_replay(agile_ctx *ctx, const int32_t *d_ops, uint32_t n, void *d_bufs, int32_t *d_out,
                                 void *stream);

/* Lock-order checker (in place of the paper's debug lock chain, Sec. 3.5): a host-side
 * analysis of a log of lock events.  Each blocking acquire of a lock while the thread
 * holds others adds the order "held before acquired"; a try-acquire, which never
 * waits, adds none.  An order that closes a cycle (including re-acquiring a held lock)
 * is a way for threads to wait for each other forever.  Returns the number of acquires
 * that closed a cycle (0: the order is consistent) or AGILE_EINVAL; the first cycle's
 * locks go to cycle_out (up to cap), its length to *cycle_len (may be NULL). */
#define AGILE_LOCK_ACQUIRE 0u
#define AGILE_LOCK_RELEASE 1u
#define AGILE_LOCK_TRY 2u
typedef struct {
  uint32_t thread;  /* who                                  */
  uint32_t op;      /* AGILE_LOCK_ACQUIRE / _RELEASE / _TRY  */
  uint64_t lock;    /* which lock                           */
} agile_lock_event;
AGILE_API int agile_lock_order_check(const agile_lock_event *ev, uint64_t n, uint64_t *cycle_out, uint32_t cap,
                                     uint32_t *cycle_len);

/* Synchronise the device and return the first error recorded on the GPU since the
 * last agile_check (0 if none), clearing it. */
AGILE_API int agile_check(agile_ctx *ctx);

/* Kernel parallelism (Listing 1 host side, configKernelParallelism): cap on the
 * application warps of the following calls (0 = sized from the cache per call). */
AGILE_API int agile_config_parallelism(agile_ctx *ctx, uint32_t app_warps);

/* Grid used by the library's kernels: CTAs per launch and threads per CTA. */
AGILE_API int agile_launch_shape(agile_ctx *ctx, uint32_t *ctas, uint32_t *threads);

AGILE_API const char *agile_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* AGILE_H */
