// Host side of the library (context, store, counters) and the page-level calls:
// asyncRead / asyncWrite / wait / prefetch / flush / invalidate / replay.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "agile.h"
#include "agile_ctx.cuh"
#include "agile_dev.cuh"

using namespace agile;

// ============================================================================ apps

namespace {

__device__ __forceinline__ bool page_ok(const Dev &d, uint64_t page) {
  return page < d.store_bytes / kPage;
}

// asyncRead / prefetch (Sec. 3.1, Listing 1 Methods 1 and 2).  Each app warp takes 32
// requests at a time.  prefetch_only: issue the misses and return.  Otherwise every
// page is copied line -> d_dst with the line pinned for the copy only.  ASYNC issues
// every miss of the 32 requests before the first wait; SYNC requests each page and
// waits for it before requesting the next.
struct ReadApp {
  const uint64_t *pages;
  uint32_t n;
  uint8_t *dst;
  uint64_t *tok;
  uint32_t mode;
  // no request ahead of need: the launch uses every queue pair for demand
  bool demand_only() const { return !prefetch_only; }  // reads are waited for in both modes
  int prefetch_only;
  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    for (uint64_t base = (uint64_t)a.warp * 32; base < n; base += (uint64_t)a.n_warps * 32) {
      uint64_t i = base + l;
      bool want = i < n;
      uint64_t page = want ? pages[i] : 0;
      if (want && !page_ok(d, page)) {
        set_error(d, AGILE_EINVAL);
        want = false;
      }
      if (aborted(d)) return;
      if (prefetch_only) {
        stat_warp(d, S_PREFETCHES, want ? 1u : 0u);
        if (!warp_request(d, want, page, a.q0, false, a.deadline, nullptr, nullptr, nullptr, true)) return;
        continue;
      }
      uint64_t t = AGILE_TOKEN_HIT;
      unsigned grp = __match_any_sync(kFull, want ? page : ~0ull);
      if (mode == AGILE_ASYNC) {
        if (!warp_request(d, want, page, a.q0, false, a.deadline, &t)) return;
      }
      uint32_t cnt = (uint32_t)min((uint64_t)32, n - base);
      for (uint32_t j = 0; j < cnt; ++j) {
        uint64_t pj = __shfl_sync(kFull, page, j);
        if (!__shfl_sync(kFull, (int)want, j)) continue;
        if (mode != AGILE_ASYNC) {
          uint64_t tj = AGILE_TOKEN_HIT;
          bool lead = (__ffs(__shfl_sync(kFull, grp, j)) - 1) == (int)j;
          if (lead) {
            if (!warp_request(d, l == 0, pj, a.q0, true, a.deadline, &tj)) return;
            tj = __shfl_sync(kFull, tj, 0);
            if (l == j) t = tj;
          }
        }
        uint32_t line;
        if (!warp_pin_page(d, pj, a.q0, a.deadline, line)) return;
        warp_copy_page(dst + (base + j) * kPage, line_ptr(d, line));
        __syncwarp();
        if (l == 0) cache_unpin(d, line);
      }
      if (tok && want) {
        uint64_t lt = __shfl_sync(kFull, t, __ffs(grp) - 1);
        tok[i] = lt;
      } else {
        (void)__shfl_sync(kFull, t, __ffs(grp) - 1);
      }
    }
  }
};

// asyncWrite (Sec. 3.5): the cache line is updated and a write command is issued from
// a staging copy; the page's share-table entry blocks any re-read of the store until
// the write has completed.  One page per warp at a time.
struct WriteApp {
  const uint64_t *pages;
  uint32_t n;
  const uint8_t *src;
  uint64_t *tok;
  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    for (uint64_t i = a.warp; i < n; i += a.n_warps) {
      uint64_t page = pages[i];
      if (!page_ok(d, page)) {
        if (l == 0) set_error(d, AGILE_EINVAL);
        continue;
      }
      // 1. own the page (share table), holding nothing while retrying
      int64_t sh = -1;
      uint32_t ns = 64;
      for (;;) {
        if (l == 0) sh = sh_insert(d, page, SH_WRITE);
        sh = __shfl_sync(kFull, sh, 0);
        if (sh >= 0) break;
        if (gtimer() > a.deadline || aborted(d)) {
          if (l == 0) set_error(d, -110);
          return;
        }
        backoff(ns);
      }
      // 2. find or claim the line
      uint32_t line = 0;
      int how = -1;  // 0 pinned hit, 1 claimed
      Issued is{};
      is.q = 0xFFFFFFFFu;
      for (;;) {
        if (l == 0) {
          int pr = cache_probe(d, page, true, line);
          if (pr == P_HIT) {
            how = 0;
          } else if (pr == P_MISS) {
            int m = cache_miss(d, page, a.q0, line, is, false, sh);
            how = (m == M_ISSUED) ? 1 : -1;
          } else {
            how = -1;
          }
        }
        how = __shfl_sync(kFull, how, 0);
        if (how >= 0) break;
        if (gtimer() > a.deadline || aborted(d)) {
          if (l == 0) {
            set_error(d, -110);
            sh_remove(d, (uint64_t)sh);
          }
          return;
        }
        backoff(ns);
      }
      line = __shfl_sync(kFull, line, 0);
      if (!warp_ring(d, l == 0 && is.q != 0xFFFFFFFFu, is.q, is.slot, is.ticket, a.deadline)) return;
      // 3. new contents into the line; publish it READY (a full page supersedes it)
      warp_copy_page(line_ptr(d, line), src + i * kPage);
      __threadfence();
      __syncwarp();
      // The line stays pinned until the write is decided, so that it still holds this
      // page when it is marked MODIFIED below.  A MODIFIED line's pending write is
      // superseded by this page's write; otherwise the page now owes the store a write.
      if (l == 0) {
        bool was_dirty = false;
        if (how == 0) {
          uint64_t old = atomicAnd(&d.tag[line], ~1ull);  // MODIFIED (3) or READY (2) -> READY
          was_dirty = tag_state(old) == ST_MODIFIED;
        } else {
          atomicAdd(&d.tag[line], 1ull + PIN1);  // BUSY -> READY, pinned
        }
        if (!was_dirty) note_dirty(d, page);
      }
      // 4. write command from a staging copy.  A reservation can fail under contention
      // as well as on full queues, so it is retried for a while (slots are freed by
      // completions, which never need a cache line) before the write is left to a
      // later write-back of the MODIFIED line.
      uint32_t q = 0, slot = 0, ticket = 0;
      int ok = 0;
      uint32_t ns2 = 64;
      for (int tries = 0; tries < 48; ++tries) {
        if (l == 0) ok = sq_reserve_dev(d, a.q0, dev_of_page(d, page), 1, q, slot, ticket);
        ok = __shfl_sync(kFull, ok, 0);
        if (ok || aborted(d)) break;
        backoff(ns2, 2048);
      }
      uint64_t t = AGILE_TOKEN_HIT;
      if (ok) {
        q = __shfl_sync(kFull, q, 0);
        slot = __shfl_sync(kFull, slot, 0);
        ticket = __shfl_sync(kFull, ticket, 0);
        uint8_t *stg = d.staging + ((uint64_t)q * d.depth + slot) * kPage;
        warp_copy_page(stg, src + i * kPage);
        __threadfence();
        __syncwarp();
        if (l == 0) {
          sq_commit(d, q, slot, ticket, OP_WRITE, (uint64_t)stg, page, ctx_make(CTX_WB, (uint32_t)sh, 0));
          atomicAdd(stat_ptr(d, S_WRITEBACKS), 1ull);
          cache_unpin(d, line);
        }
        if (!warp_ring(d, l == 0, q, slot, ticket, a.deadline)) return;
        t = make_token(q, slot, ticket);
      } else if (l == 0) {
        // no queue slot: keep the data as a MODIFIED line, written back later
        atomicOr(&d.tag[line], 1ull);
        cache_unpin(d, line);
        sh_remove(d, (uint64_t)sh);
      }
      if (tok && l == 0) tok[i] = t;
    }
  }
};

// Write back every MODIFIED line (Sec. 3.4 case (d) write-back, as a bulk operation).
// Lines are partitioned among app warps; a warp repeats its pass until its lines are
// clean.  Each write-back owns the page's share-table entry until completion.
struct FlushApp {
  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    uint32_t ns = 64;
    for (int pass = 0;; ++pass) {
      bool dirty_left = false;
      for (uint64_t base = (uint64_t)a.warp * 32; base < d.nlines; base += (uint64_t)a.n_warps * 32) {
        uint64_t line = base + l;
        bool mine = false;
        int64_t sh = -1;
        uint32_t q = 0, slot = 0, ticket = 0;
        uint64_t t = 0;
        if (line < d.nlines) {
          t = ld_rlx64(&d.tag[line]);
          if (tag_state(t) == ST_MODIFIED) {
            dirty_left = true;
            if ((t & (PIN_MASK | TAG_WB)) == 0) {
              sh = sh_insert(d, tag_page(t), SH_WRITE);
              if (sh >= 0) {
                // MODIFIED -> READY with the write-back bit: the line stays valid for
                // readers and cannot be evicted until the write completes
                uint64_t clean = (t & ~1ull) | TAG_WB;
                if (atomicCAS(&d.tag[line], (unsigned long long)t, (unsigned long long)clean) == t) {
                  if (sq_reserve_dev(d, a.q0, dev_of_page(d, tag_page(t)), 1, q, slot, ticket)) {
                    mine = true;
                  } else {
                    atomicOr(&d.tag[line], 1ull);
                    atomicAnd(&d.tag[line], ~TAG_WB);
                    sh_remove(d, (uint64_t)sh);
                  }
                } else {
                  sh_remove(d, (uint64_t)sh);
                }
              }
            }
          }
        }
        unsigned who = __ballot_sync(kFull, mine);
        while (who) {
          int j = __ffs(who) - 1;
          who &= who - 1;
          uint64_t lj = __shfl_sync(kFull, line, j);
          uint32_t qj = __shfl_sync(kFull, q, j), sj = __shfl_sync(kFull, slot, j);
          warp_copy_page(d.staging + ((uint64_t)qj * d.depth + sj) * kPage, line_ptr(d, lj));
        }
        __threadfence();
        __syncwarp();
        if (mine) {
          uint8_t *stg = d.staging + ((uint64_t)q * d.depth + slot) * kPage;
          sq_commit(d, q, slot, ticket, OP_WRITE, (uint64_t)stg, tag_page(t),
                    ctx_make(CTX_WB, (uint32_t)sh, (uint32_t)(line + 1)));
          atomicAdd(stat_ptr(d, S_WRITEBACKS), 1ull);
        }
        if (!warp_ring(d, mine, q, slot, ticket, a.deadline)) return;
      }
      if (!__any_sync(kFull, dirty_left)) return;
      if (gtimer() > a.deadline || aborted(d)) {
        if (l == 0) set_error(d, -110);
        return;
      }
      backoff(ns);
    }
  }
};

// Validation: one thread serves the requests strictly one after the other (sync).
struct ReplayApp {
  const uint64_t *pages;
  uint32_t n;
  int32_t *codes;
  __device__ void run(const Dev &d, const AppCtx &a) const {
    if (a.warp != 0) return;
    unsigned l = lane_id();
    for (uint32_t i = 0; i < n; ++i) {
      uint64_t page = pages[i];
      int code = 0;
      if (!page_ok(d, page)) {
        if (l == 0) set_error(d, AGILE_EINVAL);
        return;
      }
      uint32_t ns = 64;
      for (;;) {
        int done = 0, issued = 0, ring = 0;
        uint32_t line = 0;
        Issued is{};
        if (l == 0) {
          int pr = cache_probe(d, page, false, line);
          if (pr == P_HIT) {
            done = 1;
            atomicAdd(stat_ptr(d, S_HITS), 1ull);
          } else if (pr == P_MISS) {
            int m = cache_miss(d, page, a.q0, line, is);
            ring = m == M_ISSUED;
            if (m == M_ISSUED) {
              issued = 1;
              code = is.code;
            }
          }
        }
        done = __shfl_sync(kFull, done, 0);
        if (done) break;
        issued = __shfl_sync(kFull, issued, 0);
        if (!warp_ring(d, l == 0 && ring, is.q, is.slot, is.ticket, a.deadline)) return;
        if (issued) {
          // wait for the fill with nothing held
          line = __shfl_sync(kFull, line, 0);
          for (;;) {
            uint64_t t = ld_acq64(&d.tag[line]);
            if (!(tag_page(t) == page && tag_state(t) == ST_BUSY)) break;
            if (gtimer() > a.deadline) {
              if (l == 0) set_error(d, -110);
              return;
            }
            __nanosleep(64);
          }
          break;
        }
        if (gtimer() > a.deadline) {
          if (l == 0) set_error(d, -110);
          return;
        }
        backoff(ns);
      }
      if (l == 0) codes[i] = code;
    }
  }
};

// wait (Sec. 3.2.1): tokens are final once the issuing call has drained, so this only
// reads the completion words.
__global__ void wait_kernel(Dev d, const uint64_t *tok, uint32_t n, int32_t *status) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint64_t t = tok[i];
  if (t == AGILE_TOKEN_HIT) {
    status[i] = 0;
    return;
  }
  uint32_t q = (uint32_t)(t >> 48), slot = (uint32_t)(t >> 32) & 0xFFFFu, ticket = (uint32_t)t;
  if (q >= d.Q || slot >= d.depth) {
    status[i] = AGILE_EINVAL;
    return;
  }
  uint64_t w = ld_acq64(&d.cmpl[(uint64_t)q * d.depth + slot]);
  uint32_t wt = (uint32_t)(w >> 32);
  if (!(w & 1) || (int32_t)(wt - ticket) < 0) {
    status[i] = AGILE_ETIMEDOUT;
  } else if (wt == ticket && ((w >> 1) & 0x7FFF) != 0) {
    status[i] = AGILE_EIO;
  } else {
    status[i] = 0;
  }
}

// Streams n16 16-byte words from pinned host memory (mapped) into HBM: each thread keeps
// four loads in flight, the grid strides over the buffer.
__global__ void link_probe_kernel(const uint8_t *src, uint8_t *dst, uint64_t n16) {
  const int4 *s = (const int4 *)src;
  int4 *t = (int4 *)dst;
  uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    int4 v0 = ld_cg16(s + i), v1 = ld_cg16(s + i + stride), v2 = ld_cg16(s + i + 2 * stride),
         v3 = ld_cg16(s + i + 3 * stride);
    st_cg16(t + i, v0);
    st_cg16(t + i + stride, v1);
    st_cg16(t + i + 2 * stride, v2);
    st_cg16(t + i + 3 * stride, v3);
  }
  for (; i < n16; i += stride) st_cg16(t + i, ld_cg16(s + i));
}

__global__ void invalidate_range_kernel(Dev d, uint64_t p0, uint64_t p1) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= d.nlines) return;
  uint64_t t = d.tag[i];
  if (tag_state(t) != ST_INVALID && tag_page(t) >= p0 && tag_page(t) <= p1) d.tag[i] = 0;
}

}  // namespace

// ============================================================================ host API

// Queues that carry prefetches: `req` (0 = half, rounded down to a multiple of the
// devices; AGILE_NO_PREFETCH_QUEUES = none); -1 when `req` cannot be used.
static int64_t prefetch_queue_count(uint32_t req, uint32_t Q, uint32_t ndev) {
  if (req == AGILE_NO_PREFETCH_QUEUES) return 0;
  if (req == 0) {
    uint32_t per = Q / ndev;  // queues per device
    return per >= 2 ? (int64_t)(per / 2) * ndev : 0;
  }
  if (req % ndev || req >= Q) return -1;
  return req;
}

static void *dalloc(agile_ctx *c, size_t bytes) {
  void *p = nullptr;
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
  if (cudaMemset(p, 0, bytes) != cudaSuccess) {
    cudaFree(p);
    return nullptr;
  }
  c->dallocs.push_back(p);
  return p;
}

extern "C" {

void agile_config_default(agile_config *cfg) {
  if (!cfg) return;
  memset(cfg, 0, sizeof(*cfg));
  cfg->store_bytes = 64ull << 20;
  cfg->cache_bytes = 4ull << 20;
  cfg->ways = 8;
  cfg->num_queues = 128;
  cfg->queue_depth = 256;
  cfg->wait_timeout_ns = 10ull * 1000 * 1000 * 1000;
  cfg->prefetch_depth = 1;
}

const char *agile_strerror(int code) {
  switch (code) {
    case AGILE_OK: return "ok";
    case AGILE_EIO: return "I/O error reported by a completion";
    case AGILE_EAGAIN: return "no cache line or queue slot available";
    case AGILE_ENOMEM: return "out of memory";
    case AGILE_ENODEV: return "no such device";
    case AGILE_EINVAL: return "invalid argument";
    case AGILE_ETIMEDOUT: return "bounded wait timed out on the GPU";
    case AGILE_ECUDA: return "CUDA runtime error";
    default: return "unknown error";
  }
}

int agile_init(const agile_config *cfg_in, agile_ctx **out) {
  if (!cfg_in || !out) return AGILE_EINVAL;
  *out = nullptr;
  agile_config cfg = *cfg_in;
  if (cfg.nvme_path) return AGILE_ENODEV;
  if (cfg.store_bytes == 0 || cfg.store_bytes % kPage) return AGILE_EINVAL;
  if (cfg.ways == 0 || cfg.ways > 32) return AGILE_EINVAL;
  if (cfg.num_queues == 0 || cfg.num_queues > 65535) return AGILE_EINVAL;
  uint32_t dep = cfg.queue_depth;
  if (dep < 64 || dep > 65536 || (dep & (dep - 1))) return AGILE_EINVAL;
  uint64_t sets = cfg.cache_bytes / ((uint64_t)cfg.ways * kPage);
  if (sets == 0 || sets > 0xFFFFFFFFull) return AGILE_EINVAL;
  if (cfg.fault_rate < 0 || cfg.fault_rate > 1 || cfg.emu_queue_gbps < 0) return AGILE_EINVAL;
  if (cfg.emu_device_read_gbps < 0 || cfg.emu_device_write_gbps < 0) return AGILE_EINVAL;
  if (cfg.num_devices == 0) cfg.num_devices = 1;
  if (cfg.num_devices > cfg.num_queues || cfg.num_queues % cfg.num_devices) return AGILE_EINVAL;
  if (cfg.cache_policy > AGILE_POLICY_FIFO) return AGILE_EINVAL;
  if (prefetch_queue_count(cfg.prefetch_queues, cfg.num_queues, cfg.num_devices) < 0) return AGILE_EINVAL;
  if (cfg.wait_timeout_ns == 0) cfg.wait_timeout_ns = 10ull * 1000 * 1000 * 1000;
  if (cfg.prefetch_depth == 0) cfg.prefetch_depth = 1;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return AGILE_ENODEV;
  if (cfg.device < 0 || cfg.device >= ndev) return AGILE_ENODEV;
  if (cudaSetDevice(cfg.device) != cudaSuccess) return AGILE_ECUDA;
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, cfg.device);
  if (!coop) return AGILE_ENODEV;

  agile_ctx *c = new agile_ctx();
  c->cfg = cfg;
  c->device = cfg.device;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, cfg.device);
  Dev &d = c->dev;

  if (cudaHostAlloc(&c->store_host, cfg.store_bytes, cudaHostAllocMapped | cudaHostAllocPortable) != cudaSuccess) {
    delete c;
    return AGILE_ENOMEM;
  }
  memset(c->store_host, 0, cfg.store_bytes);
  void *sdev = nullptr;
  if (cudaHostGetDevicePointer(&sdev, c->store_host, 0) != cudaSuccess) {
    cudaFreeHost(c->store_host);
    delete c;
    return AGILE_ECUDA;
  }
  d.store = (uint8_t *)sdev;
  d.store_bytes = cfg.store_bytes;

  d.sets = (uint32_t)sets;
  d.ways = cfg.ways;
  d.nlines = sets * cfg.ways;
  uint64_t Q = cfg.num_queues, D = dep;
  uint32_t buckets = 1024;
  while ((uint64_t)buckets < Q * D) buckets <<= 1;
  d.sh_mask = buckets - 1;
  d.Q = (uint32_t)Q;
  d.Qp = (uint32_t)prefetch_queue_count(cfg.prefetch_queues, cfg.num_queues, cfg.num_devices);
  d.depth = dep;
  d.dmask = dep - 1;
  d.dlog = 0;
  while ((1u << d.dlog) < dep) d.dlog++;

  bool ok = true;
  auto A = [&](size_t bytes) {
    void *p = dalloc(c, bytes);
    if (!p) ok = false;
    return p;
  };
  d.lines = (uint8_t *)A(d.nlines * kPage);
  d.tag = (unsigned long long *)A(d.nlines * 8);
  d.hand = (uint32_t *)A(sets * 4);
  d.sh_key = (unsigned long long *)A((uint64_t)buckets * 4 * 8);
  d.sh_val = (unsigned long long *)A((uint64_t)buckets * 4 * 8);
  d.sq = (Sqe *)A(Q * D * sizeof(Sqe));
  d.cq_size = 2 * dep;
  d.cq = (Cqe *)A(Q * 2 * D * sizeof(Cqe));
  d.sqe_state = (unsigned long long *)A(Q * D * 8);
  d.cmd_ctx = (unsigned long long *)A(Q * D * 8);
  d.cmpl = (unsigned long long *)A(Q * D * 8);
  d.sq_resv = (unsigned long long *)A(Q * 8);
  d.sq_tail = (uint32_t *)A(Q * 4);
  d.sq_lock = (uint32_t *)A(Q * 4);
  d.sq_db = (uint32_t *)A(Q * 4);
  d.cq_db = (uint32_t *)A(Q * 4);
  d.cq_poll = (uint32_t *)A(Q * 16);
  d.emu = (uint32_t *)A(Q * 16);
  d.emu_busy = (unsigned long long *)A(Q * 8);
  d.emu_arrival = (unsigned long long *)A(Q * D * 8);
  d.staging = (uint8_t *)A(Q * D * kPage);
  uint64_t store_pages = cfg.store_bytes / kPage;
  d.pg_reads = (uint32_t *)A(store_pages * 4);
  d.pg_writes = (uint32_t *)A(store_pages * 4);
  d.pg_dirty = (uint32_t *)A(store_pages * 4);
  d.trace_cap = cfg.trace_records;
  d.trace = cfg.trace_records ? (TraceRec *)A((uint64_t)cfg.trace_records * sizeof(TraceRec)) : nullptr;
  d.trace_n = (uint32_t *)A(16);
  d.ev = cfg.trace_records ? (unsigned long long *)A((uint64_t)cfg.trace_records * 16) : nullptr;
  d.ev_n = (uint32_t *)A(16);
  d.ndev = cfg.num_devices;
  d.policy = cfg.cache_policy;
  d.dev_busy = (unsigned long long *)A((uint64_t)cfg.num_devices * 8);
  if (cfg.share_slots) {
    uint32_t ub = 256;  // buckets of 4 slots, at most half full
    while ((uint64_t)ub * 2 < cfg.share_slots && ub < (1u << 30)) ub <<= 1;
    d.ub_mask = ub - 1;
    d.ub_key = (unsigned long long *)A((uint64_t)ub * 4 * 8);
    d.ub_buf = (unsigned long long *)A((uint64_t)ub * 4 * 8);
    d.ub_meta = (unsigned long long *)A((uint64_t)ub * 4 * 8);
    d.ub_tok = (unsigned long long *)A((uint64_t)ub * 4 * 8);
  }
  d.run = (RunState *)A(sizeof(RunState));
  d.stats = (unsigned long long *)A((size_t)kStatShards * S_COUNT * 8);
  d.err_sticky = (int32_t *)A(16);
  if (!ok) {
    agile_destroy(c);
    return AGILE_ENOMEM;
  }
  // Alg. 1 expects phase 1 on the first pass; the emulated device posts phase 1 first
  {
    std::vector<uint32_t> init(Q * 4, 0);
    for (uint64_t q = 0; q < Q; ++q) init[q * 4 + 2] = 1;
    if (cudaMemcpy(d.cq_poll, init.data(), Q * 16, cudaMemcpyHostToDevice) != cudaSuccess) {
      agile_destroy(c);
      return AGILE_ECUDA;
    }
  }
  d.lat_ns = cfg.emu_latency_ns;
  d.ns_per_page = cfg.emu_queue_gbps > 0 ? (uint64_t)llround(kPage / cfg.emu_queue_gbps) : 0;
  d.ns_rd_dev = cfg.emu_device_read_gbps > 0 ? (uint64_t)llround(kPage / cfg.emu_device_read_gbps) : 0;
  d.ns_wr_dev = cfg.emu_device_write_gbps > 0 ? (uint64_t)llround(kPage / cfg.emu_device_write_gbps) : 0;
  d.fault_flags = cfg.fault_flags;
  d.fault_thresh = (uint32_t)fmin(4294967295.0, cfg.fault_rate * 4294967296.0);
  d.seed = cfg.seed;
  d.timeout_ns = cfg.wait_timeout_ns;
  d.extra_engines = cfg.emu_extra_engines == AGILE_NO_EXTRA_ENGINES
                        ? 0u
                        : (cfg.emu_extra_engines ? cfg.emu_extra_engines : 0xFFFFFFFFu);
  d.prefetch_depth = cfg.prefetch_depth;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    agile_destroy(c);
    return AGILE_ECUDA;
  }
  *out = c;
  return AGILE_OK;
}

int agile_flush(agile_ctx *c, void *stream) {
  if (!c) return AGILE_EINVAL;
  return launch_engine(c, FlushApp{}, stream);
}

int agile_destroy(agile_ctx *c) {
  if (!c) return AGILE_OK;
  cudaSetDevice(c->device);
  if (c->dev.tag && c->dev.run) {
    agile_flush(c, nullptr);
    cudaDeviceSynchronize();
  }
  for (void *p : c->dallocs) cudaFree(p);
  if (c->bfs_hubq) cudaFree(c->bfs_hubq);
  if (c->bfs_vis) cudaFree(c->bfs_vis);
  if (c->train_scratch) cudaFree(c->train_scratch);
  if (c->emb_scratch) cudaFree(c->emb_scratch);
  if (c->store_host) cudaFreeHost(c->store_host);
  delete c;
  return AGILE_OK;
}

int agile_invalidate(agile_ctx *c, void *stream) {
  if (!c) return AGILE_EINVAL;
  int r = agile_flush(c, stream);
  if (r) return r;
  cudaStream_t s = as_stream(stream);
  AGILE_CUDA_TRY(cudaMemsetAsync(c->dev.tag, 0, c->dev.nlines * 8, s));
  AGILE_CUDA_TRY(cudaMemsetAsync(c->dev.hand, 0, (size_t)c->dev.sets * 4, s));
  return AGILE_OK;
}

int agile_store_write(agile_ctx *c, uint64_t off, const void *src, uint64_t n) {
  if (!c || (!src && n)) return AGILE_EINVAL;
  if (off > c->cfg.store_bytes || n > c->cfg.store_bytes - off) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  // bring the store up to date, then drop cached copies of the pages being replaced
  int r = agile_flush(c, nullptr);
  if (r) return r;
  uint64_t p0 = off / kPage, p1 = (off + n - 1) / kPage;
  invalidate_range_kernel<<<(unsigned)((c->dev.nlines + 255) / 256), 256>>>(c->dev, p0, p1);
  AGILE_CUDA_TRY(cudaGetLastError());
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  memcpy((uint8_t *)c->store_host + off, src, n);
  return AGILE_OK;
}

int agile_store_read(agile_ctx *c, uint64_t off, void *dst, uint64_t n) {
  if (!c || (!dst && n)) return AGILE_EINVAL;
  if (off > c->cfg.store_bytes || n > c->cfg.store_bytes - off) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  memcpy(dst, (const uint8_t *)c->store_host + off, n);
  return AGILE_OK;
}

int agile_read_async(agile_ctx *c, const uint64_t *d_pages, uint32_t n, void *d_dst, agile_token *d_tok,
                     uint32_t mode, void *stream) {
  if (!c || (n && (!d_pages || !d_dst)) || mode > 1) return AGILE_EINVAL;
  if (((uintptr_t)d_dst) & 15) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  ReadApp app{d_pages, n, (uint8_t *)d_dst, d_tok, mode, 0};
  return launch_engine(c, app, stream, warps_for_cache(c, mode == AGILE_ASYNC ? 48 : 4, 8));
}

int agile_prefetch(agile_ctx *c, const uint64_t *d_pages, uint32_t n, void *stream) {
  if (!c || (n && !d_pages)) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  ReadApp app{d_pages, n, nullptr, nullptr, AGILE_ASYNC, 1};
  return launch_engine(c, app, stream, warps_for_cache(c, 48, 8));
}

int agile_write_async(agile_ctx *c, const uint64_t *d_pages, uint32_t n, const void *d_src, agile_token *d_tok,
                      void *stream) {
  if (!c || (n && (!d_pages || !d_src))) return AGILE_EINVAL;
  if (((uintptr_t)d_src) & 15) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  WriteApp app{d_pages, n, (const uint8_t *)d_src, d_tok};
  return launch_engine(c, app, stream, warps_for_cache(c, 4, 8));
}

int agile_wait(agile_ctx *c, const agile_token *d_tok, uint32_t n, int32_t *d_status, void *stream) {
  if (!c || (n && (!d_tok || !d_status))) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  wait_kernel<<<(n + 255) / 256, 256, 0, as_stream(stream)>>>(c->dev, d_tok, n, d_status);
  AGILE_CUDA_TRY(cudaGetLastError());
  return AGILE_OK;
}

int agile_cache_replay(agile_ctx *c, const uint64_t *d_pages, uint32_t n, int32_t *d_codes, void *stream) {
  if (!c || (n && (!d_pages || !d_codes))) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  ReplayApp app{d_pages, n, d_codes};
  return launch_engine(c, app, stream);
}

int agile_cache_tags(agile_ctx *c, uint64_t *out) {
  if (!c || !out) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  AGILE_CUDA_TRY(cudaMemcpy(out, c->dev.tag, c->dev.nlines * 8, cudaMemcpyDeviceToHost));
  return AGILE_OK;
}

uint64_t agile_cache_lines(agile_ctx *c) { return c ? c->dev.nlines : 0; }
uint32_t agile_cache_sets(agile_ctx *c) { return c ? c->dev.sets : 0; }

int agile_stats(agile_ctx *c, agile_stats_t *out) {
  if (!c || !out) return AGILE_EINVAL;
  static_assert(sizeof(agile_stats_t) == S_COUNT * 8, "stats layout");
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  std::vector<unsigned long long> sh((size_t)kStatShards * S_COUNT);
  AGILE_CUDA_TRY(cudaMemcpy(sh.data(), c->dev.stats, sh.size() * 8, cudaMemcpyDeviceToHost));
  uint64_t *o = (uint64_t *)out;
  for (int s = 0; s < S_COUNT; ++s) {
    uint64_t v = 0;
    for (int k = 0; k < kStatShards; ++k) v += sh[(size_t)k * S_COUNT + s];
    o[s] = v;
  }
  return AGILE_OK;
}

int agile_reset_stats(agile_ctx *c) {
  if (!c) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  AGILE_CUDA_TRY(cudaMemset(c->dev.stats, 0, (size_t)kStatShards * S_COUNT * 8));
  uint64_t pages = c->cfg.store_bytes / kPage;
  AGILE_CUDA_TRY(cudaMemset(c->dev.pg_reads, 0, pages * 4));
  AGILE_CUDA_TRY(cudaMemset(c->dev.pg_writes, 0, pages * 4));
  AGILE_CUDA_TRY(cudaMemset(c->dev.pg_dirty, 0, pages * 4));
  AGILE_CUDA_TRY(cudaMemset(c->dev.trace_n, 0, 4));
  AGILE_CUDA_TRY(cudaMemset(c->dev.ev_n, 0, 4));
  return AGILE_OK;
}

int agile_events(agile_ctx *c, uint64_t *out, uint32_t cap, uint32_t *n_out) {
  if (!c || (cap && !out)) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t n = 0;
  AGILE_CUDA_TRY(cudaMemcpy(&n, c->dev.ev_n, 4, cudaMemcpyDeviceToHost));
  if (n_out) *n_out = n;
  uint32_t k = std::min(std::min(n, c->dev.trace_cap), cap);
  if (k && c->dev.ev) AGILE_CUDA_TRY(cudaMemcpy(out, c->dev.ev, (size_t)k * 16, cudaMemcpyDeviceToHost));
  return AGILE_OK;
}

int agile_set_device_model(agile_ctx *c, uint32_t ndev, uint32_t lat_ns, double queue_gbps, double rd_gbps,
                           double wr_gbps) {
  if (!c) return AGILE_EINVAL;
  if (ndev == 0) ndev = 1;
  if (ndev > c->cfg.num_queues || c->cfg.num_queues % ndev) return AGILE_EINVAL;
  if (queue_gbps < 0 || rd_gbps < 0 || wr_gbps < 0) return AGILE_EINVAL;
  int64_t qp = prefetch_queue_count(c->cfg.prefetch_queues, c->cfg.num_queues, ndev);
  if (qp < 0) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  if (ndev > c->cfg.num_devices) {
    // the per-device booking words: one per device
    unsigned long long *nb = nullptr;
    AGILE_CUDA_TRY(cudaMalloc(&nb, (size_t)ndev * 8));
    c->dallocs.push_back(nb);
    c->dev.dev_busy = nb;
  }
  AGILE_CUDA_TRY(cudaMemset(c->dev.dev_busy, 0, (size_t)ndev * 8));
  AGILE_CUDA_TRY(cudaMemset(c->dev.emu_busy, 0, (size_t)c->dev.Q * 8));
  // The device without a model advances only its fetch counters; with a model it also
  // counts the commands it has seen (arrival stamps).  Between calls every command has
  // been served, so each queue's "seen" counter is set to its fetch counter.
  {
    std::vector<uint32_t> emu((size_t)c->dev.Q * 4);
    AGILE_CUDA_TRY(cudaMemcpy(emu.data(), c->dev.emu, emu.size() * 4, cudaMemcpyDeviceToHost));
    for (uint64_t q = 0; q < c->dev.Q; ++q) emu[q * 4 + 1] = emu[q * 4];
    AGILE_CUDA_TRY(cudaMemcpy(c->dev.emu, emu.data(), emu.size() * 4, cudaMemcpyHostToDevice));
  }
  c->cfg.num_devices = std::max(c->cfg.num_devices, ndev);
  c->dev.ndev = ndev;
  c->dev.Qp = (uint32_t)qp;
  c->dev.lat_ns = lat_ns;
  c->dev.ns_per_page = queue_gbps > 0 ? (uint64_t)llround(kPage / queue_gbps) : 0;
  c->dev.ns_rd_dev = rd_gbps > 0 ? (uint64_t)llround(kPage / rd_gbps) : 0;
  c->dev.ns_wr_dev = wr_gbps > 0 ? (uint64_t)llround(kPage / wr_gbps) : 0;
  c->cfg.emu_latency_ns = lat_ns;
  c->cfg.emu_queue_gbps = queue_gbps;
  c->cfg.emu_device_read_gbps = rd_gbps;
  c->cfg.emu_device_write_gbps = wr_gbps;
  return AGILE_OK;
}

int agile_device_view(agile_ctx *c, void *out, uint64_t size) {
  if (!c || !out || size != sizeof(Dev)) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  Dev d = c->dev;
  d.app_active = c->cfg.app_warps;
  memcpy(out, &d, sizeof(Dev));
  return AGILE_OK;
}

int agile_run_reset(agile_ctx *c, void *stream) {
  if (!c) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  run_reset_kernel<<<1, 128, 0, as_stream(stream)>>>(c->dev.run);
  AGILE_CUDA_TRY(cudaGetLastError());
  return AGILE_OK;
}

int agile_page_io(agile_ctx *c, uint64_t page0, uint64_t n, uint32_t *reads, uint32_t *writes, uint32_t *dirtied) {
  if (!c) return AGILE_EINVAL;
  uint64_t pages = c->cfg.store_bytes / kPage;
  if (page0 > pages || n > pages - page0) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  if (n == 0) return AGILE_OK;
  if (reads) AGILE_CUDA_TRY(cudaMemcpy(reads, c->dev.pg_reads + page0, n * 4, cudaMemcpyDeviceToHost));
  if (writes) AGILE_CUDA_TRY(cudaMemcpy(writes, c->dev.pg_writes + page0, n * 4, cudaMemcpyDeviceToHost));
  if (dirtied) AGILE_CUDA_TRY(cudaMemcpy(dirtied, c->dev.pg_dirty + page0, n * 4, cudaMemcpyDeviceToHost));
  return AGILE_OK;
}

int agile_trace(agile_ctx *c, agile_trace_rec *out, uint32_t cap, uint32_t *n_out) {
  static_assert(sizeof(agile_trace_rec) == sizeof(TraceRec), "trace record layout");
  if (!c || (cap && !out)) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  uint32_t n = 0;
  AGILE_CUDA_TRY(cudaMemcpy(&n, c->dev.trace_n, 4, cudaMemcpyDeviceToHost));
  if (n_out) *n_out = n;
  uint32_t k = std::min(std::min(n, c->dev.trace_cap), cap);
  if (k) AGILE_CUDA_TRY(cudaMemcpy(out, c->dev.trace, (size_t)k * sizeof(TraceRec), cudaMemcpyDeviceToHost));
  return AGILE_OK;
}

int agile_link_probe(agile_ctx *c, void *d_dst, uint64_t bytes, uint32_t ctas, uint32_t reps, double *gbps) {
  if (!c || !d_dst || !gbps || bytes == 0 || bytes % kPage || bytes > c->cfg.store_bytes) return AGILE_EINVAL;
  if (((uintptr_t)d_dst) & 15) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  if (ctas == 0) ctas = 2u * (uint32_t)c->sms;
  if (reps == 0) reps = 1;
  cudaEvent_t a, b;
  AGILE_CUDA_TRY(cudaEventCreate(&a));
  AGILE_CUDA_TRY(cudaEventCreate(&b));
  double best = 0;
  for (uint32_t r = 0; r < reps; ++r) {
    cudaEventRecord(a, 0);
    link_probe_kernel<<<ctas, 512>>>(c->dev.store, (uint8_t *)d_dst, bytes / 16);
    cudaEventRecord(b, 0);
    cudaError_t e = cudaEventSynchronize(b);
    float ms = 0;
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (e != cudaSuccess) {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      fprintf(stderr, "agile_link_probe: %s\n", cudaGetErrorString(e));
      return AGILE_ECUDA;
    }
    if (ms > 0) best = std::max(best, bytes / (ms * 1e-3) / 1e9);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *gbps = best;
  return AGILE_OK;
}

int agile_check(agile_ctx *c) {
  if (!c) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  AGILE_CUDA_TRY(cudaDeviceSynchronize());
  int32_t e = 0;
  AGILE_CUDA_TRY(cudaMemcpy(&e, c->dev.err_sticky, 4, cudaMemcpyDeviceToHost));
  AGILE_CUDA_TRY(cudaMemset(c->dev.err_sticky, 0, 4));
  return e ? -e : AGILE_OK;
}

int agile_config_parallelism(agile_ctx *c, uint32_t app_warps) {
  if (!c) return AGILE_EINVAL;
  c->cfg.app_warps = app_warps;
  return AGILE_OK;
}

int agile_launch_shape(agile_ctx *c, uint32_t *ctas, uint32_t *threads) {
  if (!c) return AGILE_EINVAL;
  if (ctas) *ctas = (uint32_t)engine_grid<ReadApp>(c);
  if (threads) *threads = kThreads;
  return AGILE_OK;
}

}  // extern "C"
