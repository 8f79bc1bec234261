// Serving loop: continuous batching of embedding-bag lookup requests (the serving
// extension of the Sec. 4.4 lookups).  One long-running engine launch keeps the queues,
// the device and the cache state resident while requests of any size arrive:
//   - the host writes request descriptors into a ring in mapped pinned memory and
//     publishes each one by its sequence number (release); it never launches work;
//   - application warp 0 is the scheduler: it reads the ring (system-scope acquire) and
//     admits a request, oldest first, once the free cache-line budget (half of the
//     cache's lines) covers the lines it may hold (its indices + 1, at most the budget),
//     or when nothing else is running.  Queue slots need no budget of their own: a
//     request takes at most one slot per missing page, every slot comes back with its
//     completion, and a full queue only sends the issuing warp to the next queue;
//   - every other application warp takes bags from the oldest admitted request that
//     still has unclaimed bags (a shared cursor moves past fully claimed requests), so
//     requests that arrive while others run are served alongside them;
//   - the warp that finishes the last bag of a request writes the request's completion
//     word into host memory (system-scope release) and returns its budget.
// A bag is computed exactly as by agile_embedding_bag (same rows, same order, same
// rounding), so a request's result is the same alone and in any mix.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <thread>
#include <vector>

#include "agile.h"
#include "agile_ctx.cuh"
#include "agile_dev.cuh"

using namespace agile;

struct ServeSlot {  // one ring entry, host-written
  uint64_t table_byte0;
  uint64_t idx, offsets, out;  // device pointers
  uint32_t rows, dim, n_bags, pad;
  unsigned long long seq;  // written last: sequence number + 1 once the entry is valid
};

namespace {

__device__ __forceinline__ uint64_t ld_acq_sys64(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_vol_sys64(const void *p) {
  uint64_t v;
  asm volatile("ld.volatile.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_vol_sys32(const void *p) {
  uint32_t v;
  asm volatile("ld.volatile.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel_sys64(unsigned long long *p, uint64_t v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// device-side state of the session (device memory, zeroed at start)
struct ServeDev {
  unsigned long long admitted;   // requests admitted so far (sequence numbers < admitted)
  unsigned long long cursor;     // first admitted request that may still have bags to hand out
  unsigned long long finished;   // requests finished
  unsigned long long used;       // budget in use (lines)
  uint32_t stop_seen;
  uint32_t pad;
};

struct ReqState {  // per ring entry (device memory)
  unsigned long long seq;  // request this entry currently holds + 1
  uint32_t next_bag;       // next bag to hand out
  uint32_t bags_done;
  uint32_t n_bags;
  uint32_t need;           // budget held
};

struct ServeApp {
  ServeSlot *ring;              // host-mapped
  unsigned long long *done;     // host-mapped [ring]
  const uint32_t *stop;         // host-mapped
  ServeDev *sd;
  ReqState *rs;
  uint32_t ring_n;
  uint64_t budget;              // lines that admitted requests may hold together
  uint32_t mode;
  // serving requests only what it sums: every queue pair carries demand
  bool demand_only() const { return true; }
  uint32_t group;

  __device__ void schedule(const Dev &d, const AppCtx &a) const {
    // lane 0 only
    uint64_t next = sd->admitted;
    uint32_t ns = 256;
    for (;;) {
      if (gtimer() > a.deadline || aborted(d)) {
        set_error(d, -110);
        st_rlx32(&sd->stop_seen, 1u);
        return;
      }
      const ServeSlot *slot = &ring[next % ring_n];
      uint64_t sq = ld_acq_sys64(&slot->seq);
      if (sq == next + 1) {
        uint32_t n_bags = ld_vol_sys32(&slot->n_bags);
        const int64_t *off = (const int64_t *)ld_vol_sys64(&slot->offsets);
        uint64_t nidx = n_bags ? (uint64_t)ld_cg_s64(&off[n_bags]) : 0;
        uint64_t need = nidx + 1 < budget ? nidx + 1 : budget;
        // admission: the request's lines must fit in the free budget (oldest first)
        if (ld_acq64(&sd->used) + need <= budget || ld_acq64(&sd->finished) == next) {
          atomicAdd(&sd->used, (unsigned long long)need);
          ReqState *r = &rs[next % ring_n];
          r->next_bag = 0;
          r->bags_done = 0;
          r->n_bags = n_bags;
          r->need = (uint32_t)need;
          __threadfence();
          st_rel64(&r->seq, next + 1);
          if (n_bags == 0) {  // nothing to compute: finished at admission
            atomicAdd(&sd->used, (unsigned long long)(-(int64_t)need));
            st_rel_sys64(&done[next % ring_n], next + 1);
            atomicAdd(&sd->finished, 1ull);
          }
          ++next;
          st_rel64(&sd->admitted, next);
          ns = 256;
          continue;
        }
      } else if (ld_vol_sys32(stop) && ld_acq64(&sd->finished) == next) {
        st_rlx32(&sd->stop_seen, 1u);  // every request published before stop is finished
        return;
      }
      __nanosleep(ns);
      ns = ns < 4096 ? ns * 2 : 4096;
    }
  }

  // one bag of request `q` (entry e): the same arithmetic as agile_embedding_bag
  __device__ bool bag(const Dev &d, const AppCtx &a, const ServeSlot *slot, uint32_t b) const {
    unsigned l = lane_id();
    uint64_t table_byte0 = ld_vol_sys64(&slot->table_byte0);
    uint32_t rows = ld_vol_sys32(&slot->rows), dim = ld_vol_sys32(&slot->dim);
    const int64_t *idx = (const int64_t *)ld_vol_sys64(&slot->idx);
    const int64_t *off = (const int64_t *)ld_vol_sys64(&slot->offsets);
    float *out = (float *)ld_vol_sys64(&slot->out);
    uint64_t page0 = table_byte0 / kPage;
    uint32_t nf4 = dim / 4;
    float4 acc[1] = {make_float4(0.f, 0.f, 0.f, 0.f)};
    int64_t s = ld_cg_s64(&off[b]), e = ld_cg_s64(&off[b + 1]);
    for (int64_t i0 = s; i0 < e; i0 += 32) {
      int64_t i = i0 + l;
      uint64_t r = i < e ? (uint64_t)ld_cg_s64(&idx[i]) : 0;
      if (i < e && r >= rows) {
        set_error(d, AGILE_EINVAL);
        r = 0;
      }
      uint32_t cnt = (uint32_t)min((int64_t)32, e - i0);
      uint64_t byte = r * dim * 4;
      if (mode == AGILE_ASYNC && !warp_request(d, l < cnt, page0 + byte / kPage, a.q0, false, a.deadline))
        return false;
      for (uint32_t g0 = 0; g0 < cnt; g0 += group) {
        uint32_t g1 = min(cnt, g0 + group);
        if (!gather_sum<1>(d, a, g0, g1, page0 + byte / kPage, (uint32_t)(byte % kPage), nf4, acc)) return false;
      }
    }
    if (l < nf4) ((float4 *)(out + (uint64_t)b * dim))[l] = acc[0];
    return true;
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    if (a.warp == 0) {
      if (l == 0) schedule(d, a);
      __syncwarp();
      return;
    }
    uint32_t ns = 64;
    for (;;) {
      // find a bag: oldest admitted request with bags left
      int act = 0;  // 0 idle, 1 bag, 2 exit
      uint64_t q = 0;
      uint32_t b = 0;
      if (l == 0) {
        uint64_t adm = ld_acq64(&sd->admitted);
        uint64_t cur = ld_acq64(&sd->cursor);
        act = ld_rlx32(&sd->stop_seen) && cur >= adm ? 2 : 0;
        for (uint64_t k = cur; k < adm && act == 0; ++k) {
          ReqState *r = &rs[k % ring_n];
          if (ld_acq64(&r->seq) != k + 1) break;
          uint32_t nb = ld_rlx32(&r->n_bags);
          if (ld_rlx32(&r->next_bag) >= nb) {
            if (k == cur) {
              atomicMax(&sd->cursor, k + 1);
              cur = k + 1;
            }
            continue;
          }
          uint32_t got = atomicAdd(&r->next_bag, 1u);
          if (got < nb) {
            act = 1;
            q = k;
            b = got;
          }
        }
      }
      act = __shfl_sync(kFull, act, 0);
      if (act == 2 || aborted(d)) return;
      if (act == 0) {
        if (gtimer() > a.deadline) {
          if (l == 0) set_error(d, -110);
          return;
        }
        __nanosleep(ns);
        ns = ns < 2048 ? ns * 2 : 2048;
        continue;
      }
      ns = 64;
      q = __shfl_sync(kFull, q, 0);
      b = __shfl_sync(kFull, b, 0);
      const ServeSlot *slot = &ring[q % ring_n];
      if (!bag(d, a, slot, b)) return;
      __threadfence_system();
      __syncwarp();
      if (l == 0) {
        ReqState *r = &rs[q % ring_n];
        uint32_t nb = ld_rlx32(&r->n_bags);
        if (atomicAdd(&r->bags_done, 1u) + 1 == nb) {
          // last bag: publish completion to the host, return the budget
          atomicAdd(&sd->used, (unsigned long long)(-(int64_t)r->need));
          st_rel_sys64(&done[q % ring_n], q + 1);
          atomicAdd(&sd->finished, 1ull);
        }
      }
    }
  }
};

}  // namespace

struct agile_server {
  agile_ctx *ctx;
  uint32_t ring_n;
  ServeSlot *ring;           // pinned mapped host memory
  unsigned long long *done;  // pinned mapped host memory
  uint32_t *stop;            // pinned mapped host memory
  void *dstate;              // device: ServeDev + ReqState[ring]
  uint64_t next_seq;
  cudaStream_t stream;
};

extern "C" {

int agile_serve_start(agile_ctx *c, uint32_t ring_slots, uint32_t mode, uint64_t session_ns, void *stream,
                      agile_server **out) {
  if (!c || !out || mode > 1 || ring_slots == 0 || ring_slots > (1u << 20)) return AGILE_EINVAL;
  *out = nullptr;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  agile_server *s = new agile_server();
  s->ctx = c;
  s->ring_n = ring_slots;
  s->stream = as_stream(stream);
  if (cudaHostAlloc((void **)&s->ring, sizeof(ServeSlot) * ring_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void **)&s->done, 8ull * ring_slots, cudaHostAllocMapped) != cudaSuccess ||
      cudaHostAlloc((void **)&s->stop, 64, cudaHostAllocMapped) != cudaSuccess ||
      cudaMalloc(&s->dstate, sizeof(ServeDev) + sizeof(ReqState) * ring_slots) != cudaSuccess) {
    if (s->ring) cudaFreeHost(s->ring);
    if (s->done) cudaFreeHost(s->done);
    if (s->stop) cudaFreeHost(s->stop);
    delete s;
    return AGILE_ENOMEM;
  }
  memset(s->ring, 0, sizeof(ServeSlot) * ring_slots);
  memset(s->done, 0, 8ull * ring_slots);
  memset(s->stop, 0, 64);
  AGILE_CUDA_TRY(cudaMemsetAsync(s->dstate, 0, sizeof(ServeDev) + sizeof(ReqState) * ring_slots, s->stream));
  void *ring_d = nullptr, *done_d = nullptr, *stop_d = nullptr;
  AGILE_CUDA_TRY(cudaHostGetDevicePointer(&ring_d, s->ring, 0));
  AGILE_CUDA_TRY(cudaHostGetDevicePointer(&done_d, s->done, 0));
  AGILE_CUDA_TRY(cudaHostGetDevicePointer(&stop_d, s->stop, 0));
  uint32_t warps = warps_for_cache(c, 4, 32);
  // pin groups sized by the warps that run (one of them schedules)
  uint32_t run = running_app_warps<ServeApp>(c, warps + 1);
  ServeApp app{(ServeSlot *)ring_d, (unsigned long long *)done_d, (const uint32_t *)stop_d,
               (ServeDev *)s->dstate, (ReqState *)((ServeDev *)s->dstate + 1), ring_slots,
               c->dev.nlines / 2, mode, std::max<uint32_t>(1, std::min<uint32_t>(32, (uint32_t)(c->dev.nlines / (2ull * run))))};
  uint64_t saved = c->dev.session_ns;
  c->dev.session_ns = session_ns ? session_ns : 60ull * 1000 * 1000 * 1000;
  int r = launch_engine(c, app, stream, warps + 1);
  c->dev.session_ns = saved;
  if (r) {
    cudaFreeHost(s->ring);
    cudaFreeHost(s->done);
    cudaFreeHost(s->stop);
    cudaFree(s->dstate);
    delete s;
    return r;
  }
  *out = s;
  return AGILE_OK;
}

int agile_serve_submit(agile_server *s, const agile_lookup_req *req, uint64_t *seq_out) {
  if (!s || !req) return AGILE_EINVAL;
  if (req->dim == 0 || req->dim > 128 || req->dim % 4 || kPage % (req->dim * 4) || req->table_byte0 % kPage ||
      req->table_byte0 + (uint64_t)req->rows * req->dim * 4 > s->ctx->cfg.store_bytes || !req->d_offsets ||
      (req->n_bags && (!req->d_idx || !req->d_out)) || (((uintptr_t)req->d_out) & 15))
    return AGILE_EINVAL;
  uint64_t q = s->next_seq;
  // the ring entry is free once the request that used it last has finished
  if (q >= s->ring_n) {
    volatile unsigned long long *dn = s->done;
    if (dn[q % s->ring_n] != q - s->ring_n + 1) return AGILE_EAGAIN;
  }
  ServeSlot *slot = &s->ring[q % s->ring_n];
  slot->table_byte0 = req->table_byte0;
  slot->idx = (uint64_t)req->d_idx;
  slot->offsets = (uint64_t)req->d_offsets;
  slot->out = (uint64_t)req->d_out;
  slot->rows = req->rows;
  slot->dim = req->dim;
  slot->n_bags = req->n_bags;
  std::atomic_thread_fence(std::memory_order_release);
  reinterpret_cast<std::atomic<unsigned long long> *>(&slot->seq)->store(q + 1, std::memory_order_release);
  s->next_seq = q + 1;
  if (seq_out) *seq_out = q;
  return AGILE_OK;
}

int agile_serve_poll(agile_server *s, uint64_t seq) {
  if (!s) return AGILE_EINVAL;
  if (seq >= s->next_seq) return AGILE_EINVAL;
  volatile unsigned long long *dn = s->done;
  uint64_t v = dn[seq % s->ring_n];
  if (v >= seq + 1) return 1;  // this request, or a later one that reused the entry
  return 0;
}

int agile_serve_stop(agile_server *s) {
  if (!s) return AGILE_EINVAL;
  std::atomic_thread_fence(std::memory_order_release);
  reinterpret_cast<std::atomic<uint32_t> *>(s->stop)->store(1, std::memory_order_release);
  cudaError_t e = cudaStreamSynchronize(s->stream);
  int r = agile_check(s->ctx);
  cudaFreeHost(s->ring);
  cudaFreeHost(s->done);
  cudaFreeHost(s->stop);
  cudaFree(s->dstate);
  delete s;
  if (e != cudaSuccess) return AGILE_ECUDA;
  return r;
}

int agile_serve_replay(agile_ctx *c, const agile_lookup_req *reqs, uint32_t n, const uint64_t *arrival_ns,
                       uint64_t *latency_ns, uint32_t mode, void *stream) {
  if (!c || (n && (!reqs || !arrival_ns || !latency_ns))) return AGILE_EINVAL;
  agile_server *s = nullptr;
  uint64_t span = n ? arrival_ns[n - 1] : 0;
  int r = agile_serve_start(c, std::max<uint32_t>(64, std::min<uint32_t>(n ? n : 1, 4096)), mode,
                            span + 60ull * 1000 * 1000 * 1000, stream, &s);
  if (r) return r;
  using clk = std::chrono::steady_clock;
  std::vector<char> fin(n, 0);
  uint32_t next = 0, finished = 0;
  auto t0 = clk::now();
  auto deadline = t0 + std::chrono::nanoseconds(span) + std::chrono::seconds(60);
  uint32_t lowest = 0;
  while (finished < n) {
    auto now = clk::now();
    if (now > deadline) break;
    // submit every request whose arrival time has come (a full ring defers it)
    while (next < n && now - t0 >= std::chrono::nanoseconds(arrival_ns[next])) {
      uint64_t q;
      int rr = agile_serve_submit(s, &reqs[next], &q);
      if (rr == AGILE_EAGAIN) break;
      if (rr) {
        agile_serve_stop(s);
        return rr;
      }
      ++next;
    }
    for (uint32_t i = lowest; i < next; ++i) {
      if (fin[i]) continue;
      if (agile_serve_poll(s, i) == 1) {
        fin[i] = 1;
        // from the request's arrival time: time spent waiting for a ring entry counts
        auto arrived = t0 + std::chrono::nanoseconds(arrival_ns[i]);
        latency_ns[i] = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(clk::now() - arrived).count();
        ++finished;
      }
    }
    while (lowest < next && fin[lowest]) ++lowest;
  }
  int rs = agile_serve_stop(s);
  if (finished < n) return AGILE_ETIMEDOUT;
  return rs;
}

}  // extern "C"
