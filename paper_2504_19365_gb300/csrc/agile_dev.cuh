// Device-side state and primitives of the AGILE I/O path for sm_103a.
//
// Layout in HBM (all library-owned, allocated once per context):
//   lines      [nlines * 4096]      cache data, one 4 KiB line per store page (Sec. 2.3.3)
//   tag        [nlines] u64         {page:44 | pin:16 | wb:1 | ref:1 | state:2} (Sec. 3.4)
//   hand       [sets]   u32         clock hand per set (Sec. 4.4, clock policy)
//   sh_key/val [buckets*4] u64      in-flight share table, 4 slots per bucket (Sec. 3.4.1)
//   sq         [Q * depth] 64 B     NVMe submission entries (Sec. 2.1)
//   cq         [Q * 2*depth] 16 B   NVMe completion entries with phase bit (Sec. 2.1)
//   sqe_state  [Q * depth] u64      {ticket:62 | EMPTY/UPDATED/ISSUED} (Sec. 3.3.1)
//   cmd_ctx    [Q * depth] u64      what a completion releases (line fill, write-back)
//   cmpl       [Q * depth] u64      completion word = transaction barrier (Sec. 3.2.1)
//   sq_resv    [Q] u64              {in flight:32 | next ticket:32}
//   sq_tail/sq_lock/sq_db [Q] u32   doorbell-lock holder's tail, the lock, doorbell
//   cq_db      [Q] u32              CQ head doorbell
//   cq_poll    [Q*4] u32            Alg. 1 state {offset, mask, phase}
//   emu*                            emulated device: fetch/seen/CQ-slot counters, timing
//   staging    [Q * depth * 4096]   write-back sources, one page per submission slot
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace agile {

constexpr uint32_t kPage = 4096;
constexpr int kWarps = 8;             // warps per CTA: warp 0 = service, 1..7 = app
constexpr int kThreads = kWarps * 32;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- tag word (Sec. 3.4)
constexpr uint64_t ST_MASK = 3, ST_INVALID = 0, ST_BUSY = 1, ST_READY = 2, ST_MODIFIED = 3;
constexpr uint64_t TAG_REF = 1ull << 2;
constexpr uint64_t TAG_WB = 1ull << 3;
constexpr int PIN_SHIFT = 4;
constexpr uint64_t PIN1 = 1ull << PIN_SHIFT;
constexpr uint64_t PIN_MASK = 0xFFFFull << PIN_SHIFT;
constexpr int PAGE_SHIFT = 20;
__host__ __device__ __forceinline__ uint64_t tag_page(uint64_t t) { return t >> PAGE_SHIFT; }
__host__ __device__ __forceinline__ uint64_t tag_state(uint64_t t) { return t & ST_MASK; }
__host__ __device__ __forceinline__ uint64_t tag_make(uint64_t page, uint64_t st, bool ref) {
  return (page << PAGE_SHIFT) | (ref ? TAG_REF : 0) | st;
}

// replacement policies (agile.h AGILE_POLICY_*)
constexpr uint32_t kPolicyClock = 0, kPolicyFifo = 1;

// ---------------------------------------------------------------- queues (Sec. 3.3.1)
constexpr uint64_t SQE_EMPTY = 0, SQE_UPDATED = 1, SQE_ISSUED = 2;
constexpr uint32_t OP_FLUSH = 0x00, OP_WRITE = 0x01, OP_READ = 0x02;

// command context: what the completion of a command releases (CTX_BUF: a read into a
// user buffer, which releases only the page's in-flight entry)
constexpr uint64_t CTX_NOP = 0, CTX_FILL = 1, CTX_WB = 2, CTX_BUF = 3;
__host__ __device__ __forceinline__ uint64_t ctx_make(uint64_t kind, uint32_t share_slot, uint32_t idx) {
  return (kind << 60) | ((uint64_t)(share_slot & 0x0FFFFFFFu) << 32) | idx;
}

struct alignas(64) Sqe { uint32_t dw[16]; };
struct alignas(16) Cqe { uint32_t dw[4]; };

// statistic slots (mirror agile_stats_t order)
enum Stat {
  S_HITS, S_MISSES, S_BUSY_HITS, S_WARP_COALESCED, S_SHARE_RETRIES, S_EVICTIONS, S_WRITEBACKS,
  S_EAGAIN, S_SQ_FULL, S_DOORBELLS, S_COMMANDS, S_CQES, S_CQ_DOORBELLS, S_IO_ERRORS,
  S_BYTES_READ, S_BYTES_WRITTEN, S_PREFETCHES, S_TIMEOUTS, S_COUNT
};

// per-launch state, zeroed before every launch (and numbered) by run_reset_kernel
struct RunState {
  uint32_t app_done;      // app warps finished
  uint32_t error;         // first error code (negated AGILE_E*), 0 = none
  uint32_t bar_count;     // grid barrier arrivals
  uint32_t bar_gen;       // grid barrier generation
  uint32_t work[4];       // dynamic work counters
  unsigned long long acc[4];  // accumulators (edges scanned, discovered vertices, ...)
  uint32_t flag[4];
  unsigned long long epoch;  // number of this launch among the device's launches (never 0)
  // BFS slice queue, per level parity, each on a line of its own (hot words)
  alignas(128) uint32_t hub_count[2];  // slices of long adjacency lists reserved
  alignas(128) uint32_t hub_cursor[2];  // next slice ticket
  alignas(128) uint32_t units_done[2];  // warps that finished their own vertices
};

// One command as the emulated device served it (times from %globaltimer, ns).
struct TraceRec {
  unsigned long long page;    // store page of the command
  unsigned long long t_seen;  // doorbell that exposed it first read by the device (0 when
                              // the device runs without a latency or throughput model)
  unsigned long long t_start; // taken by an engine: data movement starts
  unsigned long long t_done;  // completion entry posted
  uint32_t q, cid, opcode, status;
  unsigned long long t_commit;  // the command was written to its submission slot
  uint32_t pad[2];
};

struct Dev {
  // backing store (pinned host memory, device-visible address)
  uint8_t *store;
  uint64_t store_bytes;
  // cache
  uint8_t *lines;
  unsigned long long *tag;
  uint32_t *hand;
  uint64_t nlines;
  uint32_t sets, ways;
  unsigned long long *sh_key;
  unsigned long long *sh_val;
  uint32_t sh_mask;  // buckets - 1 (power of two)
  // queues
  uint32_t Q, depth, dmask, dlog;
  uint32_t Qp;       // queues [Q - Qp, Q) carry prefetches, served after the demand queues
  uint32_t cq_size;  // CQ entries per queue = 2 * depth
  Sqe *sq;
  Cqe *cq;
  unsigned long long *sqe_state;
  unsigned long long *cmd_ctx;
  unsigned long long *cmpl;
  unsigned long long *sq_resv;
  uint32_t *sq_tail, *sq_lock, *sq_db, *cq_db, *cq_poll;
  uint32_t *emu;  // [Q*4] device counters {fetch, seen, cq slot, -}
  unsigned long long *emu_busy;     // [Q] ns at which the queue's device pipe is free
  unsigned long long *emu_arrival;  // [Q*depth] ns at which the device saw the command
  uint8_t *staging;
  // per store page: reads and writes the device served, dirty epochs the cache opened
  // (a clean line turned MODIFIED, or a write-through issued); every dirty epoch ends in
  // exactly one write
  uint32_t *pg_reads, *pg_writes, *pg_dirty;
  // command trace (optional): one record per command the device served
  struct TraceRec *trace;
  uint32_t trace_cap;
  uint32_t *trace_n;
  // application event log (optional, same capacity): {time, warp | kind << 32 | arg << 40}
  unsigned long long *ev;
  uint32_t *ev_n;
  // Share Table of user buffers (Sec. 3.4.1): 4 slots per bucket; key = page + 1,
  // buf = the buffer's address, meta = {state:8 | count:32 | closing:1}, tok = the token
  // of the read that fills the buffer (valid once the entry has left PENDING)
  unsigned long long *ub_key, *ub_buf, *ub_meta, *ub_tok;
  uint32_t ub_mask;  // buckets - 1; ub_key == nullptr: no Share Table
  // backing devices: page p lives on device p mod ndev at block p / ndev; queue q
  // belongs to device q mod ndev (Sec. 4.3: requests interleaved over the SSDs)
  uint32_t ndev;
  // replacement policy of the cache (AGILE_POLICY_*)
  uint32_t policy;
  // emulated device model
  uint64_t lat_ns, ns_per_page;
  uint64_t ns_rd_dev, ns_wr_dev;    // per-device time of one page read / written (0 = no cap)
  unsigned long long *dev_busy;     // [ndev] ns up to which the device is booked
  uint32_t fault_flags, fault_thresh;
  uint64_t seed;
  // run
  RunState *run;
  unsigned long long *stats;
  uint64_t timeout_ns;
  uint32_t prefetch_depth;
  int32_t *err_sticky;  // first error since the last agile_check
  uint32_t app_active;  // application warps that take part in this launch (0 = all)
  uint32_t extra_engines;  // idle application warps that may also serve the device
  uint64_t session_ns;  // length of a long-running launch (serving loop); 0 = timeout_ns
};

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint32_t ld_acq32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_acq64(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_rlx32(const uint32_t *p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t ld_rlx64(const unsigned long long *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel32(uint32_t *p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_rel64(unsigned long long *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rlx64(unsigned long long *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_rlx32(uint32_t *p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t atom_add_acq(unsigned long long *p, uint64_t v) {
  uint64_t old;
  asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(old) : "l"(p), "l"(v) : "memory");
  return old;
}
__device__ __forceinline__ void fence_sc() { asm volatile("fence.sc.gpu;" ::: "memory"); }
__device__ __forceinline__ void fence_ar() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// 16-byte loads/stores that bypass L1: cache lines and store pages are rewritten by
// other SMs during a launch, so nothing here may be served from a stale L1 copy.
__device__ __forceinline__ int4 ld_cg16(const void *p) {
  int4 v;
  asm volatile("ld.global.cg.v4.s32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_cg16(void *p, int4 v) {
  asm volatile("st.global.cg.v4.s32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w) : "memory");
}
__device__ __forceinline__ float4 ld_cg_f4(const void *p) {
  int4 v = ld_cg16(p);
  return make_float4(__int_as_float(v.x), __int_as_float(v.y), __int_as_float(v.z), __int_as_float(v.w));
}
__device__ __forceinline__ int32_t ld_cg_s32(const void *p) {
  int32_t v;
  asm volatile("ld.global.cg.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int64_t ld_cg_s64(const void *p) {
  int64_t v;
  asm volatile("ld.global.cg.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31; }

// counters are kept in kStatShards copies (by CTA) so that warps all over the GPU do not
// serialise on one address; the host adds the copies up
constexpr int kStatShards = 32;
__device__ __forceinline__ unsigned long long *stat_ptr(const Dev &d, int s) {
  return &d.stats[(blockIdx.x % kStatShards) * S_COUNT + s];
}

__device__ __forceinline__ void stat_add(const Dev &d, int s, uint64_t v) {
  if (v) atomicAdd(stat_ptr(d, s), (unsigned long long)v);
}
// warp-aggregated statistic: every lane passes its own count
__device__ __forceinline__ void stat_warp(const Dev &d, int s, uint32_t v) {
  unsigned b = __ballot_sync(kFull, v != 0);
  if (!b) return;
  uint32_t sum = __reduce_add_sync(kFull, v);
  if (lane_id() == 0) atomicAdd(stat_ptr(d, s), (unsigned long long)sum);
}

// Application event (lane 0 of a warp; only with the trace on): `kind` names the
// event, `arg` a small number (a level, ...).
__device__ __forceinline__ void app_event(const Dev &d, uint32_t warp, uint32_t kind, uint32_t arg) {
  if (!d.ev) return;
  uint32_t i = atomicAdd(d.ev_n, 1u);
  if (i < d.trace_cap) {
    d.ev[2 * i] = gtimer();
    d.ev[2 * i + 1] = (uint64_t)warp | ((uint64_t)(kind & 0xFF) << 32) | ((uint64_t)(arg & 0xFFFFFF) << 40);
  }
}

// A cache line of `page` turned from clean to MODIFIED (or a write-through was issued):
// the page owes the store one write.
__device__ __forceinline__ void note_dirty(const Dev &d, uint64_t page) {
  atomicAdd(&d.pg_dirty[page], 1u);
}

// record the first error of the launch and of the context
__device__ __forceinline__ void set_error(const Dev &d, int code) {
  atomicCAS(&d.run->error, 0u, (uint32_t)(-code));
  atomicCAS((uint32_t *)d.err_sticky, 0u, (uint32_t)(-code));
  if (code == -110) atomicAdd(stat_ptr(d, S_TIMEOUTS), 1ull);
}
__device__ __forceinline__ bool aborted(const Dev &d) { return ld_rlx32(&d.run->error) != 0; }

__device__ __forceinline__ void backoff(uint32_t &ns, uint32_t cap = 2048) {
  __nanosleep(ns);
  ns = ns < cap ? ns * 2 : cap;
}

// ---------------------------------------------------------------- cache geometry
// Set index: golden-ratio multiplicative hash of the page, upper 32 bits scaled to
// [0, sets).  Works for any number of sets.
__host__ __device__ __forceinline__ uint32_t set_of(uint64_t page, uint32_t sets) {
  uint64_t h = page * 0x9E3779B97F4A7C15ull;
  return (uint32_t)(((h >> 32) * (uint64_t)sets) >> 32);
}
__device__ __forceinline__ uint8_t *line_ptr(const Dev &d, uint64_t line) {
  return d.lines + line * (uint64_t)kPage;
}

// ---------------------------------------------------------------- warp page copy
// One warp moves one 4 KiB page with 16-byte accesses: 8 loads in flight per lane,
// then 8 stores, so each request is a single 512-byte coalesced transaction per step.
__device__ __forceinline__ void warp_copy_page(void *dst, const void *src) {
  const int4 *s = (const int4 *)src;
  int4 *t = (int4 *)dst;
  unsigned l = lane_id();
  int4 v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = ld_cg16(s + k * 32 + l);
#pragma unroll
  for (int k = 0; k < 8; ++k) st_cg16(t + k * 32 + l, v[k]);
}
// A single thread moves a page (rare paths: write-back copies inside a lane's miss).
__device__ __forceinline__ void lane_copy_page(void *dst, const void *src) {
  const int4 *s = (const int4 *)src;
  int4 *t = (int4 *)dst;
  for (int k = 0; k < 256; k += 16) {
    int4 v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = ld_cg16(s + k + j);
#pragma unroll
    for (int j = 0; j < 16; ++j) st_cg16(t + k + j, v[j]);
  }
}

// ================================================================ submission side
// Alg. 2, check_full: reserve n consecutive slots of queue q.  A slot is free when
// the command that used it last has completed (state EMPTY) and fewer than depth-1
// commands are outstanding (the NVMe full rule).  Never waits.
__device__ __forceinline__ bool sq_try_reserve(const Dev &d, uint32_t q, uint32_t n,
                                               uint32_t &slot, uint32_t &ticket) {
  unsigned long long *rp = &d.sq_resv[q];
  uint64_t w = ld_rlx64(rp);
  for (int tries = 0; tries < 4; ++tries) {
    uint32_t t = (uint32_t)w, infl = (uint32_t)(w >> 32);
    if (infl + n > d.depth - 1) return false;
    for (uint32_t k = 0; k < n; ++k) {
      uint64_t st = ld_acq64(&d.sqe_state[(uint64_t)q * d.depth + ((t + k) & d.dmask)]);
      if ((st & 3) != SQE_EMPTY) return false;
    }
    uint64_t nw = ((uint64_t)(infl + n) << 32) | (uint32_t)(t + n);
    uint64_t old = atomicCAS(rp, (unsigned long long)w, (unsigned long long)nw);
    if (old == w) {
      slot = t & d.dmask;
      ticket = t;
      return true;
    }
    w = old;
  }
  return false;
}

// Backing device of a store page and its block number there (4 KiB blocks).
__host__ __device__ __forceinline__ uint32_t dev_of_page(const Dev &d, uint64_t page) {
  return d.ndev > 1 ? (uint32_t)(page % d.ndev) : 0u;
}
__host__ __device__ __forceinline__ uint64_t block_of_page(const Dev &d, uint64_t page) {
  return d.ndev > 1 ? page / d.ndev : page;
}

// SQ selection (Sec. 3.3.1): among the queues of the page's device in the request's
// class -- demand queues [0, Q - Qp), prefetch queues [Q - Qp, Q) (NVMe-style
// arbitration: the device serves demand queues first, so requests made ahead of need
// only use device time that demand leaves idle) -- start at the one nearest the
// thread's own queue, on a full queue try the class's next one of the device; false
// after one pass over them.
__device__ __forceinline__ bool sq_reserve_dev(const Dev &d, uint32_t q0, uint32_t dv, uint32_t n, uint32_t &q,
                                               uint32_t &slot, uint32_t &ticket, bool pf = false) {
  const uint32_t nd = d.ndev > 1 ? d.ndev : 1u;
  const uint32_t base = pf && d.Qp ? d.Q - d.Qp : 0u;
  const uint32_t cnt = d.Qp ? (pf ? d.Qp : d.Q - d.Qp) : d.Q;
  const uint32_t per = cnt / nd;  // queues of one device in the class
  uint32_t k0 = (q0 / nd) % per;
  // a request made ahead of need tries two queues: when they are full the device is
  // saturated and the request is dropped (a hint), not spread over every queue
  const uint32_t tries = pf ? min(per, 2u) : per;
  for (uint32_t k = 0; k < tries; ++k) {
    uint32_t kk = k0 + k;
    if (kk >= per) kk -= per;
    uint32_t qq = base + kk * nd + dv;
    if (sq_try_reserve(d, qq, n, slot, ticket)) {
      q = qq;
      return true;
    }
  }
  atomicAdd(stat_ptr(d, S_SQ_FULL), 1ull);
  return false;
}

// The first queue sq_reserve_dev tries for a request of this class holds more than
// 3/4 of its depth in flight: a request made ahead of need is then dropped before it
// claims a line (one load instead of a claim, a failed reservation and an unclaim).
__device__ __forceinline__ bool sq_crowded(const Dev &d, uint32_t q0, uint32_t dv, bool pf) {
  const uint32_t nd = d.ndev > 1 ? d.ndev : 1u;
  const uint32_t base = pf && d.Qp ? d.Q - d.Qp : 0u;
  const uint32_t cnt = d.Qp ? (pf ? d.Qp : d.Q - d.Qp) : d.Q;
  const uint32_t per = cnt / nd;
  const uint32_t qq = base + ((q0 / nd) % per) * nd + dv;
  return (uint32_t)(ld_rlx64(&d.sq_resv[qq]) >> 32) > (d.depth - 1) / 4 * 3;
}

// Alg. 2, enqueue_cmd + update_SQE: write the 64-byte command, then publish the slot
// as UPDATED.  CID = slot index (unique while the command is outstanding).
__device__ __forceinline__ void sq_commit(const Dev &d, uint32_t q, uint32_t slot, uint32_t ticket,
                                          uint32_t opcode, uint64_t prp1, uint64_t page,
                                          uint64_t ctx) {
  uint64_t i = (uint64_t)q * d.depth + slot;
  uint32_t *e = d.sq[i].dw;
  uint64_t slba = block_of_page(d, page) * (kPage / 512);
  // dw2-3 (reserved in NVMe) carry the commit time for the device's trace
  uint64_t now = gtimer();
  int4 a = make_int4((int)(opcode | (slot << 16)), 1, (int)(uint32_t)now, (int)(uint32_t)(now >> 32));  // dw0-3
  int4 b = make_int4(0, 0, (int)(uint32_t)prp1, (int)(uint32_t)(prp1 >> 32));      // dw4-7
  int4 c = make_int4(0, 0, (int)(uint32_t)slba, (int)(uint32_t)(slba >> 32));      // dw8-11
  int4 f = make_int4((int)(kPage / 512 - 1), 0, 0, 0);                             // dw12-15
  st_cg16(e, a);
  st_cg16(e + 4, b);
  st_cg16(e + 8, c);
  st_cg16(e + 12, f);
  st_rlx64(&d.cmd_ctx[i], ctx);
  // the release orders the command's stores (and the caller's earlier ones) before the
  // state: whoever acquires UPDATED -- the doorbell-lock holder, then the device through
  // the doorbell -- sees them
  st_rel64(&d.sqe_state[i], ((uint64_t)ticket << 2) | SQE_UPDATED);
}

// Alg. 2, move_SQ_tail: the doorbell-lock holder turns UPDATED slots into ISSUED from
// the tail up to the first slot that is not UPDATED, then writes the doorbell once.
__device__ __forceinline__ void sq_move_tail(const Dev &d, uint32_t q) {
  uint32_t t = ld_rlx32(&d.sq_tail[q]);
  uint32_t n = 0;
  while (n < d.depth) {
    uint64_t i = (uint64_t)q * d.depth + (t & d.dmask);
    uint64_t st = ld_acq64(&d.sqe_state[i]);
    if (st != (((uint64_t)t << 2) | SQE_UPDATED)) break;
    st_rlx64(&d.sqe_state[i], ((uint64_t)t << 2) | SQE_ISSUED);
    ++t;
    ++n;
  }
  if (n) {
    st_rlx32(&d.sq_tail[q], t);
    fence_ar();
    st_rel32(&d.sq_db[q], t & d.dmask);
    atomicAdd(stat_ptr(d, S_DOORBELLS), 1ull);
  }
}

// Alg. 2, Attempt_SQDB: try the doorbell lock, move the tail if it is ours, and report
// whether our command has left the UPDATED state.
__device__ __forceinline__ bool sq_attempt_db(const Dev &d, uint32_t q, uint32_t slot, uint32_t ticket) {
  if (atomicCAS(&d.sq_lock[q], 0u, 1u) == 0u) {
    fence_ar();
    sq_move_tail(d, q);
    fence_ar();
    atomicExch(&d.sq_lock[q], 0u);
  }
  uint64_t st = ld_acq64(&d.sqe_state[(uint64_t)q * d.depth + slot]);
  return !((st >> 2) == (uint64_t)ticket && (st & 3) == SQE_UPDATED);
}

// Warp-collective doorbell batching: lanes with `has` committed a command to queue q.
// One leader per queue rings for the whole group; then every lane repeats
// Attempt_SQDB until its own command is ISSUED (bounded by the deadline).
__device__ __forceinline__ bool warp_ring(const Dev &d, bool has, uint32_t q, uint32_t slot,
                                          uint32_t ticket, uint64_t deadline) {
  unsigned m = __match_any_sync(kFull, has ? q : 0xFFFFFFFFu);
  bool leader = has && (__ffs(m) - 1 == (int)lane_id());
  bool pending = has;
  if (leader) pending = !sq_attempt_db(d, q, slot, ticket);
  __syncwarp();
  if (has && pending) {
    uint64_t st = ld_acq64(&d.sqe_state[(uint64_t)q * d.depth + slot]);
    pending = ((st >> 2) == (uint64_t)ticket && (st & 3) == SQE_UPDATED);
  }
  uint32_t ns = 32;
  while (pending) {
    if (sq_attempt_db(d, q, slot, ticket)) break;
    if (gtimer() > deadline) {
      set_error(d, -110);
      return false;
    }
    backoff(ns);
  }
  return true;
}

// ================================================================ in-flight share table
// Sec. 3.4.1: page -> request in flight.  A bucket of 4 slots per hash; the slot key is
// page+1 (0 = free).  Inserting the key is how a thread takes ownership of a page's
// miss (or write); any other thread that finds the key defers and retries.
constexpr uint64_t SH_FILL = 1, SH_WRITE = 2;
__device__ __forceinline__ uint32_t sh_bucket(const Dev &d, uint64_t page) {
  uint64_t h = (page + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
  return (uint32_t)(h >> 40) & d.sh_mask;
}
// returns slot index >= 0 when inserted, -1 when the page is already present (or a
// racing insert of the same page was seen), -2 when the bucket is full.
__device__ __forceinline__ int64_t sh_insert(const Dev &d, uint64_t page, uint64_t kind) {
  uint64_t key = page + 1;
  uint64_t base = (uint64_t)sh_bucket(d, page) * 4;
  for (int tries = 0; tries < 8; ++tries) {
    int free_k = -1;
    for (int k = 0; k < 4; ++k) {
      uint64_t v = ld_acq64(&d.sh_key[base + k]);
      if (v == key) return -1;
      if (v == 0 && free_k < 0) free_k = k;
    }
    if (free_k < 0) return -2;
    if (atomicCAS(&d.sh_key[base + free_k], 0ull, (unsigned long long)key) != 0ull) continue;
    // a racing insert of the same key into another slot: whoever sees the other backs off
    fence_sc();
    bool dup = false;
    for (int k = 0; k < 4; ++k)
      if (k != free_k && ld_acq64(&d.sh_key[base + k]) == key) dup = true;
    if (dup) {
      st_rel64(&d.sh_key[base + free_k], 0ull);
      return -1;
    }
    (void)kind;
    st_rlx64(&d.sh_val[base + free_k], 0ull);  // the token of the read, once issued
    return (int64_t)(base + free_k);
  }
  return -2;
}
__device__ __forceinline__ void sh_remove(const Dev &d, uint64_t slot) {
  st_rlx64(&d.sh_val[slot], 0ull);
  st_rel64(&d.sh_key[slot], 0ull);
}
// Token of the read in flight for `page`, ~0 when there is none (or it is not
// published yet).  The key is read again after the value: an entry removed (and maybe reused)
// meanwhile is not taken; one re-inserted for the same page carries a token of the same
// page, which is as good.
__device__ __forceinline__ uint64_t sh_token(const Dev &d, uint64_t page) {
  uint64_t key = page + 1;
  uint64_t base = (uint64_t)sh_bucket(d, page) * 4;
  for (int k = 0; k < 4; ++k) {
    if (ld_acq64(&d.sh_key[base + k]) != key) continue;
    uint64_t v = ld_acq64(&d.sh_val[base + k]);
    if (v && ld_acq64(&d.sh_key[base + k]) == key) return v - 1;
  }
  return ~0ull;
}

// ================================================================ cache (Sec. 3.4)
enum Probe { P_HIT = 0, P_BUSY = 1, P_MISS = 2 };

// Look the page up in its set.  READY/MODIFIED -> hit (case a): the reference bit is
// set and, with `pin`, the line is pinned against eviction.  BUSY -> in flight
// (case c).  Otherwise a miss.
// tags of 8 ways at once: four independent 16-byte loads from L2 (one round trip);
// every 8-byte tag is read as one access
__device__ __forceinline__ void ld_tags8(const unsigned long long *p, uint64_t t[8]) {
#pragma unroll
  for (int k = 0; k < 4; ++k)
    asm volatile("ld.global.cg.v2.u64 {%0,%1}, [%2];" : "=l"(t[2 * k]), "=l"(t[2 * k + 1]) : "l"(p + 2 * k) : "memory");
}

// The way of an 8-way tag copy that holds `page` READY or MODIFIED (its tag in t), or
// -1; unrolled, so the copy stays in registers.
__device__ __forceinline__ int match_ready8(const uint64_t pre[8], uint64_t page, uint64_t &t) {
  int w = -1;
#pragma unroll
  for (int k = 7; k >= 0; --k) {
    uint64_t st = tag_state(pre[k]);
    if ((st == ST_READY || st == ST_MODIFIED) && tag_page(pre[k]) == page) {
      w = k;
      t = pre[k];
    }
  }
  return w;
}

__device__ __forceinline__ int cache_probe(const Dev &d, uint64_t page, bool pin, uint32_t &line) {
  uint64_t base = (uint64_t)set_of(page, d.sets) * d.ways;
  uint64_t t = 0;
  int wsel = -1;
  if (d.ways == 8) {  // sets of 8 ways are 64-byte aligned: read them at once
    uint64_t pre[8];
    ld_tags8(&d.tag[base], pre);
#pragma unroll
    for (int k = 7; k >= 0; --k)
      if (tag_state(pre[k]) != ST_INVALID && tag_page(pre[k]) == page) {
        wsel = k;
        t = pre[k];
      }
  } else {
    for (uint32_t k = 0; k < d.ways && wsel < 0; ++k) {
      uint64_t tk = ld_rlx64(&d.tag[base + k]);
      if (tag_state(tk) != ST_INVALID && tag_page(tk) == page) {
        wsel = (int)k;
        t = tk;
      }
    }
  }
  if (wsel >= 0) {
    const uint32_t w = (uint32_t)wsel;
    uint64_t st = tag_state(t);
    line = (uint32_t)(base + w);
    if (st == ST_BUSY) return P_BUSY;
    if (!pin) {
      if (!(t & TAG_REF)) atomicOr(&d.tag[base + w], TAG_REF);
      return P_HIT;
    }
    uint64_t old = atom_add_acq(&d.tag[base + w], PIN1);  // line data is read after the pin
    uint64_t ost = tag_state(old);
    if (tag_page(old) == page && (ost == ST_READY || ost == ST_MODIFIED)) {
      if (!(old & TAG_REF)) atomicOr(&d.tag[base + w], TAG_REF);
      return P_HIT;
    }
    atomicAdd(&d.tag[base + w], (unsigned long long)(-(int64_t)PIN1));
    return ost == ST_BUSY && tag_page(old) == page ? P_BUSY : P_MISS;
  }
  return P_MISS;
}

__device__ __forceinline__ void cache_unpin(const Dev &d, uint32_t line) {
  atomicAdd(&d.tag[line], (unsigned long long)(-(int64_t)PIN1));
}

// Put back a victim we claimed but could not use (keeps transient pin bits of others).
__device__ __forceinline__ void cache_unclaim(const Dev &d, uint32_t line, uint64_t old_tag) {
  uint64_t cur = ld_rlx64(&d.tag[line]);
  for (int i = 0; i < 64; ++i) {
    uint64_t want = (old_tag & ~PIN_MASK) | (cur & PIN_MASK);
    uint64_t got = atomicCAS(&d.tag[line], (unsigned long long)cur, (unsigned long long)want);
    if (got == cur) return;
    cur = got;
  }
}

enum Miss { M_ISSUED = 0, M_HIT = 1, M_BUSY = 2, M_RETRY = 3 };

struct Issued {
  uint32_t q, slot, ticket;  // the command to ring (the read, when there is one)
  int code;  // 1 fill, 2 evict READY, 3 write-back MODIFIED
};

// One thread rings queue q until its command (slot, ticket) has left UPDATED (the
// doorbell-lock holder never needs a cache line, so this wait cannot close a cycle);
// false after the context's wait bound.
static __device__ __noinline__ bool lane_ring(const Dev &d, uint32_t q, uint32_t slot, uint32_t ticket) {
  uint64_t deadline = gtimer() + d.timeout_ns;
  uint32_t ns = 32;
  while (!sq_attempt_db(d, q, slot, ticket)) {
    if (gtimer() > deadline) {
      set_error(d, -110);
      return false;
    }
    backoff(ns);
  }
  return true;
}

// The rare miss whose MODIFIED victim lives on another device than the page that
// replaces it: the write-back takes a demand slot of its device, the read a slot of the
// page's device.  If the read's slot cannot be had, the write-back's slot is spent on a
// no-op command (a reserved slot must be committed) and the miss is retried holding
// nothing.  The write-back is rung here; the read is left to the caller in `is`.
// Out of line, so that the common miss path stays small.
static __device__ __noinline__ int cache_miss_split(const Dev &d, uint64_t page, uint32_t q0, uint32_t line,
                                                    Issued &is, uint64_t old, int64_t sh, int64_t sh_wb, bool pf) {
  uint32_t wq = 0, wslot = 0, wticket = 0, q = 0, slot = 0, ticket = 0;
  if (!sq_reserve_dev(d, q0, dev_of_page(d, tag_page(old)), 1, wq, wslot, wticket, false)) {
    cache_unclaim(d, line, old);
    sh_remove(d, (uint64_t)sh_wb);
    sh_remove(d, (uint64_t)sh);
    return M_RETRY;
  }
  if (!sq_reserve_dev(d, q0, dev_of_page(d, page), 1, q, slot, ticket, pf)) {
    sq_commit(d, wq, wslot, wticket, OP_FLUSH, 0, 0, ctx_make(CTX_NOP, 0, 0));
    cache_unclaim(d, line, old);
    sh_remove(d, (uint64_t)sh_wb);
    sh_remove(d, (uint64_t)sh);
    lane_ring(d, wq, wslot, wticket);
    return M_RETRY;
  }
  atomicAdd(stat_ptr(d, S_EVICTIONS), 1ull);
  uint8_t *stg = d.staging + ((uint64_t)wq * d.depth + wslot) * kPage;
  lane_copy_page(stg, line_ptr(d, line));
  fence_ar();
  sq_commit(d, wq, wslot, wticket, OP_WRITE, (uint64_t)stg, tag_page(old), ctx_make(CTX_WB, (uint32_t)sh_wb, 0));
  atomicAdd(stat_ptr(d, S_WRITEBACKS), 1ull);
  lane_ring(d, wq, wslot, wticket);
  st_rlx64(&d.sh_val[sh], (((uint64_t)q << 48) | ((uint64_t)slot << 32) | ticket) + 1);
  sq_commit(d, q, slot, ticket, OP_READ, (uint64_t)line_ptr(d, line), page, ctx_make(CTX_FILL, (uint32_t)sh, line));
  atomicAdd(stat_ptr(d, S_MISSES), 1ull);
  is.q = q;
  is.slot = slot;
  is.ticket = ticket;
  is.code = 3;
  return M_ISSUED;
}

// Cases (b) and (d) for one thread: take ownership of the page's miss in the share
// table, pick a way (lowest INVALID way, else the clock: a set reference bit is
// cleared and the hand moves on, the first unpinned, unreferenced READY or MODIFIED
// way is the victim; BUSY, pinned and write-back-pending ways are skipped), reserve
// queue slots, write back a MODIFIED victim from a staging copy and issue the read.
// Nothing here waits: on any shortage every claim is undone and M_RETRY returned.
//
// fill=false (writes of whole pages): the caller already owns the page's share entry
// `sh_own`; the way is claimed BUSY and returned without a read, the caller writes the
// line and publishes it.  A MODIFIED victim is still written back first.
// Victim search of a miss in `set` (Sec. 3.4 cases (b) and (d)): the lowest way with
// an INVALID, unpinned tag, else the clock sweep from the set's hand (a way whose
// reference bit is set has it cleared and is passed; BUSY, pinned and written-back
// ways are passed; under FIFO no bit is looked at).  Each step of the hand is a
// fetch-and-add, so misses racing in one set sweep different ways.  The chosen way is
// claimed by compare-and-swap from the tag that was read, as BUSY for the new page
// (`claimed`).  Returns the way (old = its tag before, 0 when it was INVALID; sh_wb =
// the Share Table entry of the write-back of a MODIFIED victim) or -1.  Kept out of
// line: the miss path's registers stay out of the callers' loops.
static __device__ __noinline__ int64_t pick_victim(const Dev &d, uint32_t set, uint64_t claimed, uint64_t &old,
                                                   int64_t &sh_wb) {
  const uint32_t ways = d.ways;
  const uint64_t base = (uint64_t)set * ways;
  for (uint32_t w = 0; w < ways; ++w) {
    uint64_t t = ld_rlx64(&d.tag[base + w]);
    if (t == 0 && atomicCAS(&d.tag[base + w], 0ull, (unsigned long long)claimed) == 0ull) {
      old = 0;
      return w;
    }
  }
  for (uint32_t step = 0; step < 2 * ways + 1; ++step) {
    uint32_t w = atomicAdd(&d.hand[set], 1u) % ways;
    uint64_t t = ld_rlx64(&d.tag[base + w]);
    uint64_t st = tag_state(t);
    if (st == ST_INVALID) {
      if ((t & PIN_MASK) == 0 && atomicCAS(&d.tag[base + w], (unsigned long long)t, (unsigned long long)claimed) == t) {
        old = 0;
        return w;
      }
      continue;
    }
    if (st == ST_BUSY || (t & (PIN_MASK | TAG_WB))) continue;
    if (d.policy == kPolicyClock && (t & TAG_REF)) {
      atomicAnd(&d.tag[base + w], ~TAG_REF);
      continue;
    }
    if (st == ST_MODIFIED) {
      sh_wb = sh_insert(d, tag_page(t), SH_WRITE);
      if (sh_wb < 0) continue;
    }
    if (atomicCAS(&d.tag[base + w], (unsigned long long)t, (unsigned long long)claimed) == t) {
      old = t;
      return w;
    }
    if (sh_wb >= 0) {
      sh_remove(d, (uint64_t)sh_wb);
      sh_wb = -1;
    }
  }
  return -1;
}

static __device__ int cache_miss(const Dev &d, uint64_t page, uint32_t q0, uint32_t &line, Issued &is,
                          bool fill = true, int64_t sh_own = -1, bool pf = false) {
  int64_t sh = sh_own;
  if (fill) {
    sh = sh_insert(d, page, SH_FILL);
    if (sh < 0) {
      atomicAdd(stat_ptr(d, S_SHARE_RETRIES), 1ull);
      return M_RETRY;
    }
  }
  int pr = cache_probe(d, page, false, line);
  if (pr != P_MISS) {
    if (fill) sh_remove(d, (uint64_t)sh);
    return pr == P_HIT ? M_HIT : M_BUSY;
  }
  uint32_t set = set_of(page, d.sets);
  uint64_t base = (uint64_t)set * d.ways;
  uint64_t old = 0;
  int64_t sh_wb = -1;
  int64_t victim = pick_victim(d, set, tag_make(page, ST_BUSY, true), old, sh_wb);
  if (victim < 0) {
    if (fill) sh_remove(d, (uint64_t)sh);
    atomicAdd(stat_ptr(d, S_EAGAIN), 1ull);
    return M_RETRY;
  }
  line = (uint32_t)(base + victim);
  bool wb = tag_state(old) == ST_MODIFIED;
  if (wb && fill && d.ndev > 1 && dev_of_page(d, tag_page(old)) != dev_of_page(d, page))
    return cache_miss_split(d, page, q0, line, is, old, sh, sh_wb, pf);
  // a write-back and its refill take two consecutive slots of one queue of their
  // device, reserved together (a write-back rides in the demand class: a fill waits
  // behind it)
  uint32_t q = 0, slot = 0, ticket = 0;
  uint32_t nslots = (wb ? 1u : 0u) + (fill ? 1u : 0u);
  if (nslots && !sq_reserve_dev(d, q0, dev_of_page(d, wb ? tag_page(old) : page), nslots, q, slot, ticket,
                                pf && !wb)) {
    cache_unclaim(d, line, old);
    if (wb) sh_remove(d, (uint64_t)sh_wb);
    if (fill) sh_remove(d, (uint64_t)sh);
    return M_RETRY;
  }
  is.q = q;
  is.slot = slot;
  is.ticket = ticket;
  is.code = wb ? 3 : (old ? 2 : 1);
  if (old) atomicAdd(stat_ptr(d, S_EVICTIONS), 1ull);
  if (wb) {
    uint8_t *stg = d.staging + ((uint64_t)q * d.depth + slot) * kPage;
    lane_copy_page(stg, line_ptr(d, line));
    fence_ar();
    sq_commit(d, q, slot, ticket, OP_WRITE, (uint64_t)stg, tag_page(old),
              ctx_make(CTX_WB, (uint32_t)sh_wb, 0));
    atomicAdd(stat_ptr(d, S_WRITEBACKS), 1ull);
    if (!fill) return M_ISSUED;  // the write-back is the command to ring
    slot = (slot + 1) & d.dmask;
    ticket += 1;
  }
  if (!fill) {
    is.q = 0xFFFFFFFFu;  // nothing to ring
    return M_ISSUED;
  }
  // the read's token + 1 (0 = none yet), for threads that find the page in flight
  // (Sec. 3.4 case (c)); the commit's release publishes it
  st_rlx64(&d.sh_val[sh], (((uint64_t)q << 48) | ((uint64_t)slot << 32) | ticket) + 1);
  sq_commit(d, q, slot, ticket, OP_READ, (uint64_t)line_ptr(d, line), page,
            ctx_make(CTX_FILL, (uint32_t)sh, line));
  atomicAdd(stat_ptr(d, S_MISSES), 1ull);
  is.slot = slot;
  is.ticket = ticket;
  return M_ISSUED;
}

__device__ __forceinline__ uint64_t make_token(uint32_t q, uint32_t slot, uint32_t ticket) {
  return ((uint64_t)q << 48) | ((uint64_t)slot << 32) | ticket;
}

// ---------------------------------------------------------------- warp-level requests
// Sec. 3.3.2 two-level coalescing: lanes asking for the same page are matched with
// __match_any_sync and only the lowest lane of each group goes to the cache.
//
// warp_request: every lane with `want` names a page.  Leaders probe; misses are issued
// (one doorbell per queue per warp).  With wait=false this is a prefetch: the call
// returns once every page is READY, in flight or could not be started.  With
// wait=true it returns once every page is READY (no pins are held while waiting).
// Returns false on timeout/abort.  `tok` (leaders) receives the token of the read the
// lane itself issued, AGILE_TOKEN_HIT otherwise.
// `outcome` (optional) receives, in every lane, bit 0: this call sent a read to the
// device (a page READY or already in flight adds nothing); bit 1: some hint was
// dropped because the device is saturated.
// `pf`: the pages are requested ahead of need (prefetch queues, served after demand).
// `hint`: a speculative request of an application's lookahead, dropped (no retry) when
// its first queue is crowded or no queue has room -- the device is saturated.
static __device__ bool warp_request(const Dev &d, bool want, uint64_t page, uint32_t q0, bool wait,
                             uint64_t deadline, uint64_t *tok = nullptr, int *code = nullptr,
                             uint32_t *outcome = nullptr, bool pf = false, bool hint = false) {
  unsigned grp = __match_any_sync(kFull, want ? page : ~0ull);
  int lead_lane = __ffs(grp) - 1;
  bool leader = want && lead_lane == (int)lane_id();
  stat_warp(d, S_WARP_COALESCED, (want && !leader) ? 1u : 0u);
  bool need = leader;
  uint32_t line = 0;
  bool ok = true;
  bool first = true;
  uint32_t ns = 64;
  uint32_t retries = 0;
  if (tok && leader) *tok = ~0ull;
  if (code && leader) *code = 0;
  bool dropped = false, sent = false;
  while (__any_sync(kFull, need)) {
    bool issued = false, ring = false;
    Issued is{};
    if (need) {
      int pr = cache_probe(d, page, false, line);
      if (pr == P_HIT) {
        need = false;
        if (first) atomicAdd(stat_ptr(d, S_HITS), 1ull);
      } else if (pr == P_BUSY) {
        if (first) atomicAdd(stat_ptr(d, S_BUSY_HITS), 1ull);
        if (!wait) need = false;
      } else if (hint && !wait && sq_crowded(d, q0, dev_of_page(d, page), pf)) {
        need = false;  // the device is saturated: drop the hint
        dropped = true;
      } else {
        int m = cache_miss(d, page, q0, line, is, true, -1, pf);
        ring = m == M_ISSUED;
        if (m == M_ISSUED) {
          issued = true;
          sent = true;
          if (tok) *tok = make_token(is.q, is.slot, is.ticket);
          if (code) *code = is.code;
          if (!wait) need = false;
        } else if (m == M_HIT) {
          need = false;
        } else if (m == M_BUSY) {
          if (!wait) need = false;
        } else if (!wait && (hint || ++retries >= 4)) {
          need = false;  // a prefetch is a hint: give up when nothing can be evicted now
          if (hint) dropped = true;
        }
      }
    }
    first = false;
    if (!warp_ring(d, ring, is.q, is.slot, is.ticket, deadline)) ok = false;
    if (__any_sync(kFull, need)) {
      if (need) {
        if (gtimer() > deadline || aborted(d)) {
          set_error(d, -110);
          need = false;
          ok = false;
        } else {
          // wait for the in-flight line without holding anything, then re-probe
          // (short sleeps: a fill completes within microseconds)
          uint64_t t = ld_acq64(&d.tag[line]);
          if (tag_page(t) == page && tag_state(t) == ST_BUSY) backoff(ns, 512);
          else if (!issued) backoff(ns, 512);
        }
      }
    }
  }
  if (outcome) *outcome = (__any_sync(kFull, sent) ? 1u : 0u) | (__any_sync(kFull, dropped) ? 2u : 0u);
  return __all_sync(kFull, ok);
}

// Warp-cooperative probe of one page (uniform across the warp): lane w < ways loads
// the tag of way w, so the whole set is read in one round trip; on a READY/MODIFIED
// match the matching lane pins the line.  Same outcome as cache_probe(pin=true).
__device__ __forceinline__ int warp_probe_pin(const Dev &d, uint64_t page, uint32_t &line) {
  unsigned l = lane_id();
  uint64_t base = (uint64_t)set_of(page, d.sets) * d.ways;
  uint64_t t = l < d.ways ? ld_rlx64(&d.tag[base + l]) : 0;
  bool match = l < d.ways && tag_state(t) != ST_INVALID && tag_page(t) == page;
  unsigned m = __ballot_sync(kFull, match);
  if (!m) return P_MISS;
  int w = __ffs(m) - 1;
  line = (uint32_t)(base + w);
  int pr = P_MISS;
  if ((int)l == w) {
    if (tag_state(t) == ST_BUSY) {
      pr = P_BUSY;
    } else {
      uint64_t old = atom_add_acq(&d.tag[line], PIN1);  // line data is read after the pin
      uint64_t ost = tag_state(old);
      if (tag_page(old) == page && (ost == ST_READY || ost == ST_MODIFIED)) {
        if (!(old & TAG_REF)) atomicOr(&d.tag[line], TAG_REF);
        pr = P_HIT;
      } else {
        atomicAdd(&d.tag[line], (unsigned long long)(-(int64_t)PIN1));
        pr = (ost == ST_BUSY && tag_page(old) == page) ? P_BUSY : P_MISS;
      }
    }
  }
  return __shfl_sync(kFull, pr, w);
}

// The warp needs one page pinned (uniform `page`): probe with a pin; on a miss the warp
// issues and waits with nothing pinned, then probes again.  Returns the line in every
// lane, or false on timeout/abort.  The caller unpins it (one unpin per pin).
// warp_request as one out-of-line copy: for applications whose code is large (many call
// sites of the miss path next to the service code), one shared copy keeps their hot
// loops small (fewer spills, fewer instruction-cache misses); a call costs little next
// to the round trips of a request
static __device__ __noinline__ bool warp_request_call(const Dev &d, bool want, uint64_t page, uint32_t q0,
                                                      bool wait, uint64_t deadline, bool pf = false) {
  return warp_request(d, want, page, q0, wait, deadline, nullptr, nullptr, nullptr, pf);
}

template <bool kCall = false>
static __device__ bool warp_pin_page(const Dev &d, uint64_t page, uint32_t q0, uint64_t deadline,
                              uint32_t &line_out) {
  for (int round = 0;; ++round) {
    uint32_t line = 0;
    int pr = warp_probe_pin(d, page, line);
    if (pr == P_HIT) {
      line_out = line;
      if (lane_id() == 0 && round == 0) atomicAdd(stat_ptr(d, S_HITS), 1ull);
      return true;
    }
    if (!(kCall ? warp_request_call(d, lane_id() == 0, page, q0, true, deadline)
                : warp_request(d, lane_id() == 0, page, q0, true, deadline)))
      return false;
    if (aborted(d)) return false;
    if (gtimer() > deadline) {
      if (lane_id() == 0) set_error(d, -110);
      return false;
    }
  }
}

// Asynchronous requests ahead of use pay a probe per page even when they have nothing
// to do: every page already resident or in flight, or the device saturated (the hints
// are dropped).
// A warp whose lookahead keeps finding nothing to do requests less often: after such a
// round it skips the next `span` rounds (span 1, 3, 7, ... up to 63).  A round that
// sends work to the device brings it back to every round, and so does a miss met later
// by the warp's own gather -- unless the last round was dropped for saturation (the
// gather misses then because the hints were dropped, and more lookahead would only be
// dropped again).  Skipped pages are fetched when used, as in synchronous mode.
struct Backoff {
  uint32_t skip = 0, span = 0;
  bool sat = false;
  __device__ __forceinline__ bool take() {  // true: request this round
    if (skip) {
      --skip;
      return false;
    }
    return true;
  }
  // outcome of warp_request: bit 0 work sent to the device, bit 1 hints dropped
  __device__ __forceinline__ void result(uint32_t outcome) {
    if (outcome & 1u) {
      span = 0;
      sat = false;
    } else {
      span = span < 63 ? 2 * span + 1 : 63;
      skip = span;
      sat = (outcome & 2u) != 0;
    }
  }
  __device__ __forceinline__ void missed() {
    if (!sat) skip = span = 0;
  }
};

// what an application warp knows about its launch
struct AppCtx {
  uint32_t warp;     // app warp index in [0, n_warps)
  uint32_t n_warps;  // app warps in the grid
  uint32_t q0;       // this lane's home queue (Sec. 3.3.1: by thread index)
  uint64_t deadline;
};

// ================================================================ user kernel API
// The device side of Listing 1 (Sec. 3.5) for kernels that run inside a library launch
// (agile_device.cuh launches them): a warp's lanes issue reads, continue with other
// work, test or wait for each read's token, then copy the page.  No call here waits
// while it holds a cache line or a queue slot.

// Token state (agile_test): 0 done, AGILE_EIO done with an error, 1 still in flight.
__device__ __forceinline__ int token_state(const Dev &d, uint64_t tok) {
  if (tok == ~0ull) return 0;
  uint32_t q = (uint32_t)(tok >> 48), slot = (uint32_t)(tok >> 32) & 0xFFFFu, ticket = (uint32_t)tok;
  if (q >= d.Q || slot >= d.depth) return -22;
  uint64_t w = ld_acq64(&d.cmpl[(uint64_t)q * d.depth + slot]);
  uint32_t wt = (uint32_t)(w >> 32);
  if (!(w & 1) || (int32_t)(wt - ticket) < 0) return 1;
  // a later command of the slot has completed: this one completed before it
  if (wt == ticket && ((w >> 1) & 0x7FFF) != 0) return -5;
  return 0;
}

// asyncRead, issue part (warp-collective): lanes with `want` request `page`.  The
// pages of equal requests are merged (the lowest lane goes to the cache); nothing waits
// for data.  Returns the lane's token: AGILE_TOKEN_HIT (~0) when the page was READY,
// else the token of the read that fills it -- issued here, or found in flight (the
// share table names it).  ~0 too after a deadline or an abort (the data is then fetched
// by agile_copy_page).
static __device__ uint64_t api_issue_read(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  unsigned grp = __match_any_sync(kFull, want ? page : ~0ull);
  int lead = __ffs(grp) - 1;
  bool leader = want && lead == (int)lane_id();
  uint64_t tok = ~0ull;
  bool need = leader;
  uint32_t ns = 64;
  while (__any_sync(kFull, need)) {
    bool ring = false;
    Issued is{};
    if (need) {
      uint32_t line = 0;
      int pr = cache_probe(d, page, false, line);
      if (pr == P_HIT) {
        need = false;
      } else if (pr == P_BUSY) {
        uint64_t t = sh_token(d, page);
        if (t != ~0ull) {
          tok = t;
          need = false;
        }
      } else {
        int m = cache_miss(d, page, a.q0, line, is);
        ring = m == M_ISSUED;
        if (m == M_ISSUED) {
          tok = make_token(is.q, is.slot, is.ticket);
          need = false;
        } else if (m == M_HIT) {
          need = false;
        }
      }
      if (need && (gtimer() > a.deadline || aborted(d))) need = false;
    }
    warp_ring(d, ring, is.q, is.slot, is.ticket, a.deadline);
    if (__any_sync(kFull, need)) backoff(ns, 1024);
  }
  tok = __shfl_sync(kFull, tok, lead & 31);
  return want ? tok : ~0ull;
}

// agile_test: non-blocking ("continue" while it is 1)
__device__ __forceinline__ int api_test(const Dev &d, uint64_t tok) { return token_state(d, tok); }

// agile_wait: the transaction barrier of Sec. 3.2.1 for one token, bounded: 0 done,
// AGILE_EIO done with an error, AGILE_ETIMEDOUT when `deadline_ns` (%globaltimer) passes
// first.  The caller holds no pin while it waits (the library never does); a timeout
// is returned to the caller and recorded nowhere else.
__device__ __forceinline__ int api_wait(const Dev &d, uint64_t tok, uint64_t deadline_ns) {
  uint32_t ns = 64;
  for (;;) {
    int st = token_state(d, tok);
    if (st != 1) return st;
    if (gtimer() > deadline_ns) return -110;
    backoff(ns, 1024);
  }
}

// Copy a page (uniform across the warp) from its cache line into dst (4096 bytes,
// 16-byte aligned), with the line pinned for the copy only; a page evicted since its
// read completed is requested again.  False on a timeout of the launch.
static __device__ bool api_copy_page(const Dev &d, const AppCtx &a, uint64_t page, void *dst) {
  uint32_t line;
  if (!warp_pin_page<true>(d, page, a.q0, a.deadline, line)) return false;
  warp_copy_page(dst, line_ptr(d, line));
  __syncwarp();
  if (lane_id() == 0) cache_unpin(d, line);
  return true;
}

// get_row (the synchronous read of part of a page, warp-collective, uniform arguments):
// copy bytes [off, off + nbytes) of `page` to dst, the line pinned for the copy only.
// off, nbytes and dst must be 4-byte aligned and off + nbytes at most one page; else
// AGILE_EINVAL is recorded and false returned.  False also if the launch timed out.
static __device__ bool api_get_row(const Dev &d, const AppCtx &a, uint64_t page, uint32_t off, uint32_t nbytes,
                                   void *dst) {
  if (((off | nbytes | (uint32_t)(uintptr_t)dst) & 3u) || nbytes > kPage || off > kPage - nbytes) {
    if (lane_id() == 0) set_error(d, AGILE_EINVAL);
    return false;
  }
  uint32_t line;
  if (!warp_pin_page<true>(d, page, a.q0, a.deadline, line)) return false;
  const uint8_t *src = line_ptr(d, line) + off;
  int32_t *o = (int32_t *)dst;
  for (uint32_t i = lane_id(); i < nbytes / 4; i += 32) o[i] = ld_cg_s32(src + 4 * i);
  __syncwarp();
  if (lane_id() == 0) cache_unpin(d, line);
  return true;
}

// prefetch (Listing 1 Method-1): start filling the pages of the lanes with `want`.
static __device__ bool api_prefetch(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  return warp_request_call(d, want, page, a.q0, false, a.deadline, true);
}

// Add rows [j0, j0 + k) (lane j holds row j's line `line_j` and byte offset `off`) to acc
// in increasing j, with several rows' loads in flight at once.
template <int MF4>
__device__ __forceinline__ void sum_rows(const Dev &d, uint32_t j0, uint32_t k, uint32_t line, uint32_t off,
                                         uint32_t nf4, float4 (&acc)[MF4]) {
  unsigned l = lane_id();
  constexpr int RB = MF4 >= 8 ? 1 : 8 / MF4;  // rows in flight: RB * MF4 float4 per lane
  for (uint32_t jb = 0; jb < k; jb += RB) {
    float4 v[RB][MF4];
#pragma unroll
    for (int jj = 0; jj < RB; ++jj) {
      uint32_t j = j0 + jb + jj;
      uint32_t lj = __shfl_sync(kFull, line, j & 31);
      uint32_t oj = __shfl_sync(kFull, off, j & 31);
      const uint8_t *rowp = line_ptr(d, lj) + oj;
#pragma unroll
      for (int c = 0; c < MF4; ++c) {
        uint32_t col = l + 32 * c;
        v[jj][c] = (jb + jj < k && col < nf4) ? ld_cg_f4(rowp + 16 * col) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int jj = 0; jj < RB; ++jj) {
      if (jb + jj < k) {
#pragma unroll
        for (int c = 0; c < MF4; ++c) {
          acc[c].x = __fadd_rn(acc[c].x, v[jj][c].x);
          acc[c].y = __fadd_rn(acc[c].y, v[jj][c].y);
          acc[c].z = __fadd_rn(acc[c].z, v[jj][c].z);
          acc[c].w = __fadd_rn(acc[c].w, v[jj][c].w);
        }
      }
    }
  }
}

// Sum-pool rows begin..cnt-1 into acc, added in increasing lane order (lane j holds row
// j's page `pg` and byte offset `off`).  Lane l adds the
// float4 columns l, l+32, ... (MF4 of them, dim/4 in total).
// Each round pins, in parallel, the distinct pages of the rows not yet added (one
// probe per distinct page), adds the longest run of rows from the next one whose pages
// are all pinned, and lets every pin go.  When the next row's page is not READY, the
// warp requests all missing pages without waiting, then waits for and pins that one
// page (nothing else pinned meanwhile, Sec. 2.3.2) and adds its row: every round adds
// at least one row, whatever the set conflicts among the rows.
// `missed` (optional) is set in every lane when some page had to be requested.
template <int MF4>
static __device__ bool gather_sum(const Dev &d, const AppCtx &a, uint32_t begin, uint32_t cnt, uint64_t pg, uint32_t off,
                           uint32_t nf4, float4 (&acc)[MF4], bool *missed = nullptr) {
  unsigned l = lane_id();
  uint32_t j0 = begin;
  bool first = true;
  while (j0 < cnt) {
    bool act = l >= j0 && l < cnt;
    unsigned grp = __match_any_sync(kFull, act ? pg : ~0ull);
    int lead_lane = __ffs(grp) - 1;
    bool leader = act && lead_lane == (int)l;
    if (first) stat_warp(d, S_WARP_COALESCED, (act && !leader) ? 1u : 0u);
    uint32_t line = 0;
    int pr = P_MISS;
    if (leader) pr = cache_probe(d, pg, true, line);
    if (first) stat_warp(d, S_HITS, (leader && pr == P_HIT) ? 1u : 0u);
    first = false;
    bool lhit = __shfl_sync(kFull, (int)(pr == P_HIT), lead_lane & 31) != 0;
    uint32_t myline = __shfl_sync(kFull, line, lead_lane & 31);
    unsigned hm = __ballot_sync(kFull, act && lhit);
    unsigned run = ~(hm >> j0);
    uint32_t k = run ? (uint32_t)(__ffs(run) - 1) : 32u;
    k = min(k, cnt - j0);
    if (k) sum_rows<MF4>(d, j0, k, myline, off, nf4, acc);
    __syncwarp();
    if (leader && pr == P_HIT) cache_unpin(d, line);
    if (k) {
      j0 += k;
      continue;
    }
    // row j0's page is missing: request every missing page, then wait for row j0's
    if (missed) *missed = true;
    if (!warp_request(d, leader && pr != P_HIT, pg, a.q0, false, a.deadline)) return false;
    uint64_t pj = __shfl_sync(kFull, pg, j0 & 31);
    uint32_t lj;
    if (!warp_pin_page(d, pj, a.q0, a.deadline, lj)) return false;
    uint32_t lines = __shfl_sync(kFull, myline, 0);  // placeholder value for other lanes
    lines = (l == j0) ? lj : lines;
    sum_rows<MF4>(d, j0, 1, lines, off, nf4, acc);
    __syncwarp();
    if (l == 0) cache_unpin(d, lj);
    j0 += 1;
  }
  return true;
}


// ================================================================ completion side
// Release what a completed command held (Sec. 3.2.1): the line becomes READY (or
// INVALID on an error), the share-table entry is removed, the transaction barrier
// (completion word) is set, the slot returns to EMPTY and the in-flight count drops.
__device__ __forceinline__ void complete_command(const Dev &d, uint32_t q, uint32_t cid, uint32_t status) {
  uint64_t i = (uint64_t)q * d.depth + cid;
  uint64_t ctx = ld_rlx64(&d.cmd_ctx[i]);
  uint64_t st = ld_rlx64(&d.sqe_state[i]);
  uint64_t ticket = st >> 2;
  uint64_t kind = ctx >> 60;
  uint32_t sh = (uint32_t)(ctx >> 32) & 0x0FFFFFFFu;
  uint32_t idx = (uint32_t)ctx;
  fence_ar();
  if (kind == CTX_FILL) {
    if (status == 0) {
      atomicAdd(&d.tag[idx], 1ull);  // BUSY (1) -> READY (2)
    } else {
      atomicAnd(&d.tag[idx], PIN_MASK);  // back to INVALID
    }
    sh_remove(d, sh);
  } else if (kind == CTX_WB) {
    if (idx) atomicAnd(&d.tag[idx - 1], ~TAG_WB);  // flush write-back from the line itself
    sh_remove(d, sh);
  } else if (kind == CTX_BUF) {
    sh_remove(d, sh);
  }
  if (status) atomicAdd(stat_ptr(d, S_IO_ERRORS), 1ull);
  st_rel64(&d.cmpl[i], ((ticket & 0xFFFFFFFFull) << 32) | ((uint64_t)(status & 0x7FFF) << 1) | 1ull);
  st_rel64(&d.sqe_state[i], (ticket << 2) | SQE_EMPTY);
  atomicAdd(&d.sq_resv[q], (unsigned long long)(-(int64_t)(1ull << 32)));
}

// Alg. 1, warp-centric CQ polling of queue q: lane l checks entry offset+l of the
// current 32-entry window against the expected phase; the mask accumulates found
// entries (they may arrive in any order); a full mask advances the head and rings the
// CQ doorbell.  The CQ has twice as many entries as the SQ, so with at most depth-1
// commands outstanding and at most 31 consumed entries in the open window it never
// fills (the device never has to wait for CQ space).
static __device__ bool cq_poll(const Dev &d, uint32_t q) {
  unsigned l = lane_id();
  uint32_t *ps = &d.cq_poll[q * 4];
  uint32_t offset = ld_rlx32(&ps[0]), mask = ld_rlx32(&ps[1]), phase = ld_rlx32(&ps[2]);
  uint32_t found = 0, windows = 0;
  for (int win = 0; win < 4; ++win) {
    bool valid = false;
    if (!((mask >> l) & 1u)) {
      Cqe *c = &d.cq[(uint64_t)q * d.cq_size + offset + l];
      uint32_t w3 = ld_acq32(&c->dw[3]);
      if (((w3 >> 16) & 1u) == phase) {
        complete_command(d, q, w3 & 0xFFFFu, w3 >> 17);
        valid = true;
      }
    }
    unsigned b = __ballot_sync(kFull, valid);
    found += __popc(b);
    mask |= b;
    if (mask != kFull) break;
    mask = 0;
    offset += 32;
    if (offset >= d.cq_size) {
      offset = 0;
      phase ^= 1u;
    }
    ++windows;
    __syncwarp();
    if (l == 0) {
      fence_ar();
      st_rel32(&d.cq_db[q], offset);
    }
  }
  __syncwarp();
  if (l == 0) {
    st_rlx32(&ps[0], offset);
    st_rlx32(&ps[1], mask);
    st_rlx32(&ps[2], phase);
    if (found) atomicAdd(stat_ptr(d, S_CQES), (unsigned long long)found);
    if (windows) atomicAdd(stat_ptr(d, S_CQ_DOORBELLS), (unsigned long long)windows);
  }
  __syncwarp();
  return found != 0;
}

// ================================================================ emulated device
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// The emulated NVMe device.  Every service warp is one of its engines and may serve
// any queue.  Per queue the device keeps (unwrapped counters): `fetch`, the next SQE to
// take; `seen`, how far the doorbell has been observed (commands below it carry their
// arrival time); `cqt`, the next CQ slot.  An engine takes up to kEmuBatch due commands
// in SQ order by compare-and-swap on `fetch` (a command is due once its latency has
// elapsed and the queue's throughput budget allows it), moves the pages between the
// store (pinned host memory, over the host link) and HBM, then reserves CQ slots and
// posts the CQEs {SQ head, SQ id, CID, status, phase}.  Commands of one queue complete
// in any order, as NVMe allows.
constexpr uint32_t kEmuBatch = 2;
constexpr uint64_t kEmuSlackNs = 16000;

// Returns the number of commands served, or kEmuDevFull when commands were due but
// their device was booked.  block_dev: a device this call may not book (a demand
// command of the same engine pass is waiting for it), ~0u for none.
constexpr uint32_t kEmuDevFull = 0x80000000u;
static __device__ uint32_t emu_serve(const Dev &d, uint32_t q, uint32_t block_dev = ~0u) {
  unsigned l = lane_id();
  uint32_t *es = &d.emu[q * 4];
  uint32_t f = 0, k = 0, full = 0;
  uint64_t now = gtimer();
  const uint32_t dv = d.ndev > 1 ? q % d.ndev : 0u;  // the device this queue belongs to
  const bool model = d.lat_ns || d.ns_per_page || d.ns_rd_dev || d.ns_wr_dev;
  if (l == 0 && !model) {
    // no latency model: every command the doorbell exposes is due at once.  The fetch
    // counter is read before the doorbell, so with f still current (checked by the
    // compare-and-swap) the doorbell is at most depth-1 commands ahead of it and
    // (db - f) mod depth is the exact number of unfetched commands.
    f = ld_acq32(&es[0]);
    uint32_t db = ld_acq32(&d.sq_db[q]);
    k = min((db - (f & d.dmask)) & d.dmask, kEmuBatch);
    if (k && atomicCAS(&es[0], f, f + k) != f) k = 0;
  } else if (l == 0) {
    // `seen` must be read before the doorbell: it only ever takes doorbell values read
    // earlier, so seen <= tail here and (db - seen) mod depth is the exact number of
    // newly exposed commands (never a wrapped-around difference)
    uint32_t seen = ld_acq32(&es[1]);
    uint32_t db = ld_acq32(&d.sq_db[q]);
    // stamp the arrival of commands the doorbell has newly exposed, then publish them
    uint32_t fresh = (db - (seen & d.dmask)) & d.dmask;
    if (fresh) {
      for (uint32_t i = 0; i < fresh; ++i)
        st_rlx64(&d.emu_arrival[(uint64_t)q * d.depth + ((seen + i) & d.dmask)], now);
      fence_ar();
      atomicCAS(&es[1], seen, seen + fresh);
      seen = ld_acq32(&es[1]);
    }
    f = ld_rlx32(&es[0]);
    uint32_t avail = seen - f;
    if ((int32_t)avail > 0) {
      if (avail > kEmuBatch) avail = kEmuBatch;
      while (k < avail) {
        uint64_t arr = ld_rlx64(&d.emu_arrival[(uint64_t)q * d.depth + ((f + k) & d.dmask)]);
        if (now < arr + d.lat_ns) break;
        ++k;
      }
      if (k && dv == block_dev) {
        k = 0;
        full = kEmuDevFull;
      }
      // Throughput: the batch is booked on the queue's pipe and on its device when each
      // is free (reads and writes take device time of their own).  Bookings follow each
      // other without gaps while the pipe has been idle for less than kEmuSlackNs
      // (engines poll in turns, so a pipe's next batch is picked up a little late): a
      // token bucket that may run kEmuSlackNs ahead after a pause, which moves the
      // long-run rate by less than kEmuSlackNs per pause.  Bookings of a batch that is
      // not served after all (another booking failed, or another engine took the
      // commands meanwhile) are given back.
      uint64_t qcost = d.ns_per_page * k, dcost = 0;
      bool qbooked = false, dbooked = false;
      if (k && qcost) {
        uint64_t busy = ld_rlx64(&d.emu_busy[q]);
        if (busy > now) {
          k = 0;
        } else {
          uint64_t nb = (busy + kEmuSlackNs > now ? busy : now) + qcost;
          qbooked = atomicCAS(&d.emu_busy[q], (unsigned long long)busy, (unsigned long long)nb) == busy;
          if (!qbooked) k = 0;
        }
      }
      if (k && (d.ns_rd_dev || d.ns_wr_dev)) {
        for (uint32_t i = 0; i < k; ++i) {
          uint32_t op = ld_rlx32(&d.sq[(uint64_t)q * d.depth + ((f + i) & d.dmask)].dw[0]) & 0xFFu;
          dcost += op == OP_WRITE ? d.ns_wr_dev : (op == OP_READ ? d.ns_rd_dev : 0);
        }
        uint64_t busy = ld_rlx64(&d.dev_busy[dv]);
        if (busy > now) {
          k = 0;
          full = kEmuDevFull;
        } else {
          uint64_t nb = (busy + kEmuSlackNs > now ? busy : now) + dcost;
          dbooked = atomicCAS(&d.dev_busy[dv], (unsigned long long)busy, (unsigned long long)nb) == busy;
          if (!dbooked) k = 0;
        }
      }
      if (k && atomicCAS(&es[0], f, f + k) != f) k = 0;
      if (!k) {
        if (qbooked) atomicAdd(&d.emu_busy[q], (unsigned long long)(-(int64_t)qcost));
        if (dbooked && dcost) atomicAdd(&d.dev_busy[dv], (unsigned long long)(-(int64_t)dcost));
      }
    }
  }
  k = __shfl_sync(kFull, k, 0);
  if (!k) return __shfl_sync(kFull, full, 0);
  f = __shfl_sync(kFull, f, 0);
  __syncwarp();  // lane 0's acquire of the doorbell orders the SQE reads of every lane
  // command fields: lane i < k reads SQE f+i
  uint32_t dw0 = 0, nlb = 0, status = 0;
  uint64_t prp1 = 0, slba = 0, t_commit = 0;
  bool drop = false;
  if (l < k) {
    uint64_t i = (uint64_t)q * d.depth + ((f + l) & d.dmask);
    const uint32_t *e = d.sq[i].dw;
    int4 a = ld_cg16(e), b = ld_cg16(e + 4), c = ld_cg16(e + 8), g = ld_cg16(e + 12);
    dw0 = (uint32_t)a.x;
    t_commit = (uint64_t)(uint32_t)a.z | ((uint64_t)(uint32_t)a.w << 32);
    prp1 = (uint64_t)(uint32_t)b.z | ((uint64_t)(uint32_t)b.w << 32);
    slba = (uint64_t)(uint32_t)c.z | ((uint64_t)(uint32_t)c.w << 32);
    nlb = (uint32_t)g.x & 0xFFFFu;
    uint32_t opcode = dw0 & 0xFFu;
    uint64_t nbytes = ((uint64_t)nlb + 1) * 512;
    // from here on slba is the store page of the command (block on device dv)
    slba = (d.ndev > 1 ? (slba / (kPage / 512)) * d.ndev + dv : slba / (kPage / 512));
    if (opcode != OP_FLUSH && (slba * kPage + nbytes > d.store_bytes || nbytes != kPage)) status = 0x80;
    if (d.fault_flags) {
      uint64_t h = mix64(d.seed ^ ((uint64_t)q << 40) ^ (uint64_t)(f + l));
      if ((uint32_t)(h >> 32) < d.fault_thresh) {
        if (d.fault_flags & 1u) status = 0x6;
        if (d.fault_flags & 2u) drop = true;
      }
    }
  }
  // data movement: every page of the batch has its loads in flight before any store
  int4 v[kEmuBatch][8];
  uint64_t srcs[kEmuBatch], dsts[kEmuBatch];
  bool mv[kEmuBatch];
#pragma unroll
  for (uint32_t j = 0; j < kEmuBatch; ++j) {
    uint32_t opj = __shfl_sync(kFull, dw0, j) & 0xFFu;
    uint32_t stj = __shfl_sync(kFull, status, j);
    uint64_t pj = __shfl_sync(kFull, prp1, j), sj = __shfl_sync(kFull, slba, j);
    mv[j] = j < k && stj == 0 && (opj == OP_READ || opj == OP_WRITE);
    srcs[j] = opj == OP_READ ? (uint64_t)(d.store + sj * kPage) : pj;
    dsts[j] = opj == OP_READ ? pj : (uint64_t)(d.store + sj * kPage);
    if (mv[j]) {
      const int4 *sp = (const int4 *)srcs[j];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[j][t] = ld_cg16(sp + t * 32 + l);
    }
  }
  uint32_t rd = 0, wr = 0;
#pragma unroll
  for (uint32_t j = 0; j < kEmuBatch; ++j) {
    if (mv[j]) {
      int4 *dp = (int4 *)dsts[j];
#pragma unroll
      for (int t = 0; t < 8; ++t) st_cg16(dp + t * 32 + l, v[j][t]);
      if ((__shfl_sync(kFull, dw0, j) & 0xFFu) == OP_READ) ++rd;
      else ++wr;
    }
  }
  // per-page accounting of the data moved (lane i counts command i)
  if (l < k && status == 0) {
    uint32_t opcode = dw0 & 0xFFu;
    if (opcode == OP_READ) atomicAdd(&d.pg_reads[slba], 1u);
    else if (opcode == OP_WRITE) atomicAdd(&d.pg_writes[slba], 1u);
  }
  __threadfence();
  __syncwarp();
  // completion entries
  uint32_t slot0 = 0;
  if (l == 0) slot0 = atomicAdd(&es[2], k);
  slot0 = __shfl_sync(kFull, slot0, 0);
  if (l < k) {
    uint32_t sl = slot0 + l;
    uint32_t pos = sl % d.cq_size;
    uint32_t phase = ((sl / d.cq_size) & 1u) ^ 1u;
    Cqe *c = &d.cq[(uint64_t)q * d.cq_size + pos];
    uint32_t cid = dw0 >> 16;
    if (d.trace) {
      uint32_t ti = atomicAdd(d.trace_n, 1u);
      if (ti < d.trace_cap) {
        TraceRec *tr = &d.trace[ti];
        tr->page = slba;
        tr->t_seen = model
                         ? ld_rlx64(&d.emu_arrival[(uint64_t)q * d.depth + ((f + l) & d.dmask)])
                         : 0ull;
        tr->t_start = now;
        tr->t_done = gtimer();
        tr->q = q;
        tr->cid = cid;
        tr->opcode = dw0 & 0xFFu;
        tr->status = status | (drop ? 0x10000u : 0u);
        tr->t_commit = t_commit;
      }
    }
    if (drop) {
      // the completion is lost; leave a harmless entry with the old phase
      st_rlx32(&c->dw[2], (q << 16) | ((f + l + 1) & d.dmask));
    } else {
      st_rlx32(&c->dw[0], 0u);
      st_rlx32(&c->dw[1], 0u);
      st_rlx32(&c->dw[2], (q << 16) | ((f + l + 1) & d.dmask));
      fence_ar();
      st_rel32(&c->dw[3], cid | (phase << 16) | (status << 17));
    }
  }
  if (l == 0) {
    atomicAdd(stat_ptr(d, S_COMMANDS), (unsigned long long)k);
    if (rd) atomicAdd(stat_ptr(d, S_BYTES_READ), (unsigned long long)rd * kPage);
    if (wr) atomicAdd(stat_ptr(d, S_BYTES_WRITTEN), (unsigned long long)wr * kPage);
  }
  __syncwarp();
  return k;
}

// ================================================================ engine
// One cooperative launch per library call.  Warp 0 of every CTA is a service warp:
// an engine of the emulated device for every queue, and the Alg. 1 poller of queues
// q = cta, cta + grid, ...  The other warps run the application.  No kernel of the
// library ever waits on another launch: the device, the pollers and the waiters are
// co-resident warps of one grid, and every wait is bounded by a deadline.
// `sw` of `nsw`: this engine's number among the launch's engines (rotation start).
static __device__ void service_loop(const Dev &d, uint32_t n_app, uint64_t deadline, bool poll, uint32_t sw,
                                    uint32_t nsw) {
  unsigned l = lane_id();
  uint32_t ns = 32;
  for (uint32_t iter = 0;; ++iter) {
    bool progress = false;
    // device engine: serve one queue per iteration, the first one with work found from
    // a start that rotates over the queues and differs between engines, so that every
    // queue is visited often and commands do not wait behind long scans
    // (the doorbells and fetch counters of four windows of 32 queues are read in one
    // round trip; they only select a queue, emu_serve checks them again)
    // (demand queues first: the prefetch queues are served only when no demand queue
    // has a command the device may take now; a prefetch queue does not book a device
    // that a due demand command found booked in this pass, so the device's next free
    // turn goes to the demand command)
    uint32_t block_dev = ~0u;
#pragma unroll 1
    for (uint32_t cls = 0; cls < 2 && !progress; ++cls) {
      uint32_t qsel = ~0u;
      const uint32_t base = cls ? d.Q - d.Qp : 0u, cnt = cls ? d.Qp : d.Q - d.Qp;
      if (cnt == 0) continue;
      const uint32_t r = (uint32_t)(((uint64_t)iter * nsw + sw) % cnt);
      const uint32_t windows = (cnt + 31) / 32;
      for (uint32_t w0 = 0; w0 < windows && qsel == ~0u; w0 += 4) {
        uint32_t dbv[4], fv[4];
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
          uint32_t off = (w0 + j) * 32 + l;
          dbv[j] = fv[j] = 0;
          if (off < cnt) {
            uint32_t q = base + (r + off) % cnt;
            dbv[j] = ld_rlx32(&d.sq_db[q]);
            fv[j] = ld_rlx32(&d.emu[q * 4]);
          }
        }
#pragma unroll
        for (uint32_t j = 0; j < 4; ++j) {
          uint32_t off = (w0 + j) * 32 + l;
          unsigned m = __ballot_sync(kFull, off < cnt && ((dbv[j] - (fv[j] & d.dmask)) & d.dmask) != 0);
          if (m && qsel == ~0u) qsel = base + (r + (w0 + j) * 32 + (uint32_t)(__ffs(m) - 1)) % cnt;
        }
      }
      if (qsel != ~0u) {
        uint32_t r = emu_serve(d, qsel, block_dev);
        if (r == kEmuDevFull) block_dev = d.ndev > 1 ? qsel % d.ndev : 0u;
        else if (r) progress = true;
      }
    }
    // completion side (Alg. 1) for the queues this warp polls
    if (poll)
      for (uint32_t q = sw; q < d.Q; q += nsw) progress |= cq_poll(d, q);
    if (progress) {
      ns = 32;
      continue;
    }
    uint32_t done = 0;
    if (l == 0) done = ld_acq32(&d.run->app_done);
    done = __shfl_sync(kFull, done, 0);
    if (done >= n_app) {
      bool drained = true;
      for (uint32_t q = l; q < d.Q; q += 32)
        if ((ld_acq64(&d.sq_resv[q]) >> 32) != 0) drained = false;
      if (__all_sync(kFull, drained)) break;
    }
    if (gtimer() > deadline) {
      if (l == 0) set_error(d, -110);
      break;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : 256;
  }
}

// A dedicated Alg. 1 poller of queue q: an application warp that sits out the call.
// Ends when every application warp is done and the queue has nothing in flight.
static __device__ void poller_loop(const Dev &d, uint32_t q, uint32_t n_app, uint64_t deadline) {
  unsigned l = lane_id();
  uint32_t ns = 32;
  for (;;) {
    if (cq_poll(d, q)) {
      ns = 32;
      continue;
    }
    uint32_t done = 0;
    uint64_t resv = 0;
    if (l == 0) {
      done = ld_acq32(&d.run->app_done);
      resv = ld_acq64(&d.sq_resv[q]);
    }
    done = __shfl_sync(kFull, done, 0);
    resv = __shfl_sync(kFull, resv, 0);
    if (done >= n_app && (resv >> 32) == 0) break;
    if (gtimer() > deadline) {
      if (l == 0) set_error(d, -110);
      break;
    }
    __nanosleep(ns);
    ns = ns < 256 ? ns * 2 : 256;
  }
}

// Grid barrier over the application warps only (service warps never join).
static __device__ bool app_barrier(const Dev &d, uint32_t n_app, uint64_t deadline) {
  bool ok = true;
  __syncwarp();
  if (lane_id() == 0) {
    fence_ar();
    uint32_t gen = ld_acq32(&d.run->bar_gen);
    uint32_t arrived = atomicAdd(&d.run->bar_count, 1u) + 1;
    if (arrived == n_app) {
      st_rlx32(&d.run->bar_count, 0u);
      fence_ar();
      st_rel32(&d.run->bar_gen, gen + 1);
    } else {
      uint32_t ns = 32;
      while (ld_acq32(&d.run->bar_gen) == gen) {
        if (gtimer() > deadline) {
          set_error(d, -110);
          ok = false;
          break;
        }
        __nanosleep(ns);
        ns = ns < 1024 ? ns * 2 : 1024;
      }
    }
  }
  ok = __shfl_sync(kFull, ok, 0);
  __syncwarp();
  return ok;
}


// CTAs per SM the engine is compiled for (register budget): App::kMinBlocks if the
// application asks for more occupancy, else 2
template <class App, class = void>
struct MinBlocks {
  static constexpr int value = 2;
};
template <class App>
struct MinBlocks<App, decltype((void)App::kMinBlocks, void())> {
  static constexpr int value = App::kMinBlocks;
};

template <class App>
__global__ void __launch_bounds__(kThreads, MinBlocks<App>::value) engine_kernel(Dev d, App app) {
  uint32_t warp = threadIdx.x >> 5;
  uint32_t n_app = gridDim.x * (kWarps - 1);
  uint64_t deadline = gtimer() + (d.session_ns ? d.session_ns : d.timeout_ns);
  uint32_t n_active = (d.app_active && d.app_active < n_app) ? d.app_active : n_app;
  // when at least Q application warps sit out the call, the first Q of them poll one
  // queue each, and the service warps only serve the device
  const bool pollers = n_app - n_active >= d.Q;
  if (warp == 0) {
    uint32_t idle = n_app - n_active, q_used = pollers ? d.Q : 0;
    uint32_t extra = idle > q_used ? min(idle - q_used, d.extra_engines) : 0;
    service_loop(d, n_app, deadline + d.timeout_ns, !pollers, blockIdx.x, gridDim.x + extra);
    return;
  }
  AppCtx a;
  a.warp = blockIdx.x * (kWarps - 1) + (warp - 1);
  a.n_warps = n_active;
  if (a.warp >= a.n_warps) {
    // not needed by this call: keeps the working set of the active warps in the cache.
    // The first Q such warps poll a completion queue each (when there are Q of them),
    // the next ones (up to d.extra_engines) serve the device as additional engines.
    if (lane_id() == 0) atomicAdd(&d.run->app_done, 1u);
    uint32_t idle = a.warp - a.n_warps, q_used = pollers ? d.Q : 0;
    if (idle < q_used) {
      poller_loop(d, idle, n_app, deadline + d.timeout_ns);
    } else {
      uint32_t extra = min(n_app - n_active - q_used, d.extra_engines);
      if (idle - q_used < extra)
        service_loop(d, n_app, deadline + d.timeout_ns, false, gridDim.x + (idle - q_used), gridDim.x + extra);
    }
    return;
  }
  // home queue by thread index, spread so that the lanes of a warp and the lane 0 of
  // consecutive warps all start on different queues
  a.q0 = (uint32_t)((a.warp + (uint64_t)lane_id() * ((d.Q + 31) / 32)) % d.Q);
  a.deadline = deadline;
  app.run(d, a);
  __syncwarp();
  if (lane_id() == 0) {
    fence_ar();
    atomicAdd(&d.run->app_done, 1u);
  }
}

}  // namespace agile
