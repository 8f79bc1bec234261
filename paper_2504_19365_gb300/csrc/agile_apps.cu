// Application drivers on top of the cache and queues: sum-pooled embedding bag
// (Sec. 4.4, DLRM embedding lookups) and top-down level-synchronous BFS over CSR
// (Sec. 4.5), each in a synchronous and an asynchronous mode.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>
#include <mutex>

#include "agile.h"
#include "agile_ctx.cuh"
#include "agile_dev.cuh"

using namespace agile;

namespace {

constexpr int kMaxF4 = 8;  // float4 columns per lane: dim <= 32 * 4 * 8 = 1024

template <int MF4, int MinBlocks = 2>
struct EmbApp {
  static constexpr int kMinBlocks = MinBlocks;  // CTAs per SM the kernel is compiled for
  uint64_t page0;  // first store page of the table
  uint32_t rows, dim;
  const int64_t *idx;
  const int64_t *off;
  uint32_t n_bags;
  float *out;
  uint32_t mode;
  // no request ahead of need: the launch uses every queue pair for demand
  bool demand_only() const { return mode == AGILE_SYNC; }
  uint32_t ahead;  // rows requested ahead of the one being summed (ASYNC), 1..32
  uint32_t group;  // rows pinned together at most (cache-sized), 1..32
  // bags left by the resident pass: positions 0 .. *list_n - 1 name bags list[pos]
  // (nullptr: every bag, position = bag); n_bags bounds the positions
  const uint32_t *list = nullptr;
  const uint32_t *list_n = nullptr;

  __device__ __forceinline__ uint32_t bag(uint32_t pos) const { return list ? list[pos] : pos; }

  __device__ __forceinline__ uint64_t row_page(uint64_t r) const { return page0 + (r * dim * 4) / kPage; }

  // position in the warp's stream of rows: bag b, index i
  struct Cursor {
    uint32_t b;
    int64_t i, e;
  };
  __device__ __forceinline__ void cur_init(const AppCtx &a, Cursor &c) const {
    c.b = a.warp;
    c.i = c.b < n_bags ? off[bag(c.b)] : 0;
    c.e = c.b < n_bags ? off[bag(c.b) + 1] : 0;
    skip_empty(a, c);
  }
  __device__ __forceinline__ void skip_empty(const AppCtx &a, Cursor &c) const {
    while (c.b < n_bags && c.i >= c.e) {
      c.b += a.n_warps;
      if (c.b < n_bags) {
        c.i = off[bag(c.b)];
        c.e = off[bag(c.b) + 1];
      }
    }
  }
  // issue the pages of the next `cnt` rows of the stream from cursor c (advances c);
  // rounds the backoff skips only advance the cursor
  __device__ bool issue_rows(const Dev &d, const AppCtx &a, Cursor &c, uint32_t cnt, Backoff &bo) const {
    while (cnt && c.b < n_bags) {
      uint32_t take = (uint32_t)min((int64_t)cnt, c.e - c.i);
      if (bo.take()) {
        unsigned l = lane_id();
        bool want = l < take;
        uint64_t r = want ? (uint64_t)idx[c.i + l] : 0;
        if (want && r >= rows) {
          set_error(d, AGILE_EINVAL);
          want = false;
        }
        uint32_t outcome = 0;
        if (!warp_request(d, want, row_page(r), a.q0, false, a.deadline, nullptr, nullptr, &outcome, true, true))
          return false;
        bo.result(outcome);
      }
      c.i += take;
      cnt -= take;
      skip_empty(a, c);
    }
    return true;
  }

  // A bag of at most `group` rows (one row per lane) prepared for the fast path: its
  // pages probed and pinned (one probe per distinct page) without waiting.  ok = every
  // page was READY and is now pinned.
  struct Prep {
    uint32_t b, cnt;
    bool fast, ok, leader;
    uint64_t pg;
    uint32_t off, line, myline;
  };

  __device__ void prep(const Dev &d, uint32_t b, Prep &p) const {
    unsigned l = lane_id();
    p.b = b;
    p.cnt = 0;
    p.fast = p.ok = p.leader = false;
    if (b >= n_bags) return;
    int64_t s = off[bag(b)], e = off[bag(b) + 1];
    p.cnt = (uint32_t)(e - s);
    p.fast = e > s && e - s <= (int64_t)min(group, 32u);
    if (!p.fast) return;
    bool want = l < p.cnt;
    uint64_t r = want ? (uint64_t)idx[s + l] : 0;
    if (want && r >= rows) {
      set_error(d, AGILE_EINVAL);
      r = 0;
    }
    uint64_t byte = r * dim * 4;
    p.pg = page0 + byte / kPage;
    p.off = (uint32_t)(byte % kPage);
    unsigned grp = __match_any_sync(kFull, want ? p.pg : ~0ull);
    int lead = __ffs(grp) - 1;
    p.leader = want && lead == (int)l;
    int pr = P_HIT;
    p.line = 0;
    if (p.leader) pr = cache_probe(d, p.pg, true, p.line);
    p.ok = __all_sync(kFull, !p.leader || pr == P_HIT);
    if (p.ok) {  // counted here; a bag that is not all resident is counted by gather_sum
      stat_warp(d, S_WARP_COALESCED, (want && !p.leader) ? 1u : 0u);
      stat_warp(d, S_HITS, p.leader ? 1u : 0u);
    } else if (p.leader && pr == P_HIT) {
      cache_unpin(d, p.line);  // not all resident: hold nothing, the slow path takes it
      p.leader = false;
    } else if (!p.ok) {
      p.leader = false;
    }
    p.myline = __shfl_sync(kFull, p.line, lead & 31);
  }

  __device__ void store_out(uint32_t b, const float4 (&acc)[MF4], uint32_t nf4) const {
    unsigned l = lane_id();
    float4 *o = (float4 *)(out + (uint64_t)bag(b) * dim);
#pragma unroll
    for (int k = 0; k < MF4; ++k) {
      uint32_t c = l + 32 * k;
      if (c < nf4) o[c] = acc[k];
    }
  }

  // general path for one bag: rows in groups, each group waiting for its pages as needed
  __device__ bool slow_bag(const Dev &d, const AppCtx &a, uint32_t b, uint32_t nf4, Cursor &pf, Backoff &bo) const {
    unsigned l = lane_id();
    const bool async = mode == AGILE_ASYNC;
    int64_t s = off[bag(b)], e = off[bag(b) + 1];
    float4 acc[MF4];
#pragma unroll
    for (int k = 0; k < MF4; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i0 = s; i0 < e; i0 += 32) {
      int64_t i = i0 + l;
      uint64_t r = i < e ? (uint64_t)idx[i] : 0;
      if (i < e && r >= rows) {
        set_error(d, AGILE_EINVAL);
        r = 0;
      }
      uint32_t cnt = (uint32_t)min((int64_t)32, e - i0);
      uint64_t byte = r * dim * 4;
      for (uint32_t g0 = 0; g0 < cnt; g0 += group) {
        uint32_t g1 = min(cnt, g0 + group);
        // keep the pages of the next `ahead` rows of the stream requested
        if (async && !issue_rows(d, a, pf, g1 - g0, bo)) return false;
        bool missed = false;
        if (!gather_sum<MF4>(d, a, g0, g1, page0 + byte / kPage, (uint32_t)(byte % kPage), nf4, acc, &missed))
          return false;
        if (missed) bo.missed();
      }
    }
    store_out(b, acc, nf4);
    return true;
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    if (list) {  // only the bags the resident pass left
      EmbApp me = *this;
      me.n_bags = min(n_bags, ld_acq32(list_n));
      me.list_n = nullptr;
      if (a.warp < me.n_bags) me.run_bags(d, a);
      return;
    }
    run_bags(d, a);
  }

  __device__ void run_bags(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    const uint32_t nf4 = dim / 4;
    const bool async = mode == AGILE_ASYNC;
    Cursor pf;  // prefetch cursor, `ahead` rows in front of the summation
    cur_init(a, pf);
    Backoff bo;
    if (async && !issue_rows(d, a, pf, ahead, bo)) return;
    constexpr int RB = MF4 >= 8 ? 1 : 8 / MF4;  // rows of an all-resident bag loaded before the next probe
    Prep cur;
    prep(d, a.warp, cur);
    for (uint32_t b = a.warp; b < n_bags; b += a.n_warps) {
      uint32_t nb = b + a.n_warps;
      if (!(cur.fast && cur.ok)) {
        // nothing pinned: the general path may wait
        if (async && cur.fast && !issue_rows(d, a, pf, cur.cnt, bo)) return;
        if (async && cur.fast) bo.missed();  // a short bag not all resident
        if (!slow_bag(d, a, b, nf4, pf, bo)) return;
        prep(d, nb, cur);
        continue;
      }
      // fast path: all pages of bag b are pinned.  Issue the first rows' loads, probe and
      // pin bag b+W while they are in flight, then add the rows in order.
      if (async && !issue_rows(d, a, pf, cur.cnt, bo)) return;
      float4 acc[MF4];
#pragma unroll
      for (int k = 0; k < MF4; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 v[RB][MF4];
#pragma unroll
      for (int jj = 0; jj < RB; ++jj) {
        uint32_t lj = __shfl_sync(kFull, cur.myline, jj);
        uint32_t oj = __shfl_sync(kFull, cur.off, jj);
        const uint8_t *rowp = line_ptr(d, lj) + oj;
#pragma unroll
        for (int c = 0; c < MF4; ++c) {
          uint32_t col = l + 32 * c;
          v[jj][c] = ((uint32_t)jj < cur.cnt && col < nf4) ? ld_cg_f4(rowp + 16 * col) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      Prep nxt;
      prep(d, nb, nxt);  // never waits; pins only pages that are READY
#pragma unroll
      for (int jj = 0; jj < RB; ++jj) {
        if ((uint32_t)jj < cur.cnt) {
#pragma unroll
          for (int c = 0; c < MF4; ++c) {
            acc[c].x = __fadd_rn(acc[c].x, v[jj][c].x);
            acc[c].y = __fadd_rn(acc[c].y, v[jj][c].y);
            acc[c].z = __fadd_rn(acc[c].z, v[jj][c].z);
            acc[c].w = __fadd_rn(acc[c].w, v[jj][c].w);
          }
        }
      }
      if (cur.cnt > (uint32_t)RB) sum_rows<MF4>(d, RB, cur.cnt - RB, cur.myline, cur.off, nf4, acc);
      __syncwarp();
      if (cur.leader) cache_unpin(d, cur.line);
      store_out(b, acc, nf4);
      cur = nxt;
    }
    (void)l;
  }
};

// ============================================================================ lookup + compute pipeline
// The DLRM-shaped overlap experiment (Sec. 4.2 computation-to-communication ratio;
// Sec. 4.4: in async mode the data of the next epoch is fetched during this one's compute).
// Work unit = (batch t, bag b): sum-pool `pooling` rows of each of n_tables tables
// into out[t][b][k*dim ...], then the compute phase: every output element goes through
// `iters` fused multiply-adds x = fma(x, kFmaA, kFmaB).  Warp w takes units w, w+W, ...
// in batch-major order.
//   SYNC : rows are requested when summed (a miss stalls the warp), then compute.
//   ASYNC: the warp keeps the pages of its next `ahead` rows requested (its units u,
//          u+W, ... as one row stream), so that fetch overlaps the gather and the
//          compute in front of them; `ahead` is what half of the cache holds for the
//          warps running, at most one unit.
// The compute is a phase of the same launch (not a separate kernel): the emulated
// device only runs while a library launch is resident.
constexpr float kFmaA = 0.999755859375f;  // 1 - 2^-12
constexpr float kFmaB = 0.0009765625f;    // 2^-10

template <int MF4>
struct PipeApp {
  uint64_t page0;     // first page of table 0
  uint64_t tstride;   // bytes between tables
  uint32_t n_tables, rows, dim;
  const int64_t *idx; // [batches][tables][bags][pooling]
  uint32_t pooling, n_bags, n_batches, iters;
  float *out;         // [batches][bags][tables*dim]
  uint32_t mode;
  // no request ahead of need: the launch uses every queue pair for demand
  bool demand_only() const { return mode == AGILE_SYNC; }
  uint32_t group;     // rows pinned together at most (cache-sized), 1..32
  uint32_t ahead;     // async: rows of the warp's row stream requested ahead (cache-sized)

  __device__ __forceinline__ uint64_t row_page(uint32_t k, uint64_t r) const {
    return page0 + ((uint64_t)k * tstride + r * dim * 4) / kPage;
  }

  // Position in the warp's row stream: its units u, u + W, ..., the rows of a unit in
  // table-major order.
  struct Cursor {
    uint64_t u;
    uint32_t q;
  };
  // request the pages of the next `cnt` rows of the stream from cursor c (advances c);
  // rounds the backoff skips only advance the cursor
  __device__ bool issue_ahead(const Dev &d, const AppCtx &a, Cursor &c, uint32_t cnt, uint64_t units,
                              Backoff &bo) const {
    const uint32_t per = n_tables * pooling;
    while (cnt && c.u < units) {
      uint32_t take = min(cnt, min(32u, per - c.q));
      if (bo.take()) {
        uint32_t q = c.q + lane_id();
        bool want = lane_id() < take;
        uint64_t t = c.u / n_bags, b = c.u % n_bags;
        uint32_t k = want ? q / pooling : 0, p = want ? q % pooling : 0;
        uint64_t r = want ? (uint64_t)idx[((t * n_tables + k) * n_bags + b) * pooling + p] : 0;
        if (want && r >= rows) {
          set_error(d, AGILE_EINVAL);
          want = false;
        }
        uint32_t outcome = 0;
        if (!warp_request(d, want, row_page(k, r), a.q0, false, a.deadline, nullptr, nullptr, &outcome, true, true))
          return false;
        bo.result(outcome);
      }
      c.q += take;
      cnt -= take;
      if (c.q == per) {
        c.q = 0;
        c.u += a.n_warps;
      }
    }
    return true;
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    const uint32_t nf4 = dim / 4;
    const bool async = mode == AGILE_ASYNC;
    const uint64_t units = (uint64_t)n_batches * n_bags;
    // async: the pages of the next `ahead` rows of the stream are requested before the
    // rows in front of them are gathered and computed on
    Cursor pf{a.warp, 0};
    Backoff bo;
    if (async && !issue_ahead(d, a, pf, ahead, units, bo)) return;
    for (uint64_t u = a.warp; u < units; u += a.n_warps) {
      uint64_t t = u / n_bags, b = u % n_bags;
      float *o = out + u * (uint64_t)n_tables * dim;
      for (uint32_t k = 0; k < n_tables; ++k) {
        float4 acc[MF4];
#pragma unroll
        for (int c = 0; c < MF4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        const int64_t *ix = idx + ((t * n_tables + k) * n_bags + b) * pooling;
        for (uint32_t p0 = 0; p0 < pooling; p0 += 32) {
          uint32_t cnt = min(32u, pooling - p0);
          uint64_t r = l < cnt ? (uint64_t)ix[p0 + l] : 0;
          if (r >= rows) {
            set_error(d, AGILE_EINVAL);
            r = 0;
          }
          uint64_t byte = (uint64_t)k * tstride + r * dim * 4;
          for (uint32_t g0 = 0; g0 < cnt; g0 += group) {
            uint32_t g1 = min(cnt, g0 + group);
            if (async && !issue_ahead(d, a, pf, g1 - g0, units, bo)) return;
            bool missed = false;
            if (!gather_sum<MF4>(d, a, g0, g1, page0 + byte / kPage, (uint32_t)(byte % kPage), nf4, acc, &missed))
              return;
            if (missed) bo.missed();
          }
        }
        // compute phase on this table's pooled row
#pragma unroll
        for (int c = 0; c < MF4; ++c) {
          uint32_t cc = l + 32 * c;
          if (cc < nf4) {
            float4 v = acc[c];
            for (uint32_t it = 0; it < iters; ++it) {
              v.x = __fmaf_rn(v.x, kFmaA, kFmaB);
              v.y = __fmaf_rn(v.y, kFmaA, kFmaB);
              v.z = __fmaf_rn(v.z, kFmaA, kFmaB);
              v.w = __fmaf_rn(v.w, kFmaA, kFmaB);
            }
            ((float4 *)(o + (uint64_t)k * dim))[cc] = v;
          }
        }
      }
    }
  }
};

// ============================================================================ BFS
// Level-synchronous top-down BFS (Sec. 4.5 BFS over CSR, through the cache).
// Level L: app warps claim chunks of 128 consecutive vertex ids; a lane owns one
// vertex and takes part when level[v] == L.  Its offsets[v], offsets[v+1] (int64) and
// its neighbour list (int32) are read through the cache; every neighbour u with
// level[u] == -1 gets level L+1 by compare-and-swap.  Vertices are visited in id order,
// so neighbouring lists that share a page are read while the page is resident.
// A list of at least kHub entries is not scanned by the warp that found it: it goes
// to a queue of long lists, cut into slices of kSlice entries that any warp may take,
// so one hub cannot hold up a level.  Every warp drains that queue before it reaches
// the grid barrier that ends the level; the search stops when a level discovers
// nothing.  Edges scanned = sum of the degrees of the frontier vertices of all levels.
//   SYNC : each page (offsets, columns) is requested when needed and waited for.
//   ASYNC: reads are issued before they are waited for, within the work at hand: a
//          32-vertex unit requests the list pages of all of its lanes before it scans
//          them, a sparse chunk requests its units' list pages together, and a long-list
//          slice requests all of its pages before it is scanned, so that their fetches
//          overlap.  (Requesting the pages of the next units ahead as well was measured
//          slower with the cache at an eighth of the column array: those pages were
//          evicted before their use.)
// A warp keeps at most one line pinned between steps (the page it read last) and lets
// it go before it requests or waits for any other page.
// One slice (at most kSlice entries) of a long adjacency list, queued for any warp.
struct HubEntry {
  long long p0, p1;          // column entries [p0, p1)
  unsigned long long ready;  // (launch epoch << 32) | (level + 1), written after p0, p1
  unsigned long long aux;    // SpMV: row | first slice of the row << 32 | last << 33
  unsigned long long carry;  // SpMV: (launch epoch << 32) | running sum after this slice
  unsigned long long pad[3];
};
static_assert(sizeof(HubEntry) == 64, "one slice record per 64 bytes");

// events of the BFS in the application event log (agile_events)
constexpr uint32_t kEvOwnDone = 1, kEvHubsDone = 2, kEvLevelDone = 3;

// A record is published with the number of the launch that wrote it (RunState::epoch,
// drawn on the device for every launch) and the level, so a record left by an earlier
// launch or level never looks published to a helper that reads it before its new owner
// has written it.
__device__ __forceinline__ uint64_t launch_epoch(const Dev &d) {
  return ld_rlx64(&d.run->epoch) & 0xFFFFFFFFull;
}

// kDirect: the same kernel over a CSR held in device memory (h_off, h_col), without the
// cache or the queues: the "kernel time" of the Sec. 4.5 three-step breakdown.
template <bool kDirect>
struct BfsAppT {
  uint64_t off_page0, col_page0;
  uint32_t n;
  int32_t *level;
  unsigned long long *edges_out;
  uint32_t mode;
  // its early requests (async) are for pages the warp reads right after, never a
  // lookahead: every queue pair carries demand in both modes
  bool demand_only() const { return true; }
  HubEntry *hubq;
  uint32_t hub_cap;
  uint32_t *vis;  // visited bitmap: bit u set once level[u] is set (read through L1, may lag)
  const uint8_t *h_off = nullptr, *h_col = nullptr;  // kDirect: the CSR arrays in HBM

  static constexpr uint32_t kChunk = 128;

  __device__ __forceinline__ uint64_t tag(const Dev &d, int32_t L) const {
    return (launch_epoch(d) << 32) | (uint32_t)(L + 1);
  }
  // lists of at least kHub entries go to the shared slice queue: a unit's owner scans at
  // most 32 x (kHub - 1) entries itself, so one warp holding heavy units cannot hold up
  // a level (the events of a level-2 trace showed the slowest warp at 2.6x the median
  // with kHub = 1024)
  static constexpr uint32_t kHub = 256;
  static constexpr uint32_t kSlice = 2048;

  struct Pin {
    uint64_t page;
    uint32_t line;
    bool valid;
  };

  __device__ __forceinline__ void release(const Dev &d, Pin &pc) const {
    if (pc.valid) {
      __syncwarp();
      if (lane_id() == 0) cache_unpin(d, pc.line);
      pc.valid = false;
    }
  }

  // Elements at bytes byte[0..N) of the array at store page `page0`, for the lanes'
  // elements with `want`, through the cache: the warp walks the distinct pages of the
  // requests, one pinned page at a time; the loads of all elements on the pinned page
  // are issued together.
  template <typename T, int N>
  __device__ bool gather_n(const Dev &d, const AppCtx &a, uint64_t page0, const bool (&want)[N],
                           const uint64_t (&byte)[N], T (&val)[N], Pin &pc) const {
    if constexpr (kDirect) {
      const uint8_t *base = page0 == off_page0 ? h_off : h_col;
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (want[i]) val[i] = __ldg((const T *)(base + byte[i]));
      return true;
    }
    uint64_t pg[N];
    uint32_t in[N];
    bool todo[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      pg[i] = page0 + byte[i] / kPage;
      in[i] = (uint32_t)(byte[i] % kPage);
      todo[i] = want[i];
    }
    for (;;) {
      if (pc.valid) {
        const uint8_t *base = line_ptr(d, pc.line);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (todo[i] && pg[i] == pc.page) {
            if (sizeof(T) == 8) val[i] = (T)ld_cg_s64(base + in[i]);
            else val[i] = (T)ld_cg_s32(base + in[i]);
            todo[i] = false;
          }
        }
      }
      bool any = false;
      uint64_t nxt = 0;
#pragma unroll
      for (int i = N - 1; i >= 0; --i) {
        if (todo[i]) {
          any = true;
          nxt = pg[i];
        }
      }
      unsigned m = __ballot_sync(kFull, any);
      if (!m) return true;
      uint64_t p = __shfl_sync(kFull, nxt, __ffs(m) - 1);
      release(d, pc);
      uint32_t line;
      if (!warp_pin_page<true>(d, p, a.q0, a.deadline, line)) return false;
      pc.page = p;
      pc.line = line;
      pc.valid = true;
    }
  }

  // Neighbours u[i] of the lanes (where act[i]): a set bit of the visited bitmap skips
  // u (the bitmap is read through L1 and may lag, since bits only go from 0 to 1: a
  // clear bit is confirmed against level[u]); the compare-and-swap of level[u] from -1
  // to L+1 discovers u, and its winner sets the bit.
  template <int N>
  __device__ __forceinline__ void visit_n(const bool (&act)[N], const int32_t (&u)[N], int32_t L,
                                          uint32_t &found) const {
    uint32_t w[N];
#pragma unroll
    for (int i = 0; i < N; ++i) w[i] = (act[i] && (uint32_t)u[i] < n) ? __ldca(&vis[(uint32_t)u[i] >> 5]) : ~0u;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      uint32_t b = 1u << ((uint32_t)u[i] & 31);
      if (!(w[i] & b) && ld_rlx32((const uint32_t *)&level[u[i]]) == 0xFFFFFFFFu &&
          atomicCAS((int *)&level[u[i]], -1, L + 1) == -1) {
        found++;
        atomicOr(&vis[(uint32_t)u[i] >> 5], b);
      }
    }
  }

  // both offsets of each lane's vertex (lanes with f): start s and end e of its list
  __device__ bool read_offsets(const Dev &d, const AppCtx &a, uint32_t v, bool f, int64_t &s, int64_t &e,
                               Pin &pc) const {
    bool want[2] = {f, f};
    uint64_t byte[2] = {(uint64_t)v * 8, (uint64_t)v * 8 + 8};
    int64_t val[2] = {0, 0};
    if (!gather_n<int64_t, 2>(d, a, off_page0, want, byte, val, pc)) return false;
    s = val[0];
    e = val[1];
    return true;
  }

  // Queue the lanes' lists of at least kHub entries as slices of at most kSlice entries:
  // one atomic add reserves consecutive record indices for all of the warp's slices,
  // then the warp writes the records, each published by its ready word.  A level has at
  // most (column entries) / kHub slices, which the queue holds; should a reservation
  // still run past the queue's end, its records inside the queue are published empty
  // and the lanes scan their lists here.  False for a lane that keeps its list.
  // Slices of the list [s, e) (at least kHub entries) follow the 2-page grid of the
  // column array, so that no page is shared by two slices of one list: slice 0 ends at
  // the first multiple of kSlice entries at least kHub entries past s, the following
  // ones hold kSlice entries, and a last piece of fewer than kHub entries joins the slice
  // before it.  Every slice holds at least kHub entries (so a level needs at most
  // entries / kHub records) and fewer than kSlice + 2 kHub.
  __device__ __forceinline__ static int64_t slice_b1(int64_t s) {
    return (s + kHub + kSlice - 1) / kSlice * kSlice;
  }
  __device__ __forceinline__ static uint32_t slice_count(int64_t s, int64_t e) {
    int64_t b1 = slice_b1(s);
    if (b1 >= e) return 1;
    int64_t rest = e - b1;
    uint32_t full = (uint32_t)(rest / kSlice);
    return 1 + full + ((rest % kSlice) >= kHub ? 1 : 0);
  }
  __device__ bool push_hub(const Dev &d, uint32_t deg, int64_t s, int64_t e, int32_t L) const {
    unsigned l = lane_id();
    bool hub = deg >= kHub;
    unsigned hm = __ballot_sync(kFull, hub);
    if (!hm) return false;
    uint32_t sl = hub ? slice_count(s, e) : 0;
    uint32_t incl = sl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (l >= (unsigned)o) incl += t;
    }
    uint32_t excl = incl - sl;
    uint32_t tot = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (l == 0) base = atomicAdd(&d.run->hub_count[L & 1], tot);
    base = __shfl_sync(kFull, base, 0);
    const uint64_t t = tag(d, L);
    if ((uint64_t)base + tot > hub_cap) {
      for (uint64_t j = (uint64_t)base + l; j < hub_cap; j += 32) {
        hubq[j].p0 = hubq[j].p1 = 0;
        st_rel64(&hubq[j].ready, t);
      }
      return false;  // scanned here
    }
    for (unsigned m = hm; m; m &= m - 1) {
      int h = __ffs(m) - 1;
      int64_t sh = __shfl_sync(kFull, s, h), eh = __shfl_sync(kFull, e, h);
      uint32_t bh = base + __shfl_sync(kFull, excl, h), nh = __shfl_sync(kFull, sl, h);
      const int64_t b1 = slice_b1(sh);
      for (uint32_t j = l; j < nh; j += 32) {
        HubEntry *r = &hubq[bh + j];
        r->p0 = j == 0 ? sh : b1 + (int64_t)(j - 1) * kSlice;
        r->p1 = j + 1 == nh ? eh : b1 + (int64_t)j * kSlice;
        st_rel64(&r->ready, t);
      }
    }
    return hub;
  }

  // scan the lists [s, s + dg) of the lanes, flattened over the warp (32 entries a step)
  __device__ bool scan_lists(const Dev &d, const AppCtx &a, int64_t s, uint32_t dg, int32_t L, uint32_t &found,
                             Pin &pc) const {
    unsigned l = lane_id();
    uint32_t incl = dg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (l >= (unsigned)o) incl += t;
    }
    uint32_t excl = incl - dg;
    uint32_t total = __shfl_sync(kFull, incl, 31);
    // two 32-entry steps at a time: their loads are in flight together
    for (uint32_t k0 = 0; k0 < total; k0 += 64) {
      bool act[2];
      uint64_t byte[2];
      int32_t u[2] = {0, 0};
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        uint32_t k = k0 + 32 * h + l;
        act[h] = k < total;
        // owner lane j: the last lane whose exclusive prefix is <= k
        uint32_t j = 0;
#pragma unroll
        for (int step = 16; step >= 1; step >>= 1) {
          uint32_t cand = j + step;
          uint32_t ex = __shfl_sync(kFull, excl, cand & 31);
          if (cand < 32 && ex <= k) j = cand;
        }
        int64_t sj = __shfl_sync(kFull, s, j);
        uint32_t exj = __shfl_sync(kFull, excl, j);
        byte[h] = ((uint64_t)sj + (k - exj)) * 4;
      }
      if (!gather_n<int32_t, 2>(d, a, col_page0, act, byte, u, pc)) return false;
      visit_n<2>(act, u, L, found);
    }
    return true;
  }

  // ASYNC, sparse chunks: the offsets of the chunk's frontier vertices are read, then the
  // column pages of their short lists are requested together, without waiting, before
  // the chunk's units are scanned -- so the misses of up to kChunk / 32 units overlap
  // instead of following one another.  Only when each lane has at most one page to
  // request (sparse levels): in dense ones the pages would outnumber what the cache
  // holds for the running warps.
  __device__ bool prefetch_chunk(const Dev &d, const AppCtx &a, uint32_t c0, uint32_t fbits, Pin &pc) const {
    constexpr uint32_t U = kChunk / 32;
    unsigned l = lane_id();
    // the lane's page to request (at most one over the chunk's units; two or more
    // anywhere in the warp: the chunk is not sparse, pages are requested when needed)
    uint32_t cnt = 0;
    uint64_t pg = 0;
    for (uint32_t k = 0; k < U; ++k) {
      uint32_t v = c0 + 32 * k + l;
      bool f = (fbits >> k) & 1u;
      if (!__any_sync(kFull, f)) continue;
      int64_t s0 = 0, e0 = 0;
      if (!read_offsets(d, a, v, f, s0, e0, pc)) return false;
      if (f && e0 > s0 && e0 - s0 < (int64_t)kHub) {
        uint64_t p0 = ((uint64_t)s0 * 4) / kPage, p1 = ((uint64_t)(e0 - 1) * 4) / kPage;
        cnt += (cnt == 0 || p0 != pg) ? 1u : 0u;
        cnt += p1 != p0 ? 1u : 0u;
        pg = p1;
      }
      if (!__all_sync(kFull, cnt <= 1)) return true;  // not sparse: pages when needed
    }
    bool has = cnt == 1 && !(pc.valid && pc.page == col_page0 + pg);
    if (!__any_sync(kFull, has)) return true;
    return warp_request_call(d, has, col_page0 + pg, a.q0, false, a.deadline);
  }

  // one 32-vertex unit: SYNC requests every page when needed
  // (f: the lane's vertex is in the frontier)
  __device__ bool chunk(const Dev &d, const AppCtx &a, uint32_t v0, bool f, int32_t L, uint32_t &found,
                        unsigned long long &scanned, Pin &pc) const {
    uint32_t v = v0 + lane_id();
    if (!__any_sync(kFull, f)) return true;
    int64_t s = 0, e = 0;
    if (!read_offsets(d, a, v, f, s, e, pc)) return false;
    uint32_t deg = f ? (uint32_t)(e - s) : 0;
    scanned += __reduce_add_sync(kFull, deg);
    bool hub = push_hub(d, deg, s, e, L);
    const uint32_t dg = hub ? 0 : deg;
    if (!kDirect && mode == AGILE_ASYNC) {
      // ASYNC: when the unit's lists span more than one page, the pages of every lane's
      // list (at most two, since the list is shorter than kHub entries) are requested
      // together before the scan, so that the unit's misses overlap instead of
      // following one another
      uint64_t p0 = ((uint64_t)s * 4) / kPage, p1 = dg ? ((uint64_t)(s + dg - 1) * 4) / kPage : p0;
      unsigned multi = __ballot_sync(kFull, dg && p1 != p0);
      uint64_t lo = dg ? p0 : ~0ull, hi = dg ? p1 : 0;
#pragma unroll
      for (int o = 16; o >= 1; o >>= 1) {
        lo = min(lo, (uint64_t)__shfl_xor_sync(kFull, lo, o));
        hi = max(hi, (uint64_t)__shfl_xor_sync(kFull, hi, o));
      }
      if (hi > lo) {
        bool w0 = dg && !(pc.valid && pc.page == col_page0 + p0);
        if (!warp_request_call(d, w0, col_page0 + p0, a.q0, false, a.deadline)) return false;
        if (multi && !warp_request_call(d, dg && p1 != p0, col_page0 + p1, a.q0, false, a.deadline)) return false;
      }
    }
    return scan_lists(d, a, s, dg, L, found, pc);
  }

  // Take queued slices of level L, one ticket (a record index) at a time, until every
  // slice is taken.  A ticket waits, holding no pin, for its record to be published;
  // it is past the last slice when every warp has finished its own vertices (no more
  // reservations come) and the reserved count is at most the ticket.  Each warp so ends
  // with one ticket past the last slice.  Waiting warps watch their own record and look
  // at the shared counters only now and then.
  __device__ bool help_hubs(const Dev &d, const AppCtx &a, int32_t L, uint32_t &found, Pin &pc) const {
    unsigned l = lane_id();
    const uint64_t want_tag = tag(d, L);
    const int par = L & 1;
    for (;;) {
      uint32_t k = 0;
      if (l == 0) k = atomicAdd(&d.run->hub_cursor[par], 1u);
      k = __shfl_sync(kFull, k, 0);
      if (k >= hub_cap) return true;
      HubEntry *r = &hubq[k];
      uint32_t ns = 64;
      int state = 0;  // 1: record published, 2: past the last slice
      for (uint32_t spin = 0;; ++spin) {
        if (l == 0) {
          if (ld_acq64(&r->ready) == want_tag) {
            state = 1;
          } else if ((spin & 7) == 7 && ld_acq32(&d.run->units_done[par]) >= a.n_warps &&
                     ld_acq32(&d.run->hub_count[par]) <= k) {
            state = 2;
          }
        }
        state = __shfl_sync(kFull, state, 0);
        if (state) break;
        release(d, pc);
        if (gtimer() > a.deadline || aborted(d)) {
          if (l == 0) set_error(d, -110);
          return false;
        }
        backoff(ns, 1024);
      }
      if (state == 2) return true;
      int64_t p0 = 0, p1 = 0;
      if (l == 0) {
        p0 = ld_cg_s64(&r->p0);
        p1 = ld_cg_s64(&r->p1);
      }
      p0 = __shfl_sync(kFull, p0, 0);
      p1 = __shfl_sync(kFull, p1, 0);
      if (p1 <= p0) continue;  // an empty record (a reservation past the queue's end)
      if (!kDirect && mode == AGILE_ASYNC) {
        uint64_t q0p = col_page0 + ((uint64_t)p0 * 4) / kPage, q1p = col_page0 + ((uint64_t)(p1 - 1) * 4) / kPage;
        uint64_t pg = q0p + l;
        bool want = pg <= q1p && !(pc.valid && pc.page == pg);
        if (__any_sync(kFull, want) && !warp_request_call(d, want, pg, a.q0, false, a.deadline)) return false;
      }
      for (int64_t b0 = p0; b0 < p1; b0 += 64) {
        bool on[2];
        uint64_t byte[2];
        int32_t u[2] = {0, 0};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t pos = b0 + 32 * h + l;
          on[h] = pos < p1;
          byte[h] = (uint64_t)(on[h] ? pos : p0) * 4;
        }
        if (!gather_n<int32_t, 2>(d, a, col_page0, on, byte, u, pc)) return false;
        visit_n<2>(on, u, L, found);
      }
    }
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    uint32_t nchunks = (n + kChunk - 1) / kChunk;
    unsigned long long scanned = 0;
    for (int32_t L = 0;; ++L) {
      if (a.warp == 0 && l == 0) {
        // the counters of level L+1 were last used at level L-1, whose work every warp
        // finished before barrier L-1; the discovery counter of level L+1 (three slots)
        // was last read right after barrier L-2, which every warp has left
        st_rlx32(&d.run->work[(L + 1) & 1], 0u);
        st_rlx32(&d.run->hub_count[(L + 1) & 1], 0u);
        st_rlx32(&d.run->hub_cursor[(L + 1) & 1], 0u);
        st_rlx32(&d.run->units_done[(L + 1) & 1], 0u);
        st_rlx64(&d.run->acc[1 + (L + 1) % 3], 0ull);
      }
      uint32_t found = 0;
      Pin pc{0, 0, false};
      bool ok = true;
      for (;;) {
        uint32_t c = 0;
        if (l == 0) c = atomicAdd(&d.run->work[L & 1], 1u);
        c = __shfl_sync(kFull, c, 0);
        if (c >= nchunks || aborted(d)) break;
        // the chunk's level words, all in flight together: bit k of fbits says whether
        // the lane's vertex of unit k is in the frontier (a word equal to L was written
        // at the level before and does not change during this one)
        constexpr uint32_t U = kChunk / 32;
        uint32_t lv[U];
#pragma unroll
        for (uint32_t k = 0; k < U; ++k) {
          uint32_t v = c * kChunk + 32 * k + l;
          lv[k] = v < n ? ld_rlx32((const uint32_t *)&level[v]) : 0xFFFFFFFFu;
        }
        uint32_t fbits = 0;
#pragma unroll
        for (uint32_t k = 0; k < U; ++k) fbits |= (lv[k] == (uint32_t)L ? 1u : 0u) << k;
        if (!__any_sync(kFull, fbits)) continue;
        if (!kDirect && mode == AGILE_ASYNC) ok = prefetch_chunk(d, a, c * kChunk, fbits, pc);
        for (uint32_t k = 0; k < U && ok; ++k)
          ok = chunk(d, a, c * kChunk + 32 * k, (fbits >> k) & 1u, L, found, scanned, pc);
        if (!ok) break;
      }
      // this warp queues no more slices of level L
      __syncwarp();
      if (l == 0) {
        fence_ar();
        atomicAdd(&d.run->units_done[L & 1], 1u);
        app_event(d, a.warp, kEvOwnDone, (uint32_t)L);
      }
      if (ok) help_hubs(d, a, L, found, pc);
      release(d, pc);
      uint32_t tot = __reduce_add_sync(kFull, found);
      if (l == 0 && tot) atomicAdd(&d.run->acc[1 + L % 3], (unsigned long long)tot);
      if (l == 0) app_event(d, a.warp, kEvHubsDone, (uint32_t)L);
      if (!app_barrier(d, a.n_warps, a.deadline)) return;
      if (l == 0) app_event(d, a.warp, kEvLevelDone, (uint32_t)L);
      if (aborted(d)) return;
      uint64_t disc = ld_acq64(&d.run->acc[1 + L % 3]);
      if (disc == 0) break;
    }
    if (l == 0 && scanned) atomicAdd(&d.run->acc[0], scanned);
    if (!app_barrier(d, a.n_warps, a.deadline)) return;
    if (a.warp == 0 && l == 0 && edges_out) *edges_out = ld_acq64(&d.run->acc[0]);
  }
};

using BfsApp = BfsAppT<false>;

// ============================================================================ SpMV
// y = A x over a CSR matrix on the store (Sec. 4.5 runs SpMV over the CSR graphs of its
// BFS): int64 offsets, int32 columns and FP32 values are read through the cache; x and
// y are device arrays of the caller.  Warps take chunks of kChunk consecutive rows, in
// units of 32 rows (a lane owns a row); a unit's entries are flattened over the warp,
// 32 a step, the column and the value of an entry each read through the cache.  The
// offsets, column and value arrays each keep one pinned page; before a warp waits for a
// page it lets the other two go, so it never waits while holding a pin.  A row's
// products are added in increasing entry order: within a step by a chain over the
// lanes (lane t adds its product to lane t-1's running sum), across steps through the
// owner lane's running sum, so a row of fewer than kHub entries equals the sequential
// definition bit for bit.  A row of at least kHub entries is queued as slices of
// kSlice entries (the BFS slice queue), which any warp may take: the warp computes the
// slice's products (into shared memory, all of its pages in flight together), then
// takes the running sum the row's previous slice published (a slice waits for it
// holding no pin) and adds its products to it in entry order, one add after the other;
// the row's last slice writes y[v].  Every row is therefore the sequential definition
// bit for bit; only the adds of a long row run one slice after the other.
//   SYNC : every page when needed.
//   ASYNC: a unit requests the column and value pages of all the entries it sums (at
//          most 32 of each array) right after reading its offsets, then computes, so
//          that the unit's misses overlap.  (A pipeline that requested the next units'
//          pages while computing this one was measured slower with the cache at an
//          eighth of the arrays: those pages were evicted before their use.)
// kDirect: the same kernel over a CSR held in device memory (h_off, h_col, h_val),
// without the cache or the queues (Sec. 4.5 "kernel time").
template <bool kDirect>
struct SpmvAppT {
  uint64_t off_page0, col_page0, val_page0;
  uint32_t n;    // rows
  const float *x;
  uint32_t n_x;  // columns (length of x)
  float *y;
  unsigned long long *entries_out;
  uint32_t mode;
  // its early requests (async) are for pages the warp reads right after, never a
  // lookahead: every queue pair carries demand in both modes
  bool demand_only() const { return true; }
  HubEntry *hubq;
  uint32_t hub_cap;
  const uint8_t *h_off = nullptr, *h_col = nullptr, *h_val = nullptr;  // kDirect: the CSR in HBM

  static constexpr uint32_t kChunk = 128;
  static constexpr uint32_t kHub = 1024;
  static constexpr uint32_t kSlice = 1024;  // = the products buffer of a warp

  struct Pin {
    uint64_t page;
    uint32_t line;
    bool valid;
  };

  __device__ __forceinline__ void release(const Dev &d, Pin &pc) const {
    if (pc.valid) {
      __syncwarp();
      if (lane_id() == 0) cache_unpin(d, pc.line);
      pc.valid = false;
    }
  }

  // Elements at bytes byte[0..N) of the array at store page `page0`, for the elements
  // with `want`, through pin `pc`: the warp walks the distinct pages of the requests.
  // A page that is not resident is waited for only after o1 and o2 have been let go.
  template <typename T, int N>
  __device__ bool gather(const Dev &d, const AppCtx &a, uint64_t page0, const bool (&want)[N],
                         const uint64_t (&byte)[N], T (&val)[N], Pin &pc, Pin &o1, Pin &o2) const {
    if constexpr (kDirect) {
      const uint8_t *base = page0 == off_page0 ? h_off : (page0 == col_page0 ? h_col : h_val);
#pragma unroll
      for (int i = 0; i < N; ++i)
        if (want[i]) val[i] = __ldg((const T *)(base + byte[i]));
      return true;
    }
    uint64_t pg[N];
    uint32_t in[N];
    bool todo[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      pg[i] = page0 + byte[i] / kPage;
      in[i] = (uint32_t)(byte[i] % kPage);
      todo[i] = want[i];
    }
    for (;;) {
      if (pc.valid) {
        const uint8_t *base = line_ptr(d, pc.line);
#pragma unroll
        for (int i = 0; i < N; ++i) {
          if (todo[i] && pg[i] == pc.page) {
            if (sizeof(T) == 8) {
              long long raw = ld_cg_s64(base + in[i]);
              memcpy(&val[i], &raw, 8);
            } else {
              int raw = ld_cg_s32(base + in[i]);
              memcpy(&val[i], &raw, 4);
            }
            todo[i] = false;
          }
        }
      }
      bool any = false;
      uint64_t nxt = 0;
#pragma unroll
      for (int i = N - 1; i >= 0; --i) {
        if (todo[i]) {
          any = true;
          nxt = pg[i];
        }
      }
      unsigned m = __ballot_sync(kFull, any);
      if (!m) return true;
      uint64_t p = __shfl_sync(kFull, nxt, __ffs(m) - 1);
      release(d, pc);
      uint32_t line = 0;
      if (warp_probe_pin(d, p, line) != P_HIT) {
        release(d, o1);
        release(d, o2);
        if (!warp_pin_page<true>(d, p, a.q0, a.deadline, line)) return false;
      }
      pc.page = p;
      pc.line = line;
      pc.valid = true;
    }
  }

  // product of the entry at `pos` (lanes with act): vals[pos] * x[cols[pos]], rounded
  __device__ bool product(const Dev &d, const AppCtx &a, bool act, uint64_t pos, float &prod, Pin &po, Pin &pcol,
                          Pin &pval) const {
    const bool w[1] = {act};
    const uint64_t b[1] = {pos * 4};
    int32_t col[1] = {0};
    float val[1] = {0.f};
    if (!gather<int32_t, 1>(d, a, col_page0, w, b, col, pcol, pval, po)) return false;
    if (!gather<float, 1>(d, a, val_page0, w, b, val, pval, pcol, po)) return false;
    prod = 0.f;
    if (act) {
      float xv = 0.f;
      if ((uint32_t)col[0] < n_x) xv = __ldg(&x[col[0]]);
      else set_error(d, AGILE_EINVAL);
      prod = __fmul_rn(val[0], xv);
    }
    return true;
  }

  // In-order running sums over one step: unless it starts a row segment (its `run`
  // already set by the caller), lane t adds its product to lane t-1's running sum.
  __device__ __forceinline__ float chain(float run, float prod, bool cont) const {
    unsigned l = lane_id();
#pragma unroll
    for (int t = 1; t < 32; ++t) {
      float prev = __shfl_sync(kFull, run, t - 1);
      if ((int)l == t && cont) run = __fadd_rn(prev, prod);
    }
    return run;
  }

  // both offsets of each lane's row (lanes with f)
  __device__ bool read_offsets(const Dev &d, const AppCtx &a, uint32_t v, bool f, int64_t &s, int64_t &e, Pin &po,
                               Pin &pcol, Pin &pval) const {
    const bool want[2] = {f, f};
    const uint64_t byte[2] = {(uint64_t)v * 8, (uint64_t)v * 8 + 8};
    int64_t val[2] = {0, 0};
    if (!gather<int64_t, 2>(d, a, off_page0, want, byte, val, po, pcol, pval)) return false;
    s = val[0];
    e = val[1];
    return true;
  }

  // queue the lanes' rows of at least kHub entries as slices (as the BFS does); each
  // record names its row and whether it is the row's first and last slice
  __device__ bool push_hub(const Dev &d, uint32_t v, uint32_t deg, int64_t s, int64_t e) const {
    unsigned l = lane_id();
    bool hub = deg >= kHub;
    unsigned hm = __ballot_sync(kFull, hub);
    if (!hm) return false;
    uint32_t sl = hub ? (deg + kSlice - 1) / kSlice : 0;
    uint32_t incl = sl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (l >= (unsigned)o) incl += t;
    }
    uint32_t excl = incl - sl;
    uint32_t tot = __shfl_sync(kFull, incl, 31);
    uint32_t base = 0;
    if (l == 0) base = atomicAdd(&d.run->hub_count[0], tot);
    base = __shfl_sync(kFull, base, 0);
    const uint64_t t = (launch_epoch(d) << 32) | 1u;
    if ((uint64_t)base + tot > hub_cap) {
      for (uint64_t j = (uint64_t)base + l; j < hub_cap; j += 32) {
        hubq[j].p0 = hubq[j].p1 = 0;
        st_rel64(&hubq[j].ready, t);
      }
      return false;  // summed here
    }
    for (unsigned m = hm; m; m &= m - 1) {
      int h = __ffs(m) - 1;
      int64_t sh = __shfl_sync(kFull, s, h), eh = __shfl_sync(kFull, e, h);
      uint32_t vh = __shfl_sync(kFull, v, h);
      uint32_t bh = base + __shfl_sync(kFull, excl, h), nh = __shfl_sync(kFull, sl, h);
      for (uint32_t j = l; j < nh; j += 32) {
        HubEntry *r = &hubq[bh + j];
        int64_t p0 = sh + (int64_t)j * kSlice;
        r->p0 = p0;
        r->p1 = min(eh, p0 + (int64_t)kSlice);
        r->aux = (uint64_t)vh | ((uint64_t)(j == 0) << 32) | ((uint64_t)(j + 1 == nh) << 33);
        st_rel64(&r->ready, t);
      }
    }
    return hub;
  }

  // The rows [v0, v0 + 32): lane l's row starts at entry s and has `dg` entries summed
  // here (0 for a queued row): flattened over the warp, summed in order; y written for
  // the lanes with `keep`.
  __device__ bool compute_unit(const Dev &d, const AppCtx &a, uint32_t v0, int64_t s, uint32_t dg, bool keep,
                               Pin &po, Pin &pcol, Pin &pval) const {
    unsigned l = lane_id();
    uint32_t incl = dg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(kFull, incl, o);
      if (l >= (unsigned)o) incl += t;
    }
    uint32_t excl = incl - dg;
    uint32_t total = __shfl_sync(kFull, incl, 31);
    float acc = 0.0f;  // this lane's row: running sum
    for (uint32_t k0 = 0; k0 < total; k0 += 32) {
      uint32_t k = k0 + l;
      bool act = k < total;
      // owner lane j: the last lane whose exclusive prefix is <= k
      uint32_t j = 0;
#pragma unroll
      for (int step = 16; step >= 1; step >>= 1) {
        uint32_t cand = j + step;
        uint32_t ex = __shfl_sync(kFull, excl, cand & 31);
        if (cand < 32 && ex <= k) j = cand;
      }
      int64_t sj = __shfl_sync(kFull, s, j);
      uint32_t exj = __shfl_sync(kFull, excl, j);
      float prod = 0.f;
      if (!product(d, a, act, act ? (uint64_t)sj + (k - exj) : 0, prod, po, pcol, pval)) return false;
      float carry = __shfl_sync(kFull, acc, j);
      bool first = act && (k == exj || l == 0);  // the row's first entry in this step
      float run = first ? __fadd_rn(k == exj ? 0.0f : carry, prod) : prod;
      run = chain(run, prod, act && !first);
      // the owner takes its row's running sum from the row's last lane in this step
      uint32_t endk = excl + dg;
      bool mine = dg > 0 && excl < k0 + 32 && endk > k0;
      uint32_t last = mine ? min(endk, k0 + 32) - 1 - k0 : 0;
      float got = __shfl_sync(kFull, run, last);
      if (mine) acc = got;
    }
    if (keep) y[v0 + l] = acc;
    return true;
  }

  __device__ bool next_unit(const Dev &d, uint32_t nchunks, uint32_t &chunk, uint32_t &sub, uint32_t &v0) const {
    if (sub >= kChunk) {
      uint32_t c = 0;
      if (lane_id() == 0) c = atomicAdd(&d.run->work[0], 1u);
      chunk = __shfl_sync(kFull, c, 0);
      sub = 0;
      if (chunk >= nchunks || aborted(d)) return false;
    }
    v0 = chunk * kChunk + sub;
    sub += 32;
    return v0 < n;
  }

  // ASYNC: read the unit's offsets, queue its long rows, request its column and value pages
  __device__ bool issue_unit(const Dev &d, const AppCtx &a, uint32_t v0, int64_t &s, uint32_t &dg, bool &keep,
                             unsigned long long &entries, Pin &po, Pin &pcol, Pin &pval) const {
    uint32_t v = v0 + lane_id();
    bool f = v < n;
    int64_t e = 0;
    s = 0;
    if (!read_offsets(d, a, v, f, s, e, po, pcol, pval)) return false;
    uint32_t deg = f ? (uint32_t)(e - s) : 0;
    entries += __reduce_add_sync(kFull, deg);
    bool hub = push_hub(d, v, deg, s, e);
    dg = hub ? 0 : deg;
    keep = f && !hub;
    // the entries summed here lie in one span (queued rows are holes in it): request
    // the span's pages of both arrays, at most 32 of each
    long long lo = dg ? s : LLONG_MAX, hi = dg ? s + dg : 0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      lo = min(lo, __shfl_xor_sync(kFull, lo, o));
      hi = max(hi, __shfl_xor_sync(kFull, hi, o));
    }
    if (kDirect || hi <= lo) return true;
    uint64_t c0 = ((uint64_t)lo * 4) / kPage, c1 = ((uint64_t)(hi - 1) * 4) / kPage;
    bool want = c0 + lane_id() <= c1;
    if (!warp_request_call(d, want, col_page0 + c0 + lane_id(), a.q0, false, a.deadline, true)) return false;
    return warp_request_call(d, want, val_page0 + c0 + lane_id(), a.q0, false, a.deadline, true);
  }

  // take queued slices until every slice is taken (the BFS slice queue, one level)
  __device__ bool help_hubs(const Dev &d, const AppCtx &a, Pin &po, Pin &pcol, Pin &pval) const {
    __shared__ float prod_buf[kWarps][kSlice];  // products of the slice a warp holds
    float *buf = prod_buf[threadIdx.x >> 5];
    unsigned l = lane_id();
    const uint64_t ep = launch_epoch(d);
    const uint64_t want_tag = (ep << 32) | 1u;
    for (;;) {
      uint32_t k = 0;
      if (l == 0) k = atomicAdd(&d.run->hub_cursor[0], 1u);
      k = __shfl_sync(kFull, k, 0);
      if (k >= hub_cap) return true;
      HubEntry *r = &hubq[k];
      uint32_t ns = 64;
      int state = 0;  // 1: record published, 2: past the last slice
      for (uint32_t spin = 0;; ++spin) {
        if (l == 0) {
          if (ld_acq64(&r->ready) == want_tag) {
            state = 1;
          } else if ((spin & 7) == 7 && ld_acq32(&d.run->units_done[0]) >= a.n_warps &&
                     ld_acq32(&d.run->hub_count[0]) <= k) {
            state = 2;
          }
        }
        state = __shfl_sync(kFull, state, 0);
        if (state) break;
        release(d, po);
        release(d, pcol);
        release(d, pval);
        if (gtimer() > a.deadline || aborted(d)) {
          if (l == 0) set_error(d, -110);
          return false;
        }
        backoff(ns, 1024);
      }
      if (state == 2) return true;
      int64_t p0 = 0, p1 = 0;
      uint64_t aux = 0;
      if (l == 0) {
        p0 = ld_cg_s64(&r->p0);
        p1 = ld_cg_s64(&r->p1);
        aux = (uint64_t)ld_cg_s64(&r->aux);
      }
      p0 = __shfl_sync(kFull, p0, 0);
      p1 = __shfl_sync(kFull, p1, 0);
      aux = __shfl_sync(kFull, aux, 0);
      if (p1 <= p0) continue;  // an empty record (a reservation past the queue's end)
      const uint32_t row = (uint32_t)aux;
      const bool first = (aux >> 32) & 1, last = (aux >> 33) & 1;
      release(d, po);
      if (!kDirect && mode == AGILE_ASYNC) {
        uint64_t c0 = ((uint64_t)p0 * 4) / kPage, c1 = ((uint64_t)(p1 - 1) * 4) / kPage;
        bool want = c0 + l <= c1;
        if (!warp_request_call(d, want, col_page0 + c0 + l, a.q0, false, a.deadline)) return false;
        if (!warp_request_call(d, want, val_page0 + c0 + l, a.q0, false, a.deadline)) return false;
      }
      // products of the slice, two entries a lane at a time, into the warp's buffer
      for (int64_t b0 = p0; b0 < p1; b0 += 64) {
        bool on[2];
        uint64_t byte[2];
        int32_t col[2] = {0, 0};
        float val[2] = {0.f, 0.f};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          int64_t pos = b0 + 32 * h + l;
          on[h] = pos < p1;
          byte[h] = (uint64_t)(on[h] ? pos : p0) * 4;
        }
        if (!gather<int32_t, 2>(d, a, col_page0, on, byte, col, pcol, pval, po)) return false;
        if (!gather<float, 2>(d, a, val_page0, on, byte, val, pval, pcol, po)) return false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (on[h]) {
            float xv = 0.f;
            if ((uint32_t)col[h] < n_x) xv = __ldg(&x[col[h]]);
            else set_error(d, AGILE_EINVAL);
            buf[b0 - p0 + 32 * h + l] = __fmul_rn(val[h], xv);
          }
        }
      }
      // the running sum of the row so far: +0 before its first entry, else what the
      // previous slice (the record before this one) published; waited for holding no pin
      float run = 0.0f;
      if (!first) {
        release(d, pcol);
        release(d, pval);
        const HubEntry *prev = &hubq[k - 1];
        uint64_t cw = 0;
        uint32_t ns2 = 32;
        for (;;) {
          if (l == 0) cw = ld_acq64(&prev->carry);
          cw = __shfl_sync(kFull, cw, 0);
          if ((cw >> 32) == ep) break;
          if (gtimer() > a.deadline || aborted(d)) {
            if (l == 0) set_error(d, -110);
            return false;
          }
          backoff(ns2, 256);
        }
        run = __uint_as_float((uint32_t)cw);
      }
      __syncwarp();
      if (l == 0) {
        const uint32_t cnt = (uint32_t)(p1 - p0);
        for (uint32_t i = 0; i < cnt; ++i) run = __fadd_rn(run, buf[i]);
        if (last) y[row] = run;
        else st_rel64(&r->carry, (ep << 32) | __float_as_uint(run));
      }
      __syncwarp();
    }
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    const uint32_t nchunks = (n + kChunk - 1) / kChunk;
    unsigned long long entries = 0;
    Pin po{0, 0, false}, pcol{0, 0, false}, pval{0, 0, false};
    bool ok = true;
    uint32_t chunk = 0, sub = kChunk;
    if (!kDirect && mode == AGILE_ASYNC) {
      uint32_t v0 = 0;
      while (ok && next_unit(d, nchunks, chunk, sub, v0)) {
        int64_t s = 0;
        uint32_t dg = 0;
        bool k = false;
        ok = issue_unit(d, a, v0, s, dg, k, entries, po, pcol, pval);
        if (ok) ok = compute_unit(d, a, v0, s, dg, k, po, pcol, pval);
      }
    } else {
      uint32_t v0 = 0;
      while (ok && next_unit(d, nchunks, chunk, sub, v0)) {
        uint32_t v = v0 + l;
        bool f = v < n;
        int64_t s = 0, e = 0;
        ok = read_offsets(d, a, v, f, s, e, po, pcol, pval);
        if (!ok) break;
        uint32_t deg = f ? (uint32_t)(e - s) : 0;
        entries += __reduce_add_sync(kFull, deg);
        bool hub = push_hub(d, v, deg, s, e);
        ok = compute_unit(d, a, v0, s, hub ? 0 : deg, f && !hub, po, pcol, pval);
      }
    }
    // this warp queues no more slices
    __syncwarp();
    if (l == 0) {
      fence_ar();
      atomicAdd(&d.run->units_done[0], 1u);
    }
    if (ok) help_hubs(d, a, po, pcol, pval);
    release(d, po);
    release(d, pcol);
    release(d, pval);
    if (l == 0 && entries) atomicAdd(&d.run->acc[0], entries);
    if (!app_barrier(d, a.n_warps, a.deadline)) return;
    if (a.warp == 0 && l == 0 && entries_out) *entries_out = ld_acq64(&d.run->acc[0]);
  }
};

using SpmvApp = SpmvAppT<false>;

// ============================================================================ resident pass
// First pass of agile_embedding_bag: every bag whose pages are all in the cache is summed
// here, by a light kernel that runs many warps per SM (no service warps, no miss path),
// and the others are listed for the engine launch that follows.  Within one call nothing
// can evict a line before the engine issues its first miss (a context is used by one
// stream at a time), so the tags are read with plain loads and no line is pinned.  A
// warp per bag; the pages of the bag's rows are probed once per distinct page (the
// lowest lane of each group, as the engine does), a hit sets the line's reference bit;
// a bag of more than 32 indices, with an index out of range or with a page that is not
// READY / MODIFIED is listed.  The sum is the engine's: rows in increasing index order,
// FP32, no fusion.
template <int MF4>
__global__ void __launch_bounds__(256, MF4 >= 8 ? 2 : 3) resident_bag_kernel(Dev d, uint64_t page0, uint32_t rows, uint32_t dim,
                                                           const int64_t *idx, const int64_t *off, uint32_t n_bags,
                                                           float *out, uint32_t *list, uint32_t *list_n) {
  const unsigned l = threadIdx.x & 31;
  const uint32_t nf4 = dim / 4;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  // rows whose loads are in flight together (few registers: three CTAs an SM, two for
  // the widest rows)
  constexpr int RB = MF4 >= 4 ? 2 : 8 / MF4;
  // software pipeline over the warp's bags: the offsets of the next bag are loaded
  // before this bag's tags, its indices before this bag's rows
  uint64_t b = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  int64_t s = 0, e = 0;
  uint64_t r = 0;
  if (b < n_bags) {
    s = off[b];
    e = off[b + 1];
    if ((int64_t)l < e - s && e - s <= 32) r = (uint64_t)idx[s + l];
  }
  for (; b < n_bags; b += nw) {
    const uint64_t bn = b + nw;
    int64_t sn = 0, en = 0;
    if (bn < n_bags) {
      sn = off[bn];
      en = off[bn + 1];
    }
    const int64_t cnt = e - s;
    bool ok = cnt >= 0 && cnt <= 32;
    bool want = ok && (int64_t)l < cnt;
    if (want && r >= rows) ok = false;
    uint64_t byte = (want ? r : 0) * dim * 4;
    uint64_t page = page0 + byte / kPage;
    uint32_t in = (uint32_t)(byte % kPage);
    unsigned grp = __match_any_sync(kFull, want ? page : ~0ull);
    int lead = __ffs(grp) - 1;
    bool leader = want && lead == (int)l;
    uint32_t line = 0;
    bool hit = true;
    if (leader) {
      hit = false;
      uint64_t base = (uint64_t)set_of(page, d.sets) * d.ways;
      uint64_t t = 0;
      int w = -1;
      if (d.ways == 8) {  // the set's tags in one round trip
        uint64_t pre[8];
        ld_tags8(&d.tag[base], pre);
        w = match_ready8(pre, page, t);
      } else {
        for (uint32_t k = 0; k < d.ways && w < 0; ++k) {
          uint64_t tk = ld_rlx64(&d.tag[base + k]);
          uint64_t st = tag_state(tk);
          if ((st == ST_READY || st == ST_MODIFIED) && tag_page(tk) == page) {
            w = (int)k;
            t = tk;
          }
        }
      }
      if (w >= 0) {
        line = (uint32_t)(base + w);
        hit = true;
        if (!(t & TAG_REF)) atomicOr(&d.tag[line], TAG_REF);
      }
    }
    // the next bag's indices (its offsets have arrived while the tags were read)
    uint64_t rn = 0;
    if (bn < n_bags && (int64_t)l < en - sn && en - sn <= 32) rn = (uint64_t)idx[sn + l];
    bool all = __all_sync(kFull, __all_sync(kFull, ok) && hit);
    if (!all) {
      if (l == 0) list[atomicAdd(list_n, 1u)] = (uint32_t)b;
    } else {
      stat_warp(d, S_HITS, leader ? 1u : 0u);
      stat_warp(d, S_WARP_COALESCED, (want && !leader) ? 1u : 0u);
      uint32_t myline = __shfl_sync(kFull, line, lead & 31);
      float4 acc[MF4];
#pragma unroll
      for (int c = 0; c < MF4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (uint32_t j0 = 0; j0 < (uint32_t)cnt; j0 += RB) {
        float4 v[RB][MF4];
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          uint32_t lj = __shfl_sync(kFull, myline, (j0 + jj) & 31);
          uint32_t oj = __shfl_sync(kFull, in, (j0 + jj) & 31);
          const uint8_t *rowp = line_ptr(d, lj) + oj;
#pragma unroll
          for (int c = 0; c < MF4; ++c) {
            uint32_t col = l + 32 * c;
            v[jj][c] = (j0 + jj < (uint32_t)cnt && col < nf4) ? ld_cg_f4(rowp + 16 * col)
                                                             : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          if (j0 + jj < (uint32_t)cnt) {
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
      float4 *o = (float4 *)(out + b * dim);
#pragma unroll
      for (int c = 0; c < MF4; ++c)
        if (l + 32 * c < nf4) o[l + 32 * c] = acc[c];
    }
    s = sn;
    e = en;
    r = rn;
  }
}

// ============================================================================ plain HBM gather
// The embedding bag over a table held in HBM, without the cache or the queues: the hit
// path's ceiling and the "kernel time" of its breakdown.  A warp per bag (bags
// b, b + W, ...); lane l adds the float4 columns l, l + 32, ... of the bag's rows in
// increasing index order (FP32, no fusion: the cached path's bits).  The rows of up to
// 16 indices are loaded before the first add, and the next bag's offsets are read while
// this bag's loads fly.
template <int MF4>
__global__ void __launch_bounds__(256) hbm_bag_kernel(const float *table, uint32_t rows, uint32_t dim,
                                                      const int64_t *idx, const int64_t *off, uint32_t n_bags,
                                                      float *out, int32_t *err) {
  const unsigned l = threadIdx.x & 31;
  const uint32_t nf4 = dim / 4;
  const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  constexpr int RB = MF4 >= 4 ? 4 : 16 / MF4;  // rows whose loads are in flight together
  int64_t sn = 0, en = 0;
  if (warp < n_bags) {
    sn = off[warp];
    en = off[warp + 1];
  }
  for (uint64_t b = warp; b < n_bags; b += nw) {
    const int64_t s = sn, e = en;
    if (b + nw < n_bags) {  // the next bag's offsets, in flight with this bag's loads
      sn = off[b + nw];
      en = off[b + nw + 1];
    }
    float4 acc[MF4];
#pragma unroll
    for (int c = 0; c < MF4; ++c) acc[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t i0 = s; i0 < e; i0 += 32) {
      int64_t i = i0 + l;
      uint64_t r = i < e ? (uint64_t)__ldg(&idx[i]) : 0;
      if (i < e && r >= rows) {
        atomicCAS(err, 0, 22);
        r = 0;
      }
      uint32_t cnt = (uint32_t)min((int64_t)32, e - i0);
      for (uint32_t j0 = 0; j0 < cnt; j0 += RB) {
        float4 v[RB][MF4];
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          uint64_t rj = __shfl_sync(kFull, r, (j0 + jj) & 31);
          const float4 *row = (const float4 *)(table + rj * dim);
#pragma unroll
          for (int c = 0; c < MF4; ++c) {
            uint32_t col = l + 32 * c;
            v[jj][c] = (j0 + jj < cnt && col < nf4) ? __ldg(row + col) : make_float4(0.f, 0.f, 0.f, 0.f);
          }
        }
#pragma unroll
        for (int jj = 0; jj < RB; ++jj) {
          if (j0 + jj < cnt) {
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
    float4 *o = (float4 *)(out + b * dim);
#pragma unroll
    for (int c = 0; c < MF4; ++c)
      if (l + 32 * c < nf4) o[l + 32 * c] = acc[c];
  }
}

__global__ void hbm_bag_err_kernel(Dev d, const int32_t *err) {
  if (threadIdx.x == 0 && *err) set_error(d, -(*err));
}

__global__ void bfs_init_kernel(int32_t *level, uint32_t *vis, uint32_t n, int32_t src) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i < n) level[i] = (i == (uint64_t)src) ? 0 : -1;
  if (i < (n + 31ull) / 32) vis[i] = (i == (uint64_t)src / 32) ? 1u << (src % 32) : 0u;
}

// rows a warp pins together: with `warps` warps each holding that many lines at once,
// at most half of the cache is pinned
uint32_t pin_group(const agile_ctx *c, uint32_t warps) {
  uint64_t g = c->dev.nlines / (2ull * std::max<uint32_t>(1, warps));
  return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(32, g));
}

int bfs_check(agile_ctx *c, uint64_t offsets_byte0, uint64_t cols_byte0, uint32_t n_vertices, int32_t src,
              int32_t *d_level, uint32_t mode) {
  if (!c || mode > 1 || !d_level) return AGILE_EINVAL;
  if (offsets_byte0 % kPage || cols_byte0 % kPage) return AGILE_EINVAL;
  if (n_vertices == 0 || n_vertices >= (1u << 31) || src < 0 || (uint32_t)src >= n_vertices) return AGILE_EINVAL;
  if (offsets_byte0 + ((uint64_t)n_vertices + 1) * 8 > c->cfg.store_bytes) return AGILE_EINVAL;
  if (cols_byte0 >= c->cfg.store_bytes) return AGILE_EINVAL;
  return AGILE_OK;
}

int bfs_launch(agile_ctx *c, uint64_t offsets_byte0, uint64_t cols_byte0, uint32_t n_vertices, int32_t src,
               int32_t *d_level, uint64_t *d_edges_scanned, uint32_t mode, void *stream, HubEntry *hubq,
               uint32_t hub_cap, uint32_t *vis, const int64_t *h_off = nullptr, const int32_t *h_col = nullptr) {
  cudaStream_t s = as_stream(stream);
  bfs_init_kernel<<<(n_vertices + 255) / 256, 256, 0, s>>>(d_level, vis, n_vertices, src);
  AGILE_CUDA_TRY(cudaGetLastError());
  if (d_edges_scanned) AGILE_CUDA_TRY(cudaMemsetAsync(d_edges_scanned, 0, 8, s));
  if (h_off) {
    // the CSR in HBM: offsets and columns are told apart by their (distinct) page
    // numbers 0 and 1 only
    BfsAppT<true> app{0, 1, n_vertices, d_level, (unsigned long long *)d_edges_scanned, AGILE_SYNC, hubq,
                      hub_cap, vis, (const uint8_t *)h_off, (const uint8_t *)h_col};
    return launch_engine(c, app, stream, warps_for_cache(c, 2, 32));
  }
  BfsApp app{offsets_byte0 / kPage, cols_byte0 / kPage, n_vertices, d_level,
             (unsigned long long *)d_edges_scanned, mode, hubq, hub_cap, vis};
  // about two lines per warp (one pinned, one being filled; a slice's requested pages are
  // scanned right away)
  return launch_engine(c, app, stream, warps_for_cache(c, 2, 32));
}

// ---------------------------------------------------------------- BFS without allocation
// Some callers cannot call cudaMalloc when they run a BFS: code running under stream
// capture (allocation is not allowed there), and latency-critical loops in which an
// allocation's implicit device synchronisation would stall every other stream.  For
// them agile_bfs_noalloc keeps the long-list queue, the only scratch the BFS kernel
// needs beyond the context, in this fixed device array, and the visited bitmap in a
// second one.  Every GPU that loads the library holds them (8 MiB + 4 MiB) until the
// process exits.  Host code must not pass the array's name to a kernel: on the host it
// is a stand-in symbol, not a device address, so its address is fetched once per device
// with cudaGetSymbolAddress, with that device current, on the first call on that device
// (and kept for the process: a device reset between calls is not supported).
// No queue entry needs clearing between calls: an entry is written before it is
// published, and publication carries the number the device gave the launch (one per
// kernel execution, not per host call), so what an earlier launch left behind is never
// taken for a live entry; the bitmap is cleared by every call.  All calls on one device
// share the arrays, so calls of this entry point that overlap on that GPU (from any
// context or stream) race on them.
constexpr uint32_t kNoAllocHubMax = 131072;  // entries / kHub records: graphs up to 33,554,176 entries
constexpr uint32_t kNoAllocVisWords = 1u << 20;  // vertices up to 2^25
static __device__ __align__(256) HubEntry g_bfs_hub_scratch[kNoAllocHubMax];
static __device__ __align__(256) uint32_t g_bfs_vis_scratch[kNoAllocVisWords];

int noalloc_scratch(int device, HubEntry **out, uint32_t **vis_out) {
  static std::mutex mu;
  static HubEntry *ptr[128] = {};
  static uint32_t *vptr[128] = {};
  if (device < 0 || device >= 128) return AGILE_ENODEV;
  std::lock_guard<std::mutex> g(mu);
  if (!ptr[device]) {
    void *p = nullptr, *q = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_bfs_hub_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&q, g_bfs_vis_scratch);
    if (e != cudaSuccess || !p || !q) {
      fprintf(stderr, "agile: cudaGetSymbolAddress of the BFS scratch failed: %s\n", cudaGetErrorString(e));
      return AGILE_ECUDA;
    }
    ptr[device] = (HubEntry *)p;
    vptr[device] = (uint32_t *)q;
  }
  *out = ptr[device];
  *vis_out = vptr[device];
  return AGILE_OK;
}

// Slice queue of a CSR walk (BFS, SpMV): at most `per_1024` records per 1024 column
// entries of a level -- the BFS's slices hold at least kHub = 256 entries (4), the
// SpMV's ceil(d / 1024) of a row of d >= 1024 entries at most 2 d / 1024 (2); the
// entries the store can hold beyond cols_byte0 bound them.  A reservation past the
// queue's end is still correct: the warp scans those lists itself.
int ensure_slice_entries(agile_ctx *c, uint64_t entries, uint32_t per_1024);
int ensure_slice_queue(agile_ctx *c, uint64_t cols_byte0, uint32_t per_1024 = 1) {
  return ensure_slice_entries(c, (c->cfg.store_bytes - cols_byte0) / 4, per_1024);
}
// ... the same for a list of `entries` column entries
int ensure_slice_entries(agile_ctx *c, uint64_t entries, uint32_t per_1024) {
  uint64_t cap = entries / 1024 * per_1024 + 1;
  if (cap > (1u << 22)) cap = 1u << 22;
  if (cap < 1024) cap = 1024;
  if (!c->bfs_hubq || c->bfs_hub_cap < cap) {
    if (c->bfs_hubq) cudaFree(c->bfs_hubq);
    c->bfs_hubq = nullptr;
    c->bfs_hub_cap = 0;
    AGILE_CUDA_TRY(cudaMalloc(&c->bfs_hubq, cap * sizeof(HubEntry)));
    c->bfs_hub_cap = (uint32_t)cap;
  }
  return AGILE_OK;
}

}  // namespace

extern "C" {

int agile_embedding_bag(agile_ctx *c, uint64_t table_byte0, uint32_t rows, uint32_t dim, const int64_t *d_idx,
                        const int64_t *d_offsets, uint32_t n_bags, float *d_out, uint32_t mode, void *stream) {
  if (!c || mode > 1) return AGILE_EINVAL;
  if (n_bags == 0) return AGILE_OK;
  if (!d_idx || !d_offsets || !d_out) return AGILE_EINVAL;
  if (dim == 0 || dim % 4 || dim * 4 > kPage || dim > 32 * 4 * kMaxF4) return AGILE_EINVAL;
  if (table_byte0 % kPage) return AGILE_EINVAL;
  if (table_byte0 + (uint64_t)rows * dim * 4 > c->cfg.store_bytes) return AGILE_EINVAL;
  if (((uintptr_t)d_out) & 15) return AGILE_EINVAL;
  // rows must not straddle pages: dim*4 divides the page
  if (kPage % (dim * 4)) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t st = as_stream(stream);
  // scratch: the bags the resident pass leaves to the engine, and their count
  size_t need = ((size_t)n_bags + 64) * 4;
  if (c->emb_scratch_bytes < need) {
    if (c->emb_scratch) cudaFree(c->emb_scratch);
    c->emb_scratch = nullptr;
    c->emb_scratch_bytes = 0;
    AGILE_CUDA_TRY(cudaMalloc(&c->emb_scratch, need));
    c->emb_scratch_bytes = need;
  }
  uint32_t *list_n = (uint32_t *)c->emb_scratch;
  uint32_t *list = list_n + 32;  // the count on a line of its own
  AGILE_CUDA_TRY(cudaMemsetAsync(list_n, 0, 4, st));
  // pass 1: bags whose pages are all resident, at full occupancy
  {
    auto resident = [&](auto kern) {
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
      uint64_t grid = (uint64_t)std::max(1, per_sm) * (uint64_t)c->sms;
      grid = std::min<uint64_t>(grid, ((uint64_t)n_bags + 7) / 8);
      kern<<<(uint32_t)grid, 256, 0, st>>>(c->dev, table_byte0 / kPage, rows, dim, d_idx, d_offsets, n_bags, d_out,
                                           list, list_n);
    };
    if (dim <= 128) resident(resident_bag_kernel<1>);
    else if (dim <= 256) resident(resident_bag_kernel<2>);
    else resident(resident_bag_kernel<kMaxF4>);
    AGILE_CUDA_TRY(cudaGetLastError());
  }
  // pass 2: the engine, on the bags left; one warp per bag while the rows each warp holds
  // or requests ahead fit in the cache
  uint32_t warps = std::min<uint32_t>(n_bags, warps_for_cache(c, 4, 32));
  auto go = [&](auto tag) {
    using App = decltype(tag);
    // rows requested ahead (async) and pin groups are sized by the warps that run: a
    // warp's share of the lines holds its pinned group and its lookahead.  With fewer
    // than 8 lines a warp the cache is too small for a lookahead (Sec. 4.4): a line
    // requested ahead is evicted for another warp's demand before its use, so the call
    // runs without one (as SYNC; measured on the 1,024-line cache of the 32 MiB table:
    // 8.4 M lookups/s with the lookahead, 11.7 M without, the same as SYNC).
    uint32_t run = running_app_warps<App>(c, warps);
    const bool look = mode == AGILE_ASYNC && c->dev.nlines / run >= 8;
    uint64_t ahead = look ? c->dev.nlines / (2ull * run) : 0;
    ahead = std::max<uint64_t>(1, std::min<uint64_t>(32, ahead * c->cfg.prefetch_depth));
    App app{table_byte0 / kPage, rows, dim, d_idx, d_offsets, n_bags, d_out, look ? mode : (uint32_t)AGILE_SYNC,
            (uint32_t)ahead, pin_group(c, run), list, list_n};
    return launch_engine(c, app, stream, warps);
  };
  if (dim <= 128) {
    // three CTAs per SM (fewer registers a thread, so slower service warps) pay off only
    // when the cache holds enough lines for more warps than two CTAs per SM give
    uint64_t want = c->cfg.app_warps ? c->cfg.app_warps : warps;
    if (want > (uint64_t)std::max(0, engine_grid<EmbApp<1, 2>>(c)) * (kWarps - 1)) return go(EmbApp<1, 3>{});
    return go(EmbApp<1, 2>{});
  }
  if (dim <= 256) return go(EmbApp<2>{});
  return go(EmbApp<kMaxF4>{});
}

int agile_embedding_pipeline(agile_ctx *c, uint64_t table_byte0, uint64_t table_stride, uint32_t n_tables,
                             uint32_t rows, uint32_t dim, const int64_t *d_idx, uint32_t pooling, uint32_t n_bags,
                             uint32_t n_batches, uint32_t compute_iters, float *d_out, uint32_t mode, void *stream) {
  if (!c || mode > 1) return AGILE_EINVAL;
  if (n_bags == 0 || n_batches == 0 || n_tables == 0) return AGILE_OK;
  if (!d_idx || !d_out || pooling == 0) return AGILE_EINVAL;
  if (dim == 0 || dim % 4 || dim * 4 > kPage || dim > 32 * 4 * kMaxF4 || kPage % (dim * 4)) return AGILE_EINVAL;
  if (table_byte0 % kPage || table_stride % kPage || table_stride < (uint64_t)rows * dim * 4) return AGILE_EINVAL;
  if (table_byte0 + (uint64_t)(n_tables - 1) * table_stride + (uint64_t)rows * dim * 4 > c->cfg.store_bytes)
    return AGILE_EINVAL;
  if (((uintptr_t)d_out) & 15) return AGILE_EINVAL;
  uint64_t units = (uint64_t)n_batches * n_bags;
  uint32_t per_unit = n_tables * pooling;
  // a warp per unit while the rows each warp pins or requests ahead fit in the cache:
  // half of the lines for pin groups, half for the rows requested ahead (async), at
  // most one unit ahead
  uint32_t warps = (uint32_t)std::min<uint64_t>(units, warps_for_cache(c, 4, 32));
  auto go = [&](auto tag) {
    using App = decltype(tag);
    uint32_t run = running_app_warps<App>(c, warps);
    const uint32_t group = pin_group(c, run);
    // A lookahead adds requests in flight only while the queues have room for more than
    // the warps' own demand.  The running warps' groups of rows are at most run * group
    // reads in flight, about half of that while the warps also compute; when that half
    // alone fills the queue slots, the call runs as SYNC (measured at the full grid of
    // 2,128 warps: async 0.93-1.01x sync with the lookahead, its hints mostly dropped
    // for crowded queues).
    const bool look =
        mode == AGILE_ASYNC && (uint64_t)run * group < 2ull * c->dev.Q * (c->dev.depth - 1);
    uint64_t ahead = look ? c->dev.nlines / (2ull * run) * c->cfg.prefetch_depth : 0;
    ahead = std::max<uint64_t>(1, std::min<uint64_t>(per_unit, ahead));
    App app{table_byte0 / kPage, table_stride, n_tables, rows, dim, d_idx, pooling, n_bags, n_batches,
            compute_iters, d_out, look ? mode : (uint32_t)AGILE_SYNC, group, (uint32_t)ahead};
    return launch_engine(c, app, stream, warps);
  };
  if (dim <= 128) return go(PipeApp<1>{});
  return go(PipeApp<kMaxF4>{});
}

int agile_bfs(agile_ctx *c, uint64_t offsets_byte0, uint64_t cols_byte0, uint32_t n_vertices, int32_t src,
              int32_t *d_level, uint64_t *d_edges_scanned, uint32_t mode, void *stream) {
  int r = bfs_check(c, offsets_byte0, cols_byte0, n_vertices, src, d_level, mode);
  if (r) return r;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  r = ensure_slice_queue(c, cols_byte0, 1024 / BfsApp::kHub);
  if (r) return r;
  uint64_t words = ((uint64_t)n_vertices + 31) / 32;
  if (!c->bfs_vis || c->bfs_vis_words < words) {
    if (c->bfs_vis) cudaFree(c->bfs_vis);
    c->bfs_vis = nullptr;
    AGILE_CUDA_TRY(cudaMalloc(&c->bfs_vis, words * 4));
    c->bfs_vis_words = words;
  }
  return bfs_launch(c, offsets_byte0, cols_byte0, n_vertices, src, d_level, d_edges_scanned, mode, stream,
                    (HubEntry *)c->bfs_hubq, c->bfs_hub_cap, (uint32_t *)c->bfs_vis);
}

int agile_bfs_noalloc(agile_ctx *c, uint64_t offsets_byte0, uint64_t cols_byte0, uint32_t n_vertices,
                      uint64_t n_cols, int32_t src, int32_t *d_level, uint64_t *d_edges_scanned, uint32_t mode,
                      void *stream) {
  int r = bfs_check(c, offsets_byte0, cols_byte0, n_vertices, src, d_level, mode);
  if (r) return r;
  if (n_cols > (c->cfg.store_bytes - cols_byte0) / 4) return AGILE_EINVAL;
  if (n_cols / BfsApp::kHub + 1 > kNoAllocHubMax) {
    fprintf(stderr,
            "agile_bfs_noalloc: %llu column entries need up to %llu long-list slots; this entry point "
            "has %u (graphs up to %llu column entries); use agile_bfs\n",
            (unsigned long long)n_cols, (unsigned long long)(n_cols / BfsApp::kHub + 1), kNoAllocHubMax,
            (unsigned long long)(kNoAllocHubMax - 1) * BfsApp::kHub);
    return AGILE_EINVAL;
  }
  if (((uint64_t)n_vertices + 31) / 32 > kNoAllocVisWords) {
    fprintf(stderr, "agile_bfs_noalloc: %u vertices; this entry point has a visited bitmap for up to %llu; "
            "use agile_bfs\n", n_vertices, (unsigned long long)kNoAllocVisWords * 32);
    return AGILE_EINVAL;
  }
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  HubEntry *scratch = nullptr;
  uint32_t *vis = nullptr;
  r = noalloc_scratch(c->device, &scratch, &vis);
  if (r) return r;
  return bfs_launch(c, offsets_byte0, cols_byte0, n_vertices, src, d_level, d_edges_scanned, mode, stream,
                    scratch, kNoAllocHubMax, vis);
}

int agile_embedding_bag_hbm(agile_ctx *c, const float *d_table, uint32_t rows, uint32_t dim, const int64_t *d_idx,
                            const int64_t *d_offsets, uint32_t n_bags, float *d_out, void *stream) {
  if (!c) return AGILE_EINVAL;
  if (n_bags == 0) return AGILE_OK;
  if (!d_table || !d_idx || !d_offsets || !d_out) return AGILE_EINVAL;
  if (dim == 0 || dim % 4 || dim > 32 * 4 * kMaxF4) return AGILE_EINVAL;
  if ((((uintptr_t)d_out) | ((uintptr_t)d_table)) & 15) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  // the error word lives in the context's per-launch state (flag[0]), which no launch
  // on this stream uses at the same time
  int32_t *err = (int32_t *)&c->dev.run->flag[0];
  AGILE_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
  int per_sm = 0;
  uint32_t grid;
  auto launch = [&](auto kern) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    grid = (uint32_t)std::max(1, per_sm) * (uint32_t)c->sms;
    grid = (uint32_t)std::min<uint64_t>(grid, ((uint64_t)n_bags + 7) / 8);
    kern<<<grid, 256, 0, s>>>(d_table, rows, dim, d_idx, d_offsets, n_bags, d_out, err);
  };
  if (dim <= 128) launch(hbm_bag_kernel<1>);
  else if (dim <= 256) launch(hbm_bag_kernel<2>);
  else launch(hbm_bag_kernel<kMaxF4>);
  AGILE_CUDA_TRY(cudaGetLastError());
  hbm_bag_err_kernel<<<1, 32, 0, s>>>(c->dev, err);
  AGILE_CUDA_TRY(cudaGetLastError());
  return AGILE_OK;
}

int agile_bfs_hbm(agile_ctx *c, const int64_t *d_offsets, const int32_t *d_cols, uint32_t n_vertices,
                  uint64_t n_cols, int32_t src, int32_t *d_level, uint64_t *d_edges_scanned, void *stream) {
  if (!c || !d_offsets || !d_cols || !d_level) return AGILE_EINVAL;
  if (n_vertices == 0 || n_vertices >= (1u << 31) || src < 0 || (uint32_t)src >= n_vertices) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  int r = ensure_slice_entries(c, n_cols, 1024 / BfsApp::kHub);
  if (r) return r;
  uint64_t words = ((uint64_t)n_vertices + 31) / 32;
  if (!c->bfs_vis || c->bfs_vis_words < words) {
    if (c->bfs_vis) cudaFree(c->bfs_vis);
    c->bfs_vis = nullptr;
    AGILE_CUDA_TRY(cudaMalloc(&c->bfs_vis, words * 4));
    c->bfs_vis_words = words;
  }
  return bfs_launch(c, 0, 0, n_vertices, src, d_level, d_edges_scanned, AGILE_SYNC, stream,
                    (HubEntry *)c->bfs_hubq, c->bfs_hub_cap, (uint32_t *)c->bfs_vis, d_offsets, d_cols);
}

int agile_spmv_hbm(agile_ctx *c, const int64_t *d_offsets, const int32_t *d_cols, const float *d_vals,
                   uint32_t n_rows, uint32_t n_cols, uint64_t n_entries, const float *d_x, float *d_y,
                   uint64_t *d_entries, void *stream) {
  if (!c) return AGILE_EINVAL;
  if (n_rows == 0) return AGILE_OK;
  if (!d_offsets || !d_cols || !d_vals || !d_x || !d_y) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  int r = ensure_slice_entries(c, n_entries, 2);
  if (r) return r;
  if (d_entries) AGILE_CUDA_TRY(cudaMemsetAsync(d_entries, 0, 8, as_stream(stream)));
  SpmvAppT<true> app{0, 1, 2, n_rows, d_x, n_cols, d_y, (unsigned long long *)d_entries, AGILE_SYNC,
                     (HubEntry *)c->bfs_hubq, c->bfs_hub_cap, (const uint8_t *)d_offsets, (const uint8_t *)d_cols,
                     (const uint8_t *)d_vals};
  return launch_engine(c, app, stream, warps_for_cache(c, 3, 32));
}

int agile_spmv(agile_ctx *c, uint64_t offsets_byte0, uint64_t cols_byte0, uint64_t vals_byte0, uint32_t n_rows,
               uint32_t n_cols, const float *d_x, float *d_y, uint64_t *d_entries, uint32_t mode, void *stream) {
  if (!c || mode > 1) return AGILE_EINVAL;
  if (n_rows == 0) return AGILE_OK;
  if (!d_x || !d_y) return AGILE_EINVAL;
  if (offsets_byte0 % kPage || cols_byte0 % kPage || vals_byte0 % kPage) return AGILE_EINVAL;
  if (offsets_byte0 + ((uint64_t)n_rows + 1) * 8 > c->cfg.store_bytes) return AGILE_EINVAL;
  if (cols_byte0 >= c->cfg.store_bytes || vals_byte0 >= c->cfg.store_bytes) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  int r = ensure_slice_queue(c, std::min(cols_byte0, vals_byte0), 2);
  if (r) return r;
  if (d_entries) AGILE_CUDA_TRY(cudaMemsetAsync(d_entries, 0, 8, as_stream(stream)));
  SpmvApp app{offsets_byte0 / kPage, cols_byte0 / kPage, vals_byte0 / kPage, n_rows, d_x, n_cols, d_y,
              (unsigned long long *)d_entries, mode, (HubEntry *)c->bfs_hubq, c->bfs_hub_cap};
  // each warp pins one page of each of three arrays and requests up to two units ahead
  return launch_engine(c, app, stream, warps_for_cache(c, mode == AGILE_ASYNC ? 6 : 3, 32));
}

}  // extern "C"
