// Share Table host side (Sec. 3.4.1) and the lock-order checker (Sec. 3.5).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "agile.h"
#include "agile_ctx.cuh"
#include "agile_dev.cuh"
#include "agile_share.cuh"

using namespace agile;

namespace {

// Validation: one lane runs the operations strictly one after the other, so the table
// must make the decisions of the sequential Share Table.  ops[4i..4i+3] = {op, page, a,
// b}: op 0 acquire into buffer a, 1 write 16 bytes of value b at offset a into the
// page's buffer (then mark it modified), 2 release.  out[3i..3i+2] = {acquire: index of
// the buffer returned, release: 1 when it propagated the buffer; the entry's state and
// count afterwards}.
struct ShareReplayApp {
  const int32_t *ops;
  uint32_t n;
  uint8_t *bufs;
  int32_t *out;
  __device__ void run(const Dev &d, const AppCtx &a) const {
    if (a.warp != 0) return;
    unsigned l = lane_id();
    for (uint32_t i = 0; i < n; ++i) {
      int32_t op = ops[4 * i], b = ops[4 * i + 3];
      uint64_t page = (uint64_t)(uint32_t)ops[4 * i + 1];
      int32_t a_ = ops[4 * i + 2];
      int32_t ret = -1;
      if (op == 0) {
        uint8_t *buf = nullptr;
        uint64_t tok = 0;
        int rc = share_acquire(d, a, l == 0, page, bufs + (uint64_t)a_ * kPage, &buf, &tok);
        if (l == 0 && rc == 0) {
          if (api_wait(d, tok, a.deadline) != 0) set_error(d, -110);
          ret = (int32_t)((buf - bufs) / kPage);
        }
      } else if (op == 1) {
        if (l == 0) {
          int64_t k = ub_find(d, page);
          if (k >= 0) {
            uint8_t *buf = (uint8_t *)ld_rlx64(&d.ub_buf[k]);
            for (int j = 0; j < 16; ++j) buf[a_ + j] = (uint8_t)b;
            __threadfence();
          }
          share_modified(d, true, page);
        }
      } else {
        ret = share_release(d, a, l == 0, page);
      }
      if (l == 0) {
        int32_t st = 0, cnt = 0;
        share_entry(d, page, st, cnt);
        out[3 * i] = ret;
        out[3 * i + 1] = st;
        out[3 * i + 2] = cnt;
      }
      __syncwarp();
    }
  }
};

}  // namespace

extern "C" {

int agile_share_replay(agile_ctx *c, const int32_t *d_ops, uint32_t n, void *d_bufs, int32_t *d_out, void *stream) {
  if (!c || (n && (!d_ops || !d_bufs || !d_out))) return AGILE_EINVAL;
  if (!c->dev.ub_key) return AGILE_EINVAL;
  if (((uintptr_t)d_bufs) & 15) return AGILE_EINVAL;
  if (n == 0) return AGILE_OK;
  ShareReplayApp app{d_ops, n, (uint8_t *)d_bufs, d_out};
  return launch_engine(c, app, stream, 1);
}

// Lock-order checker.  Each blocking acquire of lock L by a thread that holds the locks
// H adds the order edges h -> L (h in H); a try-acquire adds none (it never waits).
// A cycle among the edges is an order in which threads can wait for each other forever;
// re-acquiring a lock the thread holds is a cycle of one.  Returns the number of
// blocking acquires that closed a cycle (0: the order is consistent) or AGILE_EINVAL;
// the first cycle found goes to cycle_out (up to cap locks), its length to *cycle_len.
int agile_lock_order_check(const agile_lock_event *ev, uint64_t n, uint64_t *cycle_out, uint32_t cap,
                           uint32_t *cycle_len) {
  if ((n && !ev) || (cap && !cycle_out)) return AGILE_EINVAL;
  std::unordered_map<uint32_t, std::vector<uint64_t>> held;                 // thread -> locks, in order
  std::unordered_map<uint64_t, std::unordered_set<uint64_t>> after;        // lock -> locks taken after it
  int found = 0;
  bool have = false;
  if (cycle_len) *cycle_len = 0;
  // path from `from` to `to` along the edges (depth-first), into `path`
  auto reach = [&](uint64_t from, uint64_t to, std::vector<uint64_t> &path) {
    std::unordered_set<uint64_t> seen;
    std::vector<std::pair<uint64_t, std::vector<uint64_t>>> stack{{from, {from}}};
    while (!stack.empty()) {
      auto [u, p] = stack.back();
      stack.pop_back();
      if (u == to) {
        path = p;
        return true;
      }
      if (!seen.insert(u).second) continue;
      auto it = after.find(u);
      if (it == after.end()) continue;
      for (uint64_t v : it->second) {
        std::vector<uint64_t> q = p;
        q.push_back(v);
        stack.push_back({v, q});
      }
    }
    return false;
  };
  for (uint64_t i = 0; i < n; ++i) {
    const agile_lock_event &e = ev[i];
    auto &h = held[e.thread];
    if (e.op == AGILE_LOCK_RELEASE) {
      for (size_t j = h.size(); j-- > 0;)
        if (h[j] == e.lock) {
          h.erase(h.begin() + (long)j);
          break;
        }
      continue;
    }
    if (e.op == AGILE_LOCK_ACQUIRE) {
      for (uint64_t x : h) {
        std::vector<uint64_t> path;
        // a new edge x -> L closes a cycle when L already reaches x (or L == x)
        if (x == e.lock || reach(e.lock, x, path)) {
          ++found;
          if (!have) {
            have = true;
            if (x == e.lock) path = {x};
            uint32_t k = (uint32_t)std::min<size_t>(path.size(), cap);
            for (uint32_t j = 0; j < k; ++j) cycle_out[j] = path[j];
            if (cycle_len) *cycle_len = (uint32_t)path.size();
          }
          break;
        }
      }
      for (uint64_t x : h)
        if (x != e.lock) after[x].insert(e.lock);
    } else if (e.op != AGILE_LOCK_TRY) {
      return AGILE_EINVAL;
    }
    h.push_back(e.lock);
  }
  return found;
}

}  // extern "C"
