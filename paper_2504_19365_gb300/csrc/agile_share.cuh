// Share Table of user buffers (Sec. 3.4.1): user-specified buffers are shared by
// pointer between the threads that ask for the same page, with a reference count and
// MOESI-inspired states, and a modified buffer is propagated into the software cache
// once its last user lets it go.
//
// An entry maps page -> the buffer that holds it; its meta word is
//   {state:8 | count:32 | closing:1}  with states
//   PENDING (being filled; others may join and wait for the fill's token),
//   E (one user, clean), S (several, clean), M (one user, modified), O (several,
//   modified).
// acquire(page, mine): an entry of the page is joined (count + 1; E -> S, M -> O) and its
//   buffer returned; otherwise `mine` is registered and filled -- copied from the page's
//   cache line when the cache holds it, else read from the store straight into `mine`
//   (the cache is left as it is).  While the fill is set up the filler owns the page's
//   in-flight entry (Sec. 3.4.1's table of requests in flight), so no write of the page
//   and no cache fill of it can pass it.
// modified(page): the caller changed the shared buffer: E -> M, S -> O.
// release(page): count - 1; the last user of a modified buffer writes it into the
//   page's cache line (claimed, or pinned when resident), which turns MODIFIED, and the
//   entry goes away.  The paper gives this duty to the buffer's owner after the other
//   users finish; here whoever releases last does it, so that nobody waits for others.
// No lane waits while it holds a cache line; a lane that must retry holds at most the
// table entry it is setting up or closing (threads that want that page wait for it) and
// the page's in-flight entry, which no cache line's release depends on.
#pragma once
#include <cuda_runtime.h>

#include "agile.h"
#include "agile_dev.cuh"

namespace agile {

constexpr uint64_t UB_E = 1, UB_S = 2, UB_M = 3, UB_O = 4, UB_PENDING = 5;
constexpr uint64_t UB_CLOSING = 1ull << 40;

static __device__ __forceinline__ uint64_t ub_state(uint64_t m) { return m & 0xFFull; }
static __device__ __forceinline__ uint32_t ub_count(uint64_t m) { return (uint32_t)(m >> 8); }
static __device__ __forceinline__ uint64_t ub_make(uint64_t st, uint32_t cnt) { return st | ((uint64_t)cnt << 8); }

static __device__ __forceinline__ uint64_t ub_base(const Dev &d, uint64_t page) {
  uint64_t h = (page ^ 0x5851F42D4C957F2Dull) * 0x9E3779B97F4A7C15ull;
  return (uint64_t)((uint32_t)(h >> 35) & d.ub_mask) * 4;
}

// slot of the page's entry, -1 if none
static __device__ __forceinline__ int64_t ub_find(const Dev &d, uint64_t page) {
  uint64_t base = ub_base(d, page);
  for (int k = 0; k < 4; ++k)
    if (ld_acq64(&d.ub_key[base + k]) == page + 1) return (int64_t)(base + k);
  return -1;
}

// Claim a free slot for the page: >= 0 the slot (its buffer word is set and its meta
// published as PENDING with count 1), -1 the page has an entry (or a racing insert of
// it won), -2 the bucket is full.
static __device__ int64_t ub_insert(const Dev &d, uint64_t page, uint64_t buf) {
  uint64_t key = page + 1, base = ub_base(d, page);
  for (int tries = 0; tries < 8; ++tries) {
    int free_k = -1;
    for (int k = 0; k < 4; ++k) {
      uint64_t v = ld_acq64(&d.ub_key[base + k]);
      if (v == key) return -1;
      if (v == 0 && free_k < 0) free_k = k;
    }
    if (free_k < 0) return -2;
    if (atomicCAS(&d.ub_key[base + free_k], 0ull, (unsigned long long)key) != 0ull) continue;
    fence_sc();
    for (int k = 0; k < 4; ++k) {
      if (k != free_k && ld_acq64(&d.ub_key[base + k]) == key) {
        st_rel64(&d.ub_key[base + free_k], 0ull);
        return -1;
      }
    }
    st_rlx64(&d.ub_buf[base + free_k], buf);
    st_rlx64(&d.ub_tok[base + free_k], 0ull);
    st_rel64(&d.ub_meta[base + free_k], ub_make(UB_PENDING, 1));
    return (int64_t)(base + free_k);
  }
  return -2;
}

// Join the entry in slot k: true when the count went up (meta 0 = being set up or
// taken down, closing = going away: try again later).
static __device__ __forceinline__ bool ub_join(const Dev &d, uint64_t k) {
  uint64_t m = ld_acq64(&d.ub_meta[k]);
  if (m == 0 || (m & UB_CLOSING)) return false;
  uint64_t st = ub_state(m);
  uint64_t nst = st == UB_E ? UB_S : (st == UB_M ? UB_O : st);
  return atomicCAS(&d.ub_meta[k], (unsigned long long)m, (unsigned long long)ub_make(nst, ub_count(m) + 1)) == m;
}

// The filler publishes the fill's token, then turns PENDING into E (or S when others
// joined meanwhile).
static __device__ __forceinline__ void ub_ready(const Dev &d, uint64_t k, uint64_t tok) {
  st_rel64(&d.ub_tok[k], tok);
  uint64_t m = ld_acq64(&d.ub_meta[k]);
  for (;;) {
    uint32_t c = ub_count(m);
    uint64_t nm = ub_make(c > 1 ? UB_S : UB_E, c);
    uint64_t got = atomicCAS(&d.ub_meta[k], (unsigned long long)m, (unsigned long long)nm);
    if (got == m) return;
    m = got;
  }
}

// One attempt to fill the new entry k of `page` into `mine`: 1 done (*tok set; *ring
// when a read command was committed to `is`), 0 try again later.
static __device__ int ub_fill(const Dev &d, const AppCtx &a, uint64_t page, uint8_t *mine, uint64_t k, uint64_t &tok,
                       Issued &is, bool &ring) {
  int64_t sh = sh_insert(d, page, SH_FILL);
  if (sh < 0) return 0;  // the page is in flight (a fill or a write-back): later
  uint32_t line = 0;
  int pr = cache_probe(d, page, true, line);
  if (pr == P_HIT) {
    lane_copy_page(mine, line_ptr(d, line));
    fence_ar();
    cache_unpin(d, line);
    sh_remove(d, (uint64_t)sh);
    tok = ~0ull;
    ub_ready(d, k, tok);
    return 1;
  }
  if (pr == P_BUSY) {
    sh_remove(d, (uint64_t)sh);
    return 0;
  }
  uint32_t q = 0, slot = 0, ticket = 0;
  if (!sq_reserve_dev(d, a.q0, dev_of_page(d, page), 1, q, slot, ticket)) {
    sh_remove(d, (uint64_t)sh);
    return 0;
  }
  sq_commit(d, q, slot, ticket, OP_READ, (uint64_t)mine, page, ctx_make(CTX_BUF, (uint32_t)sh, 0));
  atomicAdd(stat_ptr(d, S_MISSES), 1ull);
  tok = make_token(q, slot, ticket);
  is.q = q;
  is.slot = slot;
  is.ticket = ticket;
  ring = true;
  ub_ready(d, k, tok);
  return 1;
}

// One attempt to write the buffer of a closing modified entry into the page's cache
// line: 1 done, 0 try again later.  `sh` keeps the page's in-flight entry across
// attempts (-1: not taken yet); a write-back of the line's victim may be committed to
// `is` (*ring).
static __device__ int ub_propagate(const Dev &d, const AppCtx &a, uint64_t page, const uint8_t *buf, int64_t &sh, Issued &is,
                            bool &ring) {
  if (sh < 0) {
    sh = sh_insert(d, page, SH_WRITE);
    if (sh < 0) return 0;
  }
  uint32_t line = 0;
  int pr = cache_probe(d, page, true, line);
  if (pr == P_HIT) {
    lane_copy_page(line_ptr(d, line), buf);
    fence_ar();
    uint64_t old = atomicOr(&d.tag[line], 1ull);  // READY (2) -> MODIFIED (3)
    if (tag_state(old) == ST_READY) note_dirty(d, page);
    cache_unpin(d, line);
    sh_remove(d, (uint64_t)sh);
    sh = -1;
    return 1;
  }
  if (pr == P_BUSY) return 0;
  int m = cache_miss(d, page, a.q0, line, is, false, sh);
  if (m != M_ISSUED) return 0;
  ring = is.q != 0xFFFFFFFFu;  // a MODIFIED victim's write-back
  lane_copy_page(line_ptr(d, line), buf);
  fence_ar();
  atomicAdd(&d.tag[line], 2ull);  // BUSY (1) -> MODIFIED (3)
  note_dirty(d, page);
  sh_remove(d, (uint64_t)sh);
  sh = -1;
  return 1;
}


// Warp-collective acquire: lanes with `want` ask for `page` into their buffer `mine`
// (4096 bytes, 16-byte aligned device memory).  *buf_out receives the buffer that holds
// the page (mine, or the buffer of the entry joined) and the return value the token of
// its fill (AGILE_TOKEN_HIT when it was copied from the cache): wait on it before
// reading the buffer.  Returns 0, AGILE_EAGAIN (the table's bucket is full: nothing
// acquired) or AGILE_ETIMEDOUT per lane.
static __device__ int share_acquire(const Dev &d, const AppCtx &a, bool want, uint64_t page, uint8_t *mine,
                             uint8_t **buf_out, uint64_t *tok_out) {
  int phase = want ? 0 : 3;  // 0 find or insert, 1 fill (this lane inserted), 2 wait for the token, 3 done
  int rc = 0;
  int64_t k = -1;
  uint64_t tok = ~0ull;
  uint32_t ns = 64;
  while (__any_sync(kFull, phase < 3)) {
    bool ring = false;
    Issued is{};
    is.q = 0xFFFFFFFFu;
    bool moved = false;
    if (phase == 0) {
      k = ub_find(d, page);
      if (k >= 0) {
        if (ub_join(d, (uint64_t)k)) {
          phase = 2;
          moved = true;
        }
      } else {
        k = ub_insert(d, page, (uint64_t)mine);
        if (k >= 0) {
          phase = 1;
          moved = true;
        } else if (k == -2) {
          rc = AGILE_EAGAIN;
          phase = 3;
        }
      }
    }
    if (phase == 1) {
      if (ub_fill(d, a, page, mine, (uint64_t)k, tok, is, ring)) {
        phase = 3;
        moved = true;
      }
    } else if (phase == 2) {
      // the fill's token is published before the entry leaves PENDING (any token value,
      // 0 included, is a valid token)
      if (ub_state(ld_acq64(&d.ub_meta[k])) != UB_PENDING) {
        tok = ld_rlx64(&d.ub_tok[k]);
        phase = 3;
      }
    }
    warp_ring(d, ring, is.q, is.slot, is.ticket, a.deadline);
    if (phase < 3 && !moved && gtimer() > a.deadline) {
      rc = AGILE_ETIMEDOUT;  // an entry set up by this lane stays PENDING: the launch is failing anyway
      set_error(d, -110);
      phase = 3;
    }
    if (__any_sync(kFull, phase < 3 && !moved)) backoff(ns, 1024);
  }
  if (want && rc == 0) {
    *buf_out = (uint8_t *)ld_rlx64(&d.ub_buf[k]);
    *tok_out = tok;
  }
  return want ? rc : 0;
}

// The lane changed the buffer it acquired for `page`: E -> M, S -> O.
static __device__ void share_modified(const Dev &d, bool want, uint64_t page) {
  if (!want) return;
  int64_t k = ub_find(d, page);
  if (k < 0) return;
  uint64_t m = ld_acq64(&d.ub_meta[k]);
  for (;;) {
    uint64_t st = ub_state(m);
    uint64_t nst = st == UB_E ? UB_M : (st == UB_S ? UB_O : st);
    if (nst == st) return;
    uint64_t got = atomicCAS(&d.ub_meta[k], (unsigned long long)m, (unsigned long long)((m & ~0xFFull) | nst));
    if (got == m) return;
    m = got;
  }
}

// Warp-collective release of the lanes' references to `page`.  The last reference of a
// modified buffer writes the buffer into the page's cache line (MODIFIED) before the
// entry goes away.  Returns, per lane, 1 when this lane propagated the buffer, 0 when
// not, AGILE_ETIMEDOUT when the launch's deadline passed first.
static __device__ int share_release(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  int phase = want ? 0 : 2;  // 0 drop the reference, 1 propagate then take the entry down, 2 done
  int rc = 0;
  int64_t k = -1, sh = -1;
  const uint8_t *buf = nullptr;
  uint32_t ns = 64;
  while (__any_sync(kFull, phase < 2)) {
    bool ring = false;
    Issued is{};
    is.q = 0xFFFFFFFFu;
    bool moved = false;
    if (phase == 0) {
      k = ub_find(d, page);
      if (k < 0) {
        phase = 2;  // nothing held
      } else {
        uint64_t m = ld_acq64(&d.ub_meta[k]);
        uint32_t c = ub_count(m);
        if (c > 1) {
          if (atomicCAS(&d.ub_meta[k], (unsigned long long)m, (unsigned long long)ub_make(ub_state(m), c - 1)) == m) {
            phase = 2;
            moved = true;
          }
        } else if (c == 1 && !(m & UB_CLOSING)) {
          if (atomicCAS(&d.ub_meta[k], (unsigned long long)m, (unsigned long long)(ub_state(m) | UB_CLOSING)) == m) {
            moved = true;
            uint64_t st = ub_state(m);
            buf = (const uint8_t *)ld_rlx64(&d.ub_buf[k]);
            phase = (st == UB_M || st == UB_O) ? 1 : 3;
          }
        }
      }
    }
    if (phase == 1 && ub_propagate(d, a, page, buf, sh, is, ring)) {
      rc = 1;
      phase = 3;
      moved = true;
    }
    if (phase == 3) {  // take the entry down: meta first, then the key
      st_rlx64(&d.ub_buf[k], 0ull);
      st_rlx64(&d.ub_tok[k], 0ull);
      st_rel64(&d.ub_meta[k], 0ull);
      st_rel64(&d.ub_key[k], 0ull);
      phase = 2;
    }
    warp_ring(d, ring, is.q, is.slot, is.ticket, a.deadline);
    if (phase < 2 && !moved && gtimer() > a.deadline) {
      rc = AGILE_ETIMEDOUT;
      set_error(d, -110);
      phase = 2;
    }
    if (__any_sync(kFull, phase < 2 && !moved)) backoff(ns, 1024);
  }
  return rc;
}

// (state, count) of the page's entry, (0, 0) when there is none
static __device__ void share_entry(const Dev &d, uint64_t page, int32_t &state, int32_t &count) {
  int64_t k = ub_find(d, page);
  uint64_t m = k >= 0 ? ld_acq64(&d.ub_meta[k]) : 0;
  state = (int32_t)ub_state(m);
  count = (int32_t)ub_count(m);
}

}  // namespace agile
