// A user kernel built against include/agile_device.cuh (test of the Share Table):
// request i asks for page pages[i] into its own buffer slot i.  Every request acquires
// before any is released (a grid barrier in between), so requests for one page share
// one buffer.  The request that owns the buffer (slot == i) then writes a mark into it;
// after a second barrier every request reads the mark through the shared pointer, then
// releases; the last release of each page writes the buffer into the cache.
#include <cstdint>

#include "agile_device.cuh"

namespace {

struct ShareDemo {
  const uint64_t *pages;
  uint32_t n;
  uint8_t *bufs;      // n * 4096
  int32_t *used;      // buffer slot each request got
  uint64_t *first8;   // first 8 bytes it read before the marks
  int32_t *mark_seen; // 1 when it read the owner's mark
  int32_t *propagated;

  __device__ void run(const agile::Dev &d, const agile::AppCtx &a) const {
    unsigned l = threadIdx.x & 31;
    // one request per lane: the launch runs exactly ceil(n / 32) application warps
    uint64_t i = (uint64_t)a.warp * 32 + l;
    bool want = i < n;
    uint64_t page = want ? pages[i] : 0;
    uint8_t *buf = nullptr;
    uint64_t tok = 0;
    int rc = agile::dev::share_acquire(d, a, want, page, bufs + i * 4096, &buf, &tok);
    if (want && rc == 0 && agile::dev::wait(d, tok, agile::dev::now() + 2000000000ull) == 0) {
      used[i] = (int32_t)((buf - bufs) / 4096);
      first8[i] = *(volatile uint64_t *)buf;
    } else if (want) {
      used[i] = -1 - rc;
    }
    if (!agile::dev::barrier(d, a)) return;
    bool owner = want && used[i] == (int32_t)i;
    if (owner) {
      for (int j = 0; j < 16; ++j) buf[32 + j] = (uint8_t)((page & 0xFF) ^ 0x5A);
      __threadfence();
    }
    agile::dev::share_modified(d, owner, page);
    if (!agile::dev::barrier(d, a)) return;
    if (want && used[i] >= 0) mark_seen[i] = ((volatile uint8_t *)buf)[40] == (uint8_t)((page & 0xFF) ^ 0x5A);
    int pr = agile::dev::share_release(d, a, want && used[i] >= 0, page);
    if (want) propagated[i] = pr;
  }
};

}  // namespace

extern "C" int share_demo(agile_ctx *ctx, const uint64_t *pages, uint32_t n, uint8_t *bufs, int32_t *used,
                          uint64_t *first8, int32_t *mark_seen, int32_t *propagated, void *stream) {
  ShareDemo app{pages, n, bufs, used, first8, mark_seen, propagated};
  return agile::launch_user(ctx, app, stream, (n + 31) / 32);
}
