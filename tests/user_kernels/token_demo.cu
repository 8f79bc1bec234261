// A user kernel built against include/agile_device.cuh (test of the device-side API):
// every lane requests one page, computes while the read is in flight, tests its token
// right after the request, waits for it with a bound, and copies the page to its slot
// of dst once the token is done.
#include <cstdint>

#include "agile_device.cuh"

namespace {

struct TokenDemo {
  const uint64_t *pages;
  uint32_t n;
  uint8_t *dst;        // n * 4096 bytes
  int32_t *status;     // wait result per request
  int32_t *pending;    // test result right after the request
  uint64_t wait_ns;    // bound of each wait
  uint32_t iters;      // work done between the request and the wait
  float *work;         // its result per request

  __device__ void run(const agile::Dev &d, const agile::AppCtx &a) const {
    unsigned l = threadIdx.x & 31;
    for (uint64_t base = (uint64_t)a.warp * 32; base < n; base += (uint64_t)a.n_warps * 32) {
      uint64_t i = base + l;
      bool want = i < n;
      uint64_t page = want ? pages[i] : 0;
      uint64_t tok = agile::dev::issue_read(d, a, want, page);
      if (want) pending[i] = agile::dev::test(d, tok);
      float x = want ? (float)(i & 1023) : 0.f;
      for (uint32_t k = 0; k < iters; ++k) x = __fmaf_rn(x, 0.999755859375f, 0.0009765625f);
      if (want) work[i] = x;
      int st = want ? agile::dev::wait(d, tok, agile::dev::now() + wait_ns) : 1;
      if (want) status[i] = st;
      for (uint32_t j = 0; j < 32 && base + j < n; ++j) {
        int sj = __shfl_sync(0xffffffffu, st, j);
        uint64_t pj = __shfl_sync(0xffffffffu, page, j);
        if (sj == 0 && !agile::dev::copy_page(d, a, pj, dst + (base + j) * 4096)) return;
      }
    }
  }
};

}  // namespace

extern "C" int token_demo(agile_ctx *ctx, const uint64_t *pages, uint32_t n, uint8_t *dst, int32_t *status,
                          int32_t *pending, uint64_t wait_ns, uint32_t iters, float *work, uint32_t app_warps,
                          void *stream) {
  TokenDemo app{pages, n, dst, status, pending, wait_ns, iters, work};
  return agile::launch_user(ctx, app, stream, app_warps);
}
