// A user kernel built against include/agile_device.cuh (test of the synchronous row
// read): warp w reads requests w, w + W, ... with get_row, each into its own 4096-byte
// slot of dst.
#include <cstdint>

#include "agile_device.cuh"

namespace {

struct RowDemo {
  const uint64_t *pages;
  const uint32_t *offs;
  const uint32_t *lens;
  uint32_t n;
  uint8_t *dst;  // n * 4096 bytes

  __device__ void run(const agile::Dev &d, const agile::AppCtx &a) const {
    for (uint64_t i = a.warp; i < n; i += a.n_warps)
      if (!agile::dev::get_row(d, a, pages[i], offs[i], lens[i], dst + i * 4096)) return;
  }
};

}  // namespace

extern "C" int row_demo(agile_ctx *ctx, const uint64_t *pages, const uint32_t *offs, const uint32_t *lens,
                        uint32_t n, uint8_t *dst, uint32_t app_warps, void *stream) {
  RowDemo app{pages, offs, lens, n, dst};
  return agile::launch_user(ctx, app, stream, app_warps);
}
