/*
 * agile_device.cuh -- device-side API of the AGILE page I/O library for user kernels
 * (sm_103a; include with -I <package>/csrc as well, and compile with nvcc -std=c++17).
 *
 * The paper's GPU program (Listing 1, Sec. 3.5) issues asyncRead for a block into a
 * buffer, continues with other work, waits for the transfer (buf.wait) and uses the
 * data; prefetch fills the cache without waiting.  Here a user kernel is a struct
 *
 *     struct MyApp { __device__ void run(const agile::Dev &d, const agile::AppCtx &a) const; };
 *
 * whose run() is executed by every application warp of a library launch
 * (agile::launch_user below), side by side with the warps that serve the queues: the
 * emulated device and the completion pollers of Alg. 1 run in the same cooperative
 * launch, so nothing waits on another launch.  Inside run():
 *
 *   uint64_t tok = agile::dev::issue_read(d, a, want, page);   // warp-collective
 *       lanes with `want` request store page `page`; equal pages are merged within the
 *       warp (Sec. 3.3.2).  Returns the lane's token: AGILE_TOKEN_HIT when the page was
 *       READY in the cache, else the token of the read that fills it (issued by this
 *       call, or already in flight -- Sec. 3.4 case (c)).  Never waits for data.
 *   int st = agile::dev::test(d, tok);        // 1 in flight, 0 done, AGILE_EIO error
 *   int st = agile::dev::wait(d, tok, deadline_ns);
 *       the per-request transaction barrier (Sec. 3.2.1), bounded: 0 done, AGILE_EIO,
 *       or AGILE_ETIMEDOUT once %globaltimer passes deadline_ns (agile::dev::now()).
 *       A timeout is returned to the caller only (the launch itself still drains the
 *       read before it ends).  The caller must hold no cache line while it waits; the
 *       API never leaves one pinned between calls.
 *   bool ok = agile::dev::copy_page(d, a, page, dst);   // warp-collective, uniform page
 *       copy the page from its cache line to dst (4096 bytes, 16-byte aligned), the
 *       line pinned for the copy only; a page evicted since its read completed is read
 *       again.  False if the launch timed out.
 *   bool ok = agile::dev::prefetch(d, a, want, page);   // Listing 1 Method-1
 *   bool ok = agile::dev::get_row(d, a, page, off, nbytes, dst);  // warp-collective
 *       the synchronous read of a row: bytes [off, off + nbytes) of the page (4-byte
 *       aligned, within the page) copied to dst, the line pinned for the copy only and
 *       read from the store first if it is not resident.  False if the launch timed
 *       out or the arguments are out of range (AGILE_EINVAL, reported by agile_check).
 *
 * a.warp / a.n_warps give the warp's index among the application warps; a.deadline is
 * the launch's own bound (cfg.wait_timeout_ns after the start).
 *
 * Host side:  int rc = agile::launch_user(ctx, app, stream, app_warps);
 *   launches `app` on `stream` over the context's queues and cache (all of the grid's
 *   application warps when app_warps is 0, else that many).  Returns 0 or an AGILE_E*
 *   code; errors found on the GPU are reported by agile_check.  One library launch at a
 *   time may use a context (calls that overlap on the GPU race).
 */
#ifndef AGILE_DEVICE_CUH
#define AGILE_DEVICE_CUH

#include <cuda_runtime.h>

#include "agile.h"
#include "agile_dev.cuh"
#include "agile_share.cuh"

namespace agile {
namespace dev {

__device__ __forceinline__ uint64_t now() { return gtimer(); }

__device__ __forceinline__ uint64_t issue_read(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  return api_issue_read(d, a, want, page);
}
__device__ __forceinline__ int test(const Dev &d, uint64_t tok) { return api_test(d, tok); }
__device__ __forceinline__ int wait(const Dev &d, uint64_t tok, uint64_t deadline_ns) {
  return api_wait(d, tok, deadline_ns);
}
__device__ __forceinline__ bool copy_page(const Dev &d, const AppCtx &a, uint64_t page, void *dst) {
  return api_copy_page(d, a, page, dst);
}
__device__ __forceinline__ bool prefetch(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  return api_prefetch(d, a, want, page);
}
__device__ __forceinline__ bool get_row(const Dev &d, const AppCtx &a, uint64_t page, uint32_t off, uint32_t nbytes,
                                        void *dst) {
  return api_get_row(d, a, page, off, nbytes, dst);
}

// Share Table (Sec. 3.4.1; the context needs cfg.share_slots > 0), warp-collective.
// share_acquire: lanes with `want` ask for `page` in their user buffer `mine` (4096
//   bytes, 16-byte aligned).  If another user holds the page in a buffer, that buffer is
//   shared (by pointer: *buf is it) and its count goes up; else `mine` is registered and
//   filled from the cache or the store.  *tok: wait on it before reading *buf.  Returns
//   0, AGILE_EAGAIN (table bucket full) or AGILE_ETIMEDOUT.
// share_modified: the lane wrote into the shared buffer of `page`.
// share_release: drop the lane's reference; the last one of a modified buffer writes it
//   into the page's cache line (MODIFIED; the store gets it by write-back).  Returns 1
//   when this lane did that, 0 when not, AGILE_ETIMEDOUT on a timeout.
__device__ __forceinline__ int share_acquire(const Dev &d, const AppCtx &a, bool want, uint64_t page, void *mine,
                                             uint8_t **buf, uint64_t *tok) {
  return agile::share_acquire(d, a, want, page, (uint8_t *)mine, buf, tok);
}
__device__ __forceinline__ void share_modified(const Dev &d, bool want, uint64_t page) {
  agile::share_modified(d, want, page);
}
__device__ __forceinline__ int share_release(const Dev &d, const AppCtx &a, bool want, uint64_t page) {
  return agile::share_release(d, a, want, page);
}
// grid barrier over the launch's application warps (every one must call it)
__device__ __forceinline__ bool barrier(const Dev &d, const AppCtx &a) { return app_barrier(d, a.n_warps, a.deadline); }

}  // namespace dev

// Launch a user application over a context (see the comment at the top).
template <class App>
int launch_user(agile_ctx *ctx, const App &app, void *stream, uint32_t app_warps = 0) {
  Dev d;
  int r = agile_device_view(ctx, &d, sizeof(Dev));
  if (r) return r;
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AGILE_ECUDA;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return AGILE_ECUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel<App>, kThreads, 0) != cudaSuccess ||
      per_sm <= 0)
    return AGILE_ECUDA;
  d.app_active = app_warps;
  if (d.extra_engines == 0xFFFFFFFFu) d.extra_engines = (uint32_t)(per_sm * sms);  // default: one per CTA
  r = agile_run_reset(ctx, stream);
  if (r) return r;
  App a = app;
  void *args[] = {(void *)&d, (void *)&a};
  if (cudaLaunchCooperativeKernel((const void *)engine_kernel<App>, dim3(per_sm * sms), dim3(kThreads), args, 0,
                                  (cudaStream_t)stream) != cudaSuccess)
    return AGILE_ECUDA;
  return AGILE_OK;
}

}  // namespace agile

#endif  // AGILE_DEVICE_CUH
