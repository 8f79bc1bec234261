// Host-side context of the library and the launcher of the engine kernel.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

#include <cstdio>
#include <vector>

#include "agile.h"
#include "agile_dev.cuh"

#include <algorithm>

struct agile_ctx {
  agile_config cfg;
  int device = 0;
  int sms = 0;
  agile::Dev dev{};
  void *store_host = nullptr;
  std::vector<void *> dallocs;
  int last_cuda_error = 0;
  void *bfs_hubq = nullptr;  // BFS scratch: queue of long adjacency lists
  uint32_t bfs_hub_cap = 0;
  void *bfs_vis = nullptr;  // BFS scratch: visited bitmap
  uint64_t bfs_vis_words = 0;
  void *train_scratch = nullptr;  // backward scratch: sorted keys, bag of each position
  size_t train_scratch_bytes = 0;
  void *emb_scratch = nullptr;  // embedding bag: bags the resident pass left, and their count
  size_t emb_scratch_bytes = 0;
};

namespace agile {

#define AGILE_CUDA_TRY(expr)                                                         \
  do {                                                                               \
    cudaError_t e__ = (expr);                                                        \
    if (e__ != cudaSuccess) {                                                        \
      fprintf(stderr, "agile: %s failed: %s\n", #expr, cudaGetErrorString(e__));     \
      return AGILE_ECUDA;                                                            \
    }                                                                                \
  } while (0)

inline cudaStream_t as_stream(void *s) { return (cudaStream_t)s; }

// Application warps for a call whose warps each keep about `pages_per_warp` lines busy:
// enough warps to keep the queues fed, few enough that their pages fit in the cache.
inline uint32_t warps_for_cache(const agile_ctx *c, uint64_t pages_per_warp, uint32_t floor_warps) {
  uint64_t w = c->dev.nlines / (pages_per_warp ? pages_per_warp : 1);
  return (uint32_t)std::max<uint64_t>(floor_warps, w);
}

// Largest co-resident grid for this engine instantiation (cooperative launch rule:
// every CTA must be resident at once, because the service warps and the waiting app
// warps of one launch depend on each other).
template <class App>
int engine_grid(agile_ctx *c) {
  static int per_sm = -1;  // one value per instantiation
  if (per_sm < 0) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, engine_kernel<App>, kThreads, 0) != cudaSuccess)
      return 0;
    per_sm = n;
  }
  int g = per_sm * c->sms;
  if (c->cfg.max_ctas && (int)c->cfg.max_ctas < g) g = (int)c->cfg.max_ctas;
  return g;
}

// Application warps a launch of this instantiation runs when the call wants `active`
// (0 = all): the context's app_warps setting overrides `active`, the grid bounds both.
template <class App>
uint32_t running_app_warps(agile_ctx *c, uint32_t active) {
  uint64_t n_app = (uint64_t)std::max(0, engine_grid<App>(c)) * (kWarps - 1);
  uint64_t want = c->cfg.app_warps ? c->cfg.app_warps : active;
  return (uint32_t)std::max<uint64_t>(1, want && want < n_app ? want : n_app);
}

// Launches of this translation unit on the current device, counted on the device, so
// that a launch replayed from a recorded stream still gets a number of its own.
static __device__ unsigned long long g_launch_seq;

// Zero the per-launch state and give the launch its number (RunState::epoch).  Runs on
// the call's stream right before the engine kernel.
static __global__ void run_reset_kernel(RunState *r) {
  static_assert(sizeof(RunState) % 4 == 0, "RunState is cleared in 4-byte words");
  uint32_t *w = (uint32_t *)r;
  for (uint32_t i = threadIdx.x; i < sizeof(RunState) / 4; i += blockDim.x) w[i] = 0u;
  __syncthreads();
  if (threadIdx.x == 0) r->epoch = atomicAdd(&g_launch_seq, 1ull) + 1ull;
}

// `active`: application warps the call wants (0 = every app warp of the grid); the
// context's app_warps setting overrides it.
// An application that issues no request ahead of need in this call says so with
//   bool demand_only() const;
// its launch then spreads demand requests over every queue pair (no prefetch class).
template <class T, class = void>
struct has_demand_only : std::false_type {};
template <class T>
struct has_demand_only<T, std::void_t<decltype(std::declval<const T &>().demand_only())>> : std::true_type {};

template <class App>
int launch_engine(agile_ctx *c, const App &app, void *stream, uint32_t active = 0) {
  cudaStream_t s = as_stream(stream);
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  int grid = engine_grid<App>(c);
  if (grid <= 0) return AGILE_ECUDA;
  run_reset_kernel<<<1, 128, 0, s>>>(c->dev.run);
  AGILE_CUDA_TRY(cudaGetLastError());
  Dev d = c->dev;
  d.app_active = c->cfg.app_warps ? c->cfg.app_warps : active;
  if (d.extra_engines == 0xFFFFFFFFu) d.extra_engines = (uint32_t)grid;  // default: one per CTA
  if constexpr (has_demand_only<App>::value) {
    if (app.demand_only()) d.Qp = 0;
  }
  App a = app;
  void *args[] = {(void *)&d, (void *)&a};
  AGILE_CUDA_TRY(cudaLaunchCooperativeKernel((const void *)engine_kernel<App>, dim3(grid), dim3(kThreads),
                                             args, 0, s));
  return AGILE_OK;
}

}  // namespace agile
