// Backward of the cache-backed embedding bag with a fused SGD step written into the
// cached pages (the differentiable extension of the Sec. 4.4 lookups).
//
// G[r, :] = sum over every index position i with idx[i] = r of gout[bag(i), :], added in
// increasing i (= increasing (bag, i)) in FP32, one accumulator per element starting at
// +0.  With lr != 0 every touched row becomes T[r, :] - (lr * G[r, :]) (product rounded
// first, no fused multiply-add) in its cache line, which turns MODIFIED; such lines reach
// the store through the queues when they are evicted or flushed (Sec. 3.4 case (d)).
//
// Grouping the positions by row in increasing position order: keys (row << 32 | i) are
// unique, so sorting them (bitonic network, any order of equal rows is impossible) puts
// each row's positions together and in increasing i.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>

#include "agile.h"
#include "agile_ctx.cuh"
#include "agile_dev.cuh"

using namespace agile;

namespace {

constexpr int kMaxF4 = 8;  // dim <= 1024

__global__ void make_keys_kernel(const int64_t *idx, uint64_t n, uint64_t npad, uint32_t rows, uint64_t *keys,
                                 int32_t *err) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  if (i < n) {
    int64_t r = idx[i];
    if (r < 0 || (uint64_t)r >= rows) {
      atomicCAS(err, 0, 22);
      r = 0;
    }
    keys[i] = ((uint64_t)r << 32) | i;
  } else {
    keys[i] = ~0ull;
  }
}

// bag of every index position
__global__ void bag_of_kernel(const int64_t *off, uint32_t n_bags, int32_t *bag_of) {
  uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  unsigned l = threadIdx.x & 31;
  if (w >= n_bags) return;
  for (int64_t i = off[w] + l; i < off[w + 1]; i += 32) bag_of[i] = (int32_t)w;
}

// one compare-exchange step (k, j) of a bitonic sort of npad keys, ascending
__global__ void bitonic_step_kernel(uint64_t *keys, uint64_t npad, uint64_t k, uint64_t j) {
  uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  if (i >= npad) return;
  uint64_t p = i ^ j;
  if (p <= i) return;
  uint64_t a = keys[i], b = keys[p];
  bool up = (i & k) == 0;
  if (up ? (a > b) : (a < b)) {
    keys[i] = b;
    keys[p] = a;
  }
}

__global__ void set_error_kernel(Dev d, const int32_t *err) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *err) set_error(d, -(*err));
}

// The engine part: per distinct row (a segment of the sorted keys), the gradient row in
// fixed order, written out and/or applied to the cached page.
//   SYNC : the row's page is requested when the warp gets to the row.
//   ASYNC: the pages of the rows of the warp's next 32 sorted positions are requested
//          before the rows of the current 32 are processed.
template <int MF4>
struct BackwardApp {
  uint64_t page0;
  uint32_t rows, dim;
  const uint64_t *keys;
  const int32_t *bag_of;
  uint64_t n;
  const float *gout;
  float lr;
  float *grad_table;
  uint32_t mode;
  // no request ahead of need: the launch uses every queue pair for demand
  bool demand_only() const { return mode == AGILE_SYNC; }

  __device__ __forceinline__ uint32_t row_at(uint64_t j) const { return (uint32_t)(keys[j] >> 32); }

  __device__ bool prefetch(const Dev &d, const AppCtx &a, uint64_t base) const {
    uint64_t j = base + lane_id();
    bool head = j < n && (j == 0 || row_at(j) != row_at(j - 1));
    uint64_t pg = head ? page0 + ((uint64_t)row_at(j) * dim * 4) / kPage : 0;
    return warp_request(d, head, pg, a.q0, false, a.deadline, nullptr, nullptr, nullptr, true, true);
  }

  __device__ void run(const Dev &d, const AppCtx &a) const {
    unsigned l = lane_id();
    const uint32_t nf4 = dim / 4;
    const bool async = mode == AGILE_ASYNC;
    const uint64_t stride = (uint64_t)a.n_warps * 32;
    if (async && lr != 0.0f && (uint64_t)a.warp * 32 < n && !prefetch(d, a, (uint64_t)a.warp * 32)) return;
    for (uint64_t base = (uint64_t)a.warp * 32; base < n; base += stride) {
      if (async && lr != 0.0f && base + stride < n && !prefetch(d, a, base + stride)) return;
      uint64_t j = base + l;
      bool head = j < n && (j == 0 || row_at(j) != row_at(j - 1));
      unsigned m = __ballot_sync(kFull, head);
      while (m) {
        int t = __ffs(m) - 1;
        m &= m - 1;
        uint64_t j0 = base + t;
        uint32_t r = row_at(j0);
        float4 acc[MF4];
#pragma unroll
        for (int k = 0; k < MF4; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        for (uint64_t jj = j0; jj < n; ++jj) {
          uint64_t key = keys[jj];
          if ((uint32_t)(key >> 32) != r) break;
          const float *g = gout + (uint64_t)bag_of[(uint32_t)key] * dim;
#pragma unroll
          for (int k = 0; k < MF4; ++k) {
            uint32_t c = l + 32 * k;
            if (c < nf4) {
              float4 v = *(const float4 *)(g + 4 * c);
              acc[k].x = __fadd_rn(acc[k].x, v.x);
              acc[k].y = __fadd_rn(acc[k].y, v.y);
              acc[k].z = __fadd_rn(acc[k].z, v.z);
              acc[k].w = __fadd_rn(acc[k].w, v.w);
            }
          }
        }
        if (grad_table) {
          float4 *o = (float4 *)(grad_table + (uint64_t)r * dim);
#pragma unroll
          for (int k = 0; k < MF4; ++k) {
            uint32_t c = l + 32 * k;
            if (c < nf4) o[c] = acc[k];
          }
        }
        if (lr != 0.0f) {
          uint64_t byte = (uint64_t)r * dim * 4;
          uint32_t line;
          if (!warp_pin_page(d, page0 + byte / kPage, a.q0, a.deadline, line)) return;
          uint8_t *rowp = line_ptr(d, line) + byte % kPage;
#pragma unroll
          for (int k = 0; k < MF4; ++k) {
            uint32_t c = l + 32 * k;
            if (c < nf4) {
              float4 t4 = ld_cg_f4(rowp + 16 * c);
              t4.x = __fsub_rn(t4.x, __fmul_rn(lr, acc[k].x));
              t4.y = __fsub_rn(t4.y, __fmul_rn(lr, acc[k].y));
              t4.z = __fsub_rn(t4.z, __fmul_rn(lr, acc[k].z));
              t4.w = __fsub_rn(t4.w, __fmul_rn(lr, acc[k].w));
              st_cg16(rowp + 16 * c,
                      make_int4(__float_as_int(t4.x), __float_as_int(t4.y), __float_as_int(t4.z), __float_as_int(t4.w)));
            }
          }
          __threadfence();
          __syncwarp();
          if (l == 0) {
            uint64_t old = atomicOr(&d.tag[line], 1ull);  // READY (2) -> MODIFIED (3)
            if (tag_state(old) == ST_READY) note_dirty(d, page0 + byte / kPage);
            cache_unpin(d, line);
          }
        }
      }
    }
  }
};

}  // namespace

extern "C" {

int agile_embedding_bag_backward(agile_ctx *c, uint64_t table_byte0, uint32_t rows, uint32_t dim,
                                 const int64_t *d_idx, const int64_t *d_offsets, uint32_t n_bags,
                                 uint32_t n_indices, const float *d_grad_out, float lr, float *d_grad_table,
                                 uint32_t mode, void *stream) {
  if (!c || mode > 1) return AGILE_EINVAL;
  if (n_bags == 0 || n_indices == 0) return AGILE_OK;
  if (!d_idx || !d_offsets || !d_grad_out) return AGILE_EINVAL;
  if (dim == 0 || dim % 4 || dim * 4 > kPage || dim > 32 * 4 * kMaxF4 || kPage % (dim * 4)) return AGILE_EINVAL;
  if (table_byte0 % kPage || table_byte0 + (uint64_t)rows * dim * 4 > c->cfg.store_bytes) return AGILE_EINVAL;
  if (((uintptr_t)d_grad_out) & 15 || ((uintptr_t)d_grad_table) & 15) return AGILE_EINVAL;
  AGILE_CUDA_TRY(cudaSetDevice(c->device));
  cudaStream_t s = as_stream(stream);
  uint64_t n = n_indices, npad = 1;
  while (npad < n) npad <<= 1;
  // scratch: sorted keys, bag of each position, an error word
  size_t need = npad * 8 + n * 4 + 256;
  if (c->train_scratch_bytes < need) {
    if (c->train_scratch) cudaFree(c->train_scratch);
    c->train_scratch = nullptr;
    c->train_scratch_bytes = 0;
    AGILE_CUDA_TRY(cudaMalloc(&c->train_scratch, need));
    c->train_scratch_bytes = need;
  }
  uint64_t *keys = (uint64_t *)c->train_scratch;
  int32_t *bag_of = (int32_t *)(keys + npad);
  int32_t *err = (int32_t *)(((uintptr_t)(bag_of + n) + 255) & ~(uintptr_t)255);
  AGILE_CUDA_TRY(cudaMemsetAsync(err, 0, 4, s));
  make_keys_kernel<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(d_idx, n, npad, rows, keys, err);
  bag_of_kernel<<<(unsigned)((n_bags * 32ull + 255) / 256), 256, 0, s>>>(d_offsets, n_bags, bag_of);
  for (uint64_t k = 2; k <= npad; k <<= 1)
    for (uint64_t j = k >> 1; j > 0; j >>= 1)
      bitonic_step_kernel<<<(unsigned)((npad + 255) / 256), 256, 0, s>>>(keys, npad, k, j);
  set_error_kernel<<<1, 32, 0, s>>>(c->dev, err);
  AGILE_CUDA_TRY(cudaGetLastError());
  if (d_grad_table) AGILE_CUDA_TRY(cudaMemsetAsync(d_grad_table, 0, (size_t)rows * dim * 4, s));
  uint32_t warps = warps_for_cache(c, mode == AGILE_ASYNC ? 8 : 4, 32);
  if (dim <= 128) {
    BackwardApp<1> app{table_byte0 / kPage, rows, dim, keys, bag_of, n, d_grad_out, lr, d_grad_table, mode};
    return launch_engine(c, app, stream, warps);
  }
  BackwardApp<kMaxF4> app{table_byte0 / kPage, rows, dim, keys, bag_of, n, d_grad_out, lr, d_grad_table, mode};
  return launch_engine(c, app, stream, warps);
}

}  // extern "C"
