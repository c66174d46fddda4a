// Layout quality metrics of Sec. 2 (visualization quality assessment):
//   ND(X)   = sum_{i<j} 1 / |X_i - X_j|^2            (node distribution)
//   ULCV(X) = l_sigma / l_mu over the edge lengths     (uniform length
//             coefficient variance; population standard deviation)
// Both in FP64 from the given coordinates (FP32 coordinates are widened
// exactly, so differences and squared distances are those of the stored
// values). Sums are formed per warp in a fixed order and reduced per block,
// then across blocks in block order: every run gives the same result.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace pprviz {
namespace {

constexpr int kMetWarps = 8;

template <typename T>
__device__ __forceinline__ double2 xload(const T *x, int64_t i) {
  return make_double2((double)x[2 * i], (double)x[2 * i + 1]);
}

// Per block: rows i = blockIdx.x * kMetWarps + warp (one warp per row), the
// sum over j > i of 1 / d_ij^2 (lanes stride over j); a zero distance sets
// `overlap`. part[blockIdx.x] = the block's sum.
template <typename T>
__global__ void __launch_bounds__(kMetWarps * 32)
k_nd(int64_t k, const T *__restrict__ x, double *__restrict__ part, int *__restrict__ overlap) {
  __shared__ double rs[kMetWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i = (int64_t)blockIdx.x * kMetWarps + warp;
  double acc = 0.0;
  if (i < k) {
    const double2 xi = xload(x, i);
    for (int64_t j = i + 1 + lane; j < k; j += 32) {
      const double2 xj = xload(x, j);
      const double dx = xi.x - xj.x, dy = xi.y - xj.y;
      const double d2 = dx * dx + dy * dy;
      if (d2 == 0.0) atomicOr(overlap, 1);
      else acc += 1.0 / d2;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) rs[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kMetWarps; ++w) s += rs[w];
    part[blockIdx.x] = s;
  }
}

// map[view[q]] = q
__global__ void k_view_map(int32_t k, const int32_t *__restrict__ view, int32_t *__restrict__ map) {
  const int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < k) map[view[q]] = q;
}

// Edge lengths |X_map(u) - X_map(v)| over the CSR edges u -> v with both ends
// in the view: each undirected edge once (u < v), every edge of a directed
// graph. pass 0: part[b] = (sum of lengths, count); pass 1: part[b].x = sum
// of (length - mu)^2.
template <typename T>
__global__ void __launch_bounds__(kMetWarps * 32)
k_ulcv(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const int32_t *__restrict__ map,
       const T *__restrict__ x, int pass, double mu, int directed, double2 *__restrict__ part) {
  __shared__ double2 rs[kMetWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t u = (int64_t)blockIdx.x * kMetWarps + warp;
  double a = 0.0, b = 0.0;
  if (u < n) {
    const int32_t iu = map ? map[u] : (int32_t)u;
    if (iu >= 0) {
      const double2 xu = xload(x, iu);
      for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
        const int32_t v = col[p];
        if (!directed && v <= u) continue;
        const int32_t iv = map ? map[v] : v;
        if (iv < 0) continue;
        const double2 xv = xload(x, iv);
        const double dx = xu.x - xv.x, dy = xu.y - xv.y;
        const double len = sqrt(dx * dx + dy * dy);
        if (pass == 0) {
          a += len;
          b += 1.0;
        } else {
          a += (len - mu) * (len - mu);
        }
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) rs[warp] = make_double2(a, b);
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s = make_double2(0.0, 0.0);
    for (int w = 0; w < kMetWarps; ++w) {
      s.x += rs[w].x;
      s.y += rs[w].y;
    }
    part[blockIdx.x] = s;
  }
}

// out[0] = sum of part[0..nb) in order (one thread: a few thousand terms)
__global__ void k_sum_parts(int nb, const double2 *__restrict__ part, double2 *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double2 s = make_double2(0.0, 0.0);
  for (int b = 0; b < nb; ++b) {
    s.x += part[b].x;
    s.y += part[b].y;
  }
  *out = s;
}

__global__ void k_sum_parts1(int nb, const double *__restrict__ part, double *__restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < nb; ++b) s += part[b];
  *out = s;
}

}  // namespace

template <typename T>
static int metrics_run(pprviz_ctx *ctx, const T *x_d, int32_t k, const pprviz_graph *g, const int32_t *view_d,
                       double *nd_h, double *ulcv_h) {
  PPRVIZ_TRY(ws_ensure(ctx, WS_MISC, 4096));
  unsigned char *misc = static_cast<unsigned char *>(ctx->ws[WS_MISC].p);
  int *overlap = reinterpret_cast<int *>(misc);
  double2 *sum2 = reinterpret_cast<double2 *>(misc + 256);
  double *sum1 = reinterpret_cast<double *>(misc + 512);
  if (nd_h) {
    const int nb = (int)((k + kMetWarps - 1) / kMetWarps);
    PPRVIZ_TRY(ws_ensure(ctx, WS_E, sizeof(double) * (size_t)nb));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(overlap, 0, sizeof(int), ctx->stream));
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY);
      k_nd<T><<<nb, kMetWarps * 32, 0, ctx->stream>>>(k, x_d, ctx->ws[WS_E].as<double>(), overlap);
    }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_sum_parts1<<<1, 32, 0, ctx->stream>>>(nb, ctx->ws[WS_E].as<double>(), sum1); }
    PPRVIZ_LAUNCHED(ctx);
    double s = 0.0;
    int ov = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&s, sum1, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&ov, overlap, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *nd_h = ov ? INFINITY : s;
  }
  if (ulcv_h) {
    const int64_t n = g->n;
    int32_t *map = nullptr;
    if (view_d) {
      PPRVIZ_TRY(ws_ensure(ctx, WS_TROWS, sizeof(int32_t) * (size_t)n));
      map = ctx->ws[WS_TROWS].as<int32_t>();
      PPRVIZ_CUDA(ctx, cudaMemsetAsync(map, 0xFF, sizeof(int32_t) * (size_t)n, ctx->stream));
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_view_map<<<(k + 255) / 256, 256, 0, ctx->stream>>>(k, view_d, map); }
      PPRVIZ_LAUNCHED(ctx);
    }
    const int nb = (int)((n + kMetWarps - 1) / kMetWarps);
    PPRVIZ_TRY(ws_ensure(ctx, WS_B, sizeof(double2) * (size_t)nb));
    double2 *part = ctx->ws[WS_B].as<double2>();
    double2 h = make_double2(0.0, 0.0);
    double mu = 0.0;
    for (int pass = 0; pass < 2; ++pass) {
      {
        PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY);
        k_ulcv<T><<<nb, kMetWarps * 32, 0, ctx->stream>>>(n, g->rp.as<int64_t>(), g->col.as<int32_t>(), map, x_d,
                                                          pass, mu, g->directed ? 1 : 0, part);
      }
      PPRVIZ_LAUNCHED(ctx);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_sum_parts<<<1, 32, 0, ctx->stream>>>(nb, part, sum2); }
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&h, sum2, sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
      PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (pass == 0) {
        if (h.y == 0.0) {
          *ulcv_h = NAN;  // no edge inside the view
          break;
        }
        mu = h.x / h.y;
        *ulcv_h = h.y;  // edge count, kept for the second pass
      } else {
        const double m = *ulcv_h;
        *ulcv_h = sqrt(h.x / m) / mu;
      }
    }
  }
  return PPRVIZ_OK;
}

int layout_metrics(pprviz_ctx *ctx, const void *x_d, bool f64, int32_t k, const pprviz_graph *g,
                   const int32_t *view_d, double *nd_h, double *ulcv_h) {
  return f64 ? metrics_run<double>(ctx, (const double *)x_d, k, g, view_d, nd_h, ulcv_h)
             : metrics_run<float>(ctx, (const float *)x_d, k, g, view_d, nd_h, ulcv_h);
}

}  // namespace pprviz
