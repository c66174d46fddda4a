// Graph analysis for the deflated Chebyshev sweeps of the FP32 propagation.
//
// The walk matrix P of an undirected graph is self-adjoint in the inner
// product <u, v>_D = sum_i dw_i u_i v_i, so its spectrum is real. Each
// connected component C contributes the eigenvalue 1 (right eigenvector 1_C,
// left eigenvector the stationary vector dw 1_C / m_C, m_C = sum_{i in C} dw_i);
// a node without edges is a component of its own (its walk stays put). For the
// PPR system x (I - cP) = alpha e_s the coefficient of x on the stationary
// vector of C(s) is exactly x 1_C = 1 (multiply the system by 1_C), so the
// propagation can start from that vector and leave only the other modes,
// whose eigenvalues lie in [-b, b] for some b <= 1. Chebyshev semi-iteration
// on [1 - cb, 1 + cb] then converges at rate (1 - sqrt(1 - (cb)^2)) / (cb)
// instead of the rate for b = 1.
//
// This file computes, once per graph:
//  * the component root of every node (the smallest node id of its
//    component; hooking of larger roots under smaller ones with atomicMin,
//    then pointer jumping, until no edge joins two roots), and m_C per root;
//  * an estimate of b: power iteration with P^2 from v_0 = (P - I) u (which
//    has no component on any eigenvalue-1 mode, since (P - I) 1_C = 0 and P
//    is self-adjoint in <,>_D), then the Rayleigh quotient
//    b^2 ~ <P v, P v>_D / <v, v>_D. It is a lower estimate (a weighted mean
//    of lambda^2), so a margin is added; an underestimate only slows the
//    modes above it, it never breaks convergence, and the FP64 residual
//    certificate decides when a row is done.
// All reductions run in a fixed order, so the estimate (and every result
// downstream of it) is the same on every run.
#include <math.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace pprviz {

namespace {
constexpr int kSpecBlocks = 256;  // blocks of the partial-sum reductions
constexpr int kSpecIters = 12;    // P^2 power steps
constexpr int kCcMaxRounds = 64;  // hooking rounds before giving up

__global__ void k_cc_init(int64_t n, int32_t *__restrict__ parent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = (int32_t)i;
}

// bounded walk to the root (parent[x] <= x always, so at most x steps)
__device__ __forceinline__ int32_t cc_root(const int32_t *parent, int32_t x) {
  for (int it = 0; it < (1 << 20); ++it) {
    const int32_t p = parent[x];
    if (p == x) break;
    x = p;
  }
  return x;
}

// One warp per node u: for every edge (u, v) with u < v, hook the larger root
// under the smaller one.
__global__ void k_cc_hook(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          int32_t *parent, int *__restrict__ changed) {
  const int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  int ch = 0;
  for (int64_t p = rp[u] + lane; p < rp[u + 1]; p += 32) {
    const int32_t v = col[p];
    if ((int64_t)v <= u) continue;
    const int32_t ru = cc_root(parent, (int32_t)u), rv = cc_root(parent, v);
    if (ru != rv) {
      atomicMin(&parent[max(ru, rv)], min(ru, rv));
      ch = 1;
    }
  }
  if (__any_sync(0xffffffffu, ch) && lane == 0) atomicOr(changed, 1);
}

__global__ void k_cc_compress(int64_t n, int32_t *parent) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) parent[i] = cc_root(parent, parent[i]);
}

// deterministic start vector u_i in [-0.5, 0.5) (SplitMix64 finaliser of i)
__device__ __forceinline__ double start_u(int64_t i) {
  uint64_t z = (uint64_t)i + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

// out = P v (or P u - u with the start vector when v == nullptr), FP64, one warp per row:
// (P v)_j = (1 / dw_j) sum_{i in N(j)} w_ji v_i, and v_j for a node without edges.
__global__ void k_spec_spmv(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            const float *__restrict__ w, const double *__restrict__ invdw,
                            const double *__restrict__ v, double *__restrict__ out) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  const int64_t b = rp[j], e = rp[j + 1];
  double acc = 0.0;
  for (int64_t p = b + lane; p < e; p += 32) {
    const int32_t i = col[p];
    const double vi = v ? v[i] : start_u(i);
    acc += (w ? (double)w[p] : 1.0) * vi;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const double vj = v ? v[j] : start_u(j);
    const double pv = (e == b) ? vj : acc * invdw[j];
    out[j] = v ? pv : pv - vj;
  }
}

// part[blk] = sum over the block's strided share of dw_i a_i b_i (dw = 1 / invdw)
__global__ void k_spec_dot(int64_t n, const double *__restrict__ invdw, const double *__restrict__ a,
                           const double *__restrict__ b, double *__restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i] / invdw[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// out[0] = sum of part[0 .. np) in a fixed order
__global__ void k_spec_sum(int np, const double *__restrict__ part, double *__restrict__ out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0];
}

// v /= sqrt(nrm2[0]) when it is positive (keeps the power iterates in range)
__global__ void k_spec_normalise(int64_t n, const double *__restrict__ nrm2, double *__restrict__ v) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double s = nrm2[0];
  if (i < n && s > 0.0) v[i] *= 1.0 / sqrt(s);
}
}  // namespace

int graph_spectral(pprviz_ctx *ctx, const pprviz_graph *g) {
  if (g->spec_ready) return PPRVIZ_OK;
  const int64_t n = g->n;
  const unsigned nb = (unsigned)((n + 255) / 256), wb = (unsigned)((n * 32 + 255) / 256);
  PPRVIZ_CUDA(ctx, g->comp.ensure(sizeof(int32_t) * (size_t)n));
  PPRVIZ_TRY(ws_ensure(ctx, WS_SPEC, sizeof(double) * (size_t)(3 * n + kSpecBlocks + 8)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  int32_t *parent = g->comp.as<int32_t>();
  int *changed = ctx->ws[WS_FLAG].as<int>();
  const int64_t *rp = g->rp.as<int64_t>();
  const int32_t *col = g->col.as<int32_t>();
  const float *w = g->weighted ? g->w.as<float>() : nullptr;
  const double *invdw = g->invdw_d.as<double>();

  // ---- connected components
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_cc_init<<<nb, 256, 0, ctx->stream>>>(n, parent); }
  PPRVIZ_LAUNCHED(ctx);
  bool done = false;
  for (int round = 0; round < kCcMaxRounds && !done; ++round) {
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(changed, 0, sizeof(int), ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_cc_hook<<<wb, 256, 0, ctx->stream>>>(n, rp, col, parent, changed); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_cc_compress<<<nb, 256, 0, ctx->stream>>>(n, parent); }
    PPRVIZ_LAUNCHED(ctx);
    int hc = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hc, changed, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    done = hc == 0;
  }
  g->h_comp.resize((size_t)n);
  std::vector<double> h_invdw((size_t)n);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->h_comp.data(), parent, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(h_invdw.data(), invdw, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // m_C per root, summed in node order (the stationary vector's normaliser)
  g->h_mc.assign((size_t)n, 0.0);
  for (int64_t i = 0; i < n; ++i) g->h_mc[(size_t)g->h_comp[i]] += 1.0 / h_invdw[(size_t)i];

  // ---- spectral bound of the non-stationary modes
  double *va = ctx->ws[WS_SPEC].as<double>(), *vb = va + n, *part = va + 3 * n, *scal = part + kSpecBlocks;
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_spmv<<<wb, 256, 0, ctx->stream>>>(n, rp, col, w, invdw, nullptr, va); }
  PPRVIZ_LAUNCHED(ctx);
  for (int it = 0; it < kSpecIters; ++it) {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_spmv<<<wb, 256, 0, ctx->stream>>>(n, rp, col, w, invdw, va, vb); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_spmv<<<wb, 256, 0, ctx->stream>>>(n, rp, col, w, invdw, vb, va); }
    PPRVIZ_LAUNCHED(ctx);
    if (it % 4 == 3) {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_dot<<<kSpecBlocks, 256, 0, ctx->stream>>>(n, invdw, va, va, part); }
      PPRVIZ_LAUNCHED(ctx);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_sum<<<1, 256, 0, ctx->stream>>>(kSpecBlocks, part, scal); }
      PPRVIZ_LAUNCHED(ctx);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_normalise<<<nb, 256, 0, ctx->stream>>>(n, scal, va); }
      PPRVIZ_LAUNCHED(ctx);
    }
  }
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_spmv<<<wb, 256, 0, ctx->stream>>>(n, rp, col, w, invdw, va, vb); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_dot<<<kSpecBlocks, 256, 0, ctx->stream>>>(n, invdw, va, va, part); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_sum<<<1, 256, 0, ctx->stream>>>(kSpecBlocks, part, scal); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_dot<<<kSpecBlocks, 256, 0, ctx->stream>>>(n, invdw, vb, vb, part); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_spec_sum<<<1, 256, 0, ctx->stream>>>(kSpecBlocks, part, scal + 1); }
  PPRVIZ_LAUNCHED(ctx);
  double hs[2] = {0.0, 0.0};
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double b = 1.0;
  if (!done) {
    b = 1.0;  // components unresolved: keep the full interval and no deflation
  } else if (hs[0] > 0.0 && std::isfinite(hs[0]) && std::isfinite(hs[1])) {
    b = std::min(1.0, 1.05 * sqrt(std::max(0.0, hs[1] / hs[0])) + 0.02);
  } else {
    b = 0.02;  // no non-stationary mode reached: every component is trivial
  }
  g->spec_b = b;
  g->spec_deflate = done;
  g->spec_ready = true;
  return PPRVIZ_OK;
}

}  // namespace pprviz
