// P0 - graph ingest: CSR validation, degrees d(v) and view checks, on the device.
//
// The paper's input is a graph G = (V, E) with out-degree d(v) (Sec. 2.1,
// Table 1); a random walk steps from v_i to an out-neighbour (Sec. 3.1). For
// weighted graphs the step probability is w_ij / sum_j w_ij and d(v) is that
// strength. A node without edges keeps its walk (a self-loop in the walk
// matrix) and has d(v) = 0.
#include <math.h>

#include <vector>

#include "common.cuh"

namespace pprviz {

enum GraphErr : int {
  GE_ROWPTR = 1, GE_COLRANGE = 2, GE_SELFLOOP = 4, GE_UNSORTED = 8, GE_WEIGHT = 16, GE_ASYM = 32,
};

__global__ void k_validate_csr(int64_t n, int64_t nnz, const int64_t *__restrict__ rp,
                               const int32_t *__restrict__ col, const float *__restrict__ w,
                               int check_sym, int *__restrict__ flag) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int64_t b = rp[v], e = rp[v + 1];
  int bad = 0;
  if (v == 0 && b != 0) bad |= GE_ROWPTR;
  if (v == n - 1 && e != nnz) bad |= GE_ROWPTR;
  if (b > e || b < 0 || e > nnz) {
    atomicOr(flag, bad | GE_ROWPTR);
    return;
  }
  int32_t prev = -1;
  for (int64_t p = b; p < e; ++p) {
    int32_t u = col[p];
    if (u < 0 || (int64_t)u >= n) { bad |= GE_COLRANGE; continue; }
    if ((int64_t)u == v) bad |= GE_SELFLOOP;
    if (u <= prev) bad |= GE_UNSORTED;
    prev = u;
    if (w) {
      float x = w[p];
      if (!(x > 0.0f) || !isfinite(x)) bad |= GE_WEIGHT;
    }
    if (check_sym) {
      // binary search v in row u (rows are checked sorted by their own thread;
      // an unsorted row only makes this search unreliable, and is an error anyway)
      int64_t lo = rp[u], hi = rp[u + 1] - 1;
      bool found = false;
      if (lo >= 0 && hi < nnz) {
        while (lo <= hi) {
          int64_t mid = (lo + hi) >> 1;
          int32_t c = col[mid];
          if (c == (int32_t)v) { found = true; if (w && w[mid] != w[p]) bad |= GE_ASYM; break; }
          if (c < (int32_t)v) lo = mid + 1; else hi = mid - 1;
        }
      }
      if (!found) bad |= GE_ASYM;
    }
  }
  if (bad) atomicOr(flag, bad);
}

// d(v): edge count, or strength sum_j w_vj for weighted graphs unless `count`.
// The walk uses dw(v) = strength (or count when unweighted), and dw = 1 for a
// node without edges (its self-loop).
__global__ void k_degrees(int64_t n, const int64_t *__restrict__ rp, const float *__restrict__ w,
                          int count_only, double *__restrict__ deg, float *__restrict__ invdw_f,
                          double *__restrict__ invdw_d, float2 *__restrict__ dwff) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int64_t b = rp[v], e = rp[v + 1];
  double cnt = (double)(e - b);
  double s = cnt;
  if (w) {
    s = 0.0;
    for (int64_t p = b; p < e; ++p) s += (double)w[p];
  }
  deg[v] = (w && !count_only) ? s : cnt;
  double walk = (e > b) ? s : 1.0;
  invdw_d[v] = 1.0 / walk;
  invdw_f[v] = (float)(1.0 / walk);
  const float hi = (float)walk;
  dwff[v] = make_float2(hi, (float)(walk - (double)hi));
}

__global__ void k_view_check(int64_t n, int32_t k, const int32_t *__restrict__ view,
                             int32_t *__restrict__ map, int *__restrict__ flag) {
  int32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= k) return;
  int32_t v = view[q];
  if (v < 0 || (int64_t)v >= n) { atomicOr(flag, 1); return; }
  int32_t old = atomicCAS(&map[v], -1, q);
  if (old != -1) atomicOr(flag, 2);
}

static std::string graph_err_text(int f) {
  std::string s;
  if (f & GE_ROWPTR) s += " row_ptr not a valid prefix sum (row_ptr[0]=0, non-decreasing, row_ptr[n]=nnz);";
  if (f & GE_COLRANGE) s += " column id out of range;";
  if (f & GE_SELFLOOP) s += " self-loop;";
  if (f & GE_UNSORTED) s += " columns not strictly increasing within a row (unsorted or duplicate edge);";
  if (f & GE_WEIGHT) s += " weight not finite and > 0;";
  if (f & GE_ASYM) s += " CSR not symmetric (PPRVIZ_UNDIRECTED);";
  return s;
}

int graph_build(pprviz_ctx *ctx, pprviz_graph *g, uint32_t flags) {
  const int64_t n = g->n;
  const int threads = 256;
  const unsigned blocks = (unsigned)((n + threads - 1) / threads);
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  int *flag = ctx->ws[WS_FLAG].as<int>();
  {
    // validation always runs: the sweeps index state rows by column id, so an
    // out-of-range or malformed CSR must never reach them
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_validate_csr<<<blocks, threads, 0, ctx->stream>>>(
        n, g->nnz, g->rp.as<int64_t>(), g->col.as<int32_t>(), g->weighted ? g->w.as<float>() : nullptr,
        (flags & PPRVIZ_UNDIRECTED) ? 1 : 0, flag); }
    PPRVIZ_LAUNCHED(ctx);
    int hf = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (hf) return set_err(ctx, PPRVIZ_E_BAD_GRAPH, "graph validation failed:" + graph_err_text(hf));
  }
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_degrees<<<blocks, threads, 0, ctx->stream>>>(
      n, g->rp.as<int64_t>(), g->weighted ? g->w.as<float>() : nullptr,
      (flags & PPRVIZ_DEGREE_COUNT) ? 1 : 0, g->deg.as<double>(), g->invdw_f.as<float>(),
      g->invdw_d.as<double>(), g->dwff.as<float2>()); }
  PPRVIZ_LAUNCHED(ctx);
  g->h_deg.resize((size_t)n);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->h_deg.data(), g->deg.p, sizeof(double) * (size_t)n,
                                   cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  double m = 0.0;
  for (double d : g->h_deg) m += d;
  g->m = m;
  return PPRVIZ_OK;
}

// The pull CSR of a directed graph (host arrays of the validated out-edge CSR):
// row j lists the in-neighbours i of j in increasing order with the pull
// weight w_ij (1 when unweighted), so that (x P)_j = sum_i w_ij y_i with
// y = x / dw. A dangling j (no out-edge) keeps its walk: the entry (j, 1)
// (dw = 1); a j without in-edges gets (j, 0), so that no row is empty and the
// kernels' rule for empty rows (the undirected graphs' isolated nodes) never
// applies to a directed graph.
int pull_csr_build(pprviz_ctx *ctx, pprviz_graph *g, const int64_t *rp, const int32_t *col, const float *w) {
  const int64_t n = g->n;
  std::vector<int64_t> cnt((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) cnt[(size_t)col[p] + 1]++;
  std::vector<char> extra((size_t)n, 0);
  for (int64_t j = 0; j < n; ++j) {
    const bool dangling = rp[j + 1] == rp[j];
    if (dangling || cnt[(size_t)j + 1] == 0) {
      extra[(size_t)j] = 1;
      cnt[(size_t)j + 1]++;
    }
  }
  for (int64_t j = 0; j < n; ++j) cnt[(size_t)j + 1] += cnt[(size_t)j];
  const int64_t pnnz = cnt[(size_t)n];
  std::vector<int32_t> pcol((size_t)std::max<int64_t>(pnnz, 1));
  std::vector<float> pw((size_t)std::max<int64_t>(pnnz, 1));
  std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
  // sources in increasing order, so every row comes out sorted; a node's own
  // entry is placed when the scan reaches it
  for (int64_t i = 0; i < n; ++i) {
    if (extra[(size_t)i]) {
      const int64_t q = fill[(size_t)i]++;
      pcol[(size_t)q] = (int32_t)i;
      pw[(size_t)q] = (rp[i + 1] == rp[i]) ? 1.0f : 0.0f;
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      const int64_t q = fill[(size_t)col[p]]++;
      pcol[(size_t)q] = (int32_t)i;
      pw[(size_t)q] = w ? w[p] : 1.0f;
    }
  }
  cudaError_t e = g->prp.ensure(sizeof(int64_t) * (size_t)(n + 1));
  if (e == cudaSuccess) e = g->pcol.ensure(sizeof(int32_t) * pcol.size());
  if (e == cudaSuccess) e = g->pw.ensure(sizeof(float) * pw.size());
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PPRVIZ_E_OOM, "pull CSR of the directed graph: allocation failed");
  }
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->prp.p, cnt.data(), sizeof(int64_t) * (size_t)(n + 1), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->pcol.p, pcol.data(), sizeof(int32_t) * pcol.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->pw.p, pw.data(), sizeof(float) * pw.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  g->directed = true;
  return PPRVIZ_OK;
}

int view_check(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d, int32_t k) {
  PPRVIZ_TRY(ws_ensure(ctx, WS_MISC, sizeof(int32_t) * (size_t)g->n));
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  int32_t *map = ctx->ws[WS_MISC].as<int32_t>();
  int *flag = ctx->ws[WS_FLAG].as<int>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(map, 0xFF, sizeof(int32_t) * (size_t)g->n, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_view_check<<<(k + 255) / 256, 256, 0, ctx->stream>>>(g->n, k, view_d, map, flag); }
  PPRVIZ_LAUNCHED(ctx);
  int hf = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hf & 1) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "view id out of range [0, n)");
  if (hf & 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "duplicate view id");
  return PPRVIZ_OK;
}

}  // namespace pprviz
