// C ABI entry points of libpprviz (declared in include/pprviz.h): argument
// checks, host <-> device staging and dispatch to the kernels. No C++
// exception crosses this boundary.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "common.cuh"

namespace pprviz {

int set_err(pprviz_ctx *ctx, int code, const std::string &msg) {
  if (ctx) ctx->err = msg;
  return code;
}

int cuda_err(pprviz_ctx *ctx, cudaError_t e, const char *what) {
  int code = (e == cudaErrorMemoryAllocation) ? PPRVIZ_E_OOM : PPRVIZ_E_CUDA;
  return set_err(ctx, code, std::string(what) + ": " + cudaGetErrorString(e));
}

int ws_ensure(pprviz_ctx *ctx, int slot, size_t bytes) {
  if (ctx->ws_limit && !(bytes <= ctx->ws[slot].cap && ctx->ws[slot].p)) {
    // the slot grows: its old capacity is released and `bytes` taken
    size_t used = 0;
    for (int q = 0; q < WS_COUNT; ++q)
      if (q != slot) used += ctx->ws[q].cap;
    if (used + bytes > ctx->ws_limit)
      return set_err(ctx, PPRVIZ_E_OOM,
                     "device workspace limit: " + std::to_string(used + bytes) + " bytes needed, limit " +
                         std::to_string(ctx->ws_limit));
  }
  cudaError_t e = ctx->ws[slot].ensure(bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    return set_err(ctx, e == cudaErrorMemoryAllocation ? PPRVIZ_E_OOM : PPRVIZ_E_CUDA,
                   std::string("device workspace allocation failed: ") + cudaGetErrorString(e));
  }
  return PPRVIZ_OK;
}

static cudaEvent_t ev_get(pprviz_ctx *ctx) {
  if (!ctx->ev_pool.empty()) {
    cudaEvent_t e = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

ProfScope::ProfScope(pprviz_ctx *ctx, int k) : c(ctx), cls(k) {
  const int64_t nth = c->class_launches[cls]++;
  // the classes launched hundreds of times per call are sampled: one launch in prof_every
  const bool hot = cls == PPRVIZ_K_SWEEP || cls == PPRVIZ_K_LY || cls == PPRVIZ_K_APPLY || cls == PPRVIZ_K_OTHER ||
                   cls == PPRVIZ_K_PUSH;
  // launches recorded into a CUDA graph are counted, never timed: an event
  // recorded during stream capture marks no point on the device timeline
  if (c->profiling && !c->capturing && (!hot || nth % c->prof_every == 0)) {
    c->class_timed[cls]++;
    a = ev_get(c);
    b = ev_get(c);
    if (a && b) cudaEventRecord(a, c->stream);
  }
}

ProfScope::~ProfScope() {
  if (a && b) {
    cudaEventRecord(b, c->stream);
    c->ev_pending.push_back({cls, {a, b}});
  } else {
    if (a) c->ev_pool.push_back(a);
    if (b) c->ev_pool.push_back(b);
  }
}

// Stage a caller buffer on the device: returns the caller pointer itself for
// device buffers, else copies the host data into workspace slot `slot`.
static int stage_in(pprviz_ctx *ctx, const void *p, size_t bytes, bool device, int slot, const void **out) {
  if (device) {
    *out = p;
    return PPRVIZ_OK;
  }
  PPRVIZ_TRY(ws_ensure(ctx, slot, bytes));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ctx->ws[slot].p, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *out = ctx->ws[slot].p;
  return PPRVIZ_OK;
}

static int begin(pprviz_ctx *ctx) {
  ctx->err.clear();
  ctx->scnt_clear = false;
  ctx->launches = 0;
  memset(&ctx->stats, 0, sizeof(ctx->stats));
  PPRVIZ_CUDA(ctx, cudaSetDevice(ctx->device));
  return PPRVIZ_OK;
}

static int finish(pprviz_ctx *ctx, int status) {
  ctx->stats.kernel_launches = ctx->launches;
  return status;
}

template <typename TI, typename TO>
__global__ void k_cast(int64_t cnt, const TI *__restrict__ in, TO *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (TO)in[i];
}

}  // namespace pprviz

using namespace pprviz;

extern "C" {

int pprviz_create(pprviz_ctx **out, int device, void *cuda_stream) {
  if (!out) return PPRVIZ_E_INVALID_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return PPRVIZ_E_INVALID_ARG;
  }
  pprviz_ctx *ctx = new (std::nothrow) pprviz_ctx();
  if (!ctx) return PPRVIZ_E_OOM;
  ctx->device = device;
  if (cudaSetDevice(device) != cudaSuccess) {
    delete ctx;
    return PPRVIZ_E_CUDA;
  }
  if (cuda_stream) {
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->own_stream = false;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete ctx;
      return PPRVIZ_E_CUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return PPRVIZ_OK;
}

int pprviz_test_expire_wait(pprviz_ctx *ctx) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  ctx->test_expire_wait = true;
  return PPRVIZ_OK;
}

int pprviz_set_workspace_limit(pprviz_ctx *ctx, int64_t bytes) {
  if (!ctx || bytes < 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "bad context or negative limit");
  ctx->ws_limit = (size_t)bytes;
  return PPRVIZ_OK;
}

void pprviz_destroy(pprviz_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto &p : ctx->ev_pending) {
    cudaEventDestroy(p.second.first);
    cudaEventDestroy(p.second.second);
  }
  for (auto e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->side) {
    cudaStreamSynchronize(ctx->side);
    cudaStreamDestroy(ctx->side);
  }
  for (auto &b : ctx->ws) b.release();
  if (ctx->ev_t1) cudaEventDestroy(ctx->ev_t1);
  if (ctx->ev_dp) cudaEventDestroy(ctx->ev_dp);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

const char *pprviz_last_error(const pprviz_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int pprviz_sync(pprviz_ctx *ctx) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_CUDA(ctx, cudaSetDevice(ctx->device));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return PPRVIZ_OK;
}

int pprviz_get_stats(const pprviz_ctx *ctx, pprviz_stats *out) {
  if (!ctx || !out) return PPRVIZ_E_INVALID_ARG;
  *out = ctx->stats;
  return PPRVIZ_OK;
}

int pprviz_profile(pprviz_ctx *ctx, int enable) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_CUDA(ctx, cudaSetDevice(ctx->device));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (auto &p : ctx->ev_pending) {
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
  for (int i = 0; i < PPRVIZ_NKCLASS; ++i) {
    ctx->class_ms[i] = 0.0;
    ctx->class_launches[i] = 0;
    ctx->class_timed[i] = 0;
  }
  ctx->profiling = enable != 0;
  ctx->prof_every = enable > 1 ? enable : 1;
  return PPRVIZ_OK;
}

int pprviz_kernel_times(pprviz_ctx *ctx, double *ms_out, int64_t *launches_out, int64_t *timed_out) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_CUDA(ctx, cudaSetDevice(ctx->device));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // every pending pair goes back to the pool, timed or not, so that no event
  // is both pending and pooled; a pair that cannot be timed is dropped from
  // the class's timed count and reported once after the pass
  cudaError_t bad = cudaSuccess;
  for (auto &p : ctx->ev_pending) {
    float ms = 0.0f;
    const cudaError_t e = cudaEventElapsedTime(&ms, p.second.first, p.second.second);
    if (e == cudaSuccess) {
      ctx->class_ms[p.first] += ms;
    } else {
      if (bad == cudaSuccess) bad = e;
      if (ctx->class_timed[p.first] > 0) ctx->class_timed[p.first]--;
    }
    ctx->ev_pool.push_back(p.second.first);
    ctx->ev_pool.push_back(p.second.second);
  }
  ctx->ev_pending.clear();
  for (int i = 0; i < PPRVIZ_NKCLASS; ++i) {
    if (ms_out) ms_out[i] = ctx->class_ms[i];
    if (launches_out) launches_out[i] = ctx->class_launches[i];
    if (timed_out) timed_out[i] = ctx->class_timed[i];
  }
  if (bad != cudaSuccess) {
    cudaGetLastError();
    return cuda_err(ctx, bad, "cudaEventElapsedTime (kernel_times)");
  }
  return PPRVIZ_OK;
}

int pprviz_graph_upload(pprviz_ctx *ctx, int64_t n, const int64_t *row_ptr, const int32_t *col_idx,
                        const float *weights, uint32_t flags, uint32_t mem_flags, pprviz_graph **out) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  if (!out) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "out is NULL");
  *out = nullptr;
  PPRVIZ_TRY(begin(ctx));
  if (n < 1 || n > INT32_MAX) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "n must be in [1, 2^31 - 1]");
  if (!row_ptr) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "row_ptr is NULL");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  int64_t nnz = 0;
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    nnz = row_ptr[n];
  }
  if (nnz < 0) return set_err(ctx, PPRVIZ_E_BAD_GRAPH, "row_ptr[n] is negative");
  if (nnz > 0 && !col_idx) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "col_idx is NULL");
  pprviz_graph *g = new (std::nothrow) pprviz_graph();
  if (!g) return set_err(ctx, PPRVIZ_E_OOM, "host allocation failed");
  g->ctx = ctx;
  g->device = ctx->device;
  g->n = n;
  g->nnz = nnz;
  g->weighted = weights != nullptr;
  g->flags = flags;
  auto fail = [&](int s) { pprviz_graph_free(g); return s; };
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e;
  if ((e = g->rp.ensure(sizeof(int64_t) * (size_t)(n + 1))) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc row_ptr"));
  if ((e = g->col.ensure(sizeof(int32_t) * (size_t)nnz)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc col"));
  if (g->weighted && (e = g->w.ensure(sizeof(float) * (size_t)nnz)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc w"));
  if ((e = g->deg.ensure(sizeof(double) * (size_t)n)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc deg"));
  if ((e = g->invdw_f.ensure(sizeof(float) * (size_t)n)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc invdw"));
  if ((e = g->invdw_d.ensure(sizeof(double) * (size_t)n)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc invdw"));
  if ((e = g->dwff.ensure(sizeof(float2) * (size_t)n)) != cudaSuccess) return fail(cuda_err(ctx, e, "alloc dw"));
  if ((e = cudaMemcpyAsync(g->rp.p, row_ptr, sizeof(int64_t) * (size_t)(n + 1), kind, ctx->stream)) != cudaSuccess)
    return fail(cuda_err(ctx, e, "copy row_ptr"));
  if (nnz && (e = cudaMemcpyAsync(g->col.p, col_idx, sizeof(int32_t) * (size_t)nnz, kind, ctx->stream)) != cudaSuccess)
    return fail(cuda_err(ctx, e, "copy col"));
  if (g->weighted && nnz &&
      (e = cudaMemcpyAsync(g->w.p, weights, sizeof(float) * (size_t)nnz, kind, ctx->stream)) != cudaSuccess)
    return fail(cuda_err(ctx, e, "copy weights"));
  int s = graph_build(ctx, g, flags);
  if (s != PPRVIZ_OK) return fail(s);
  if (!(flags & PPRVIZ_UNDIRECTED)) {
    // directed: the pull CSR from host copies of the (validated) arrays
    std::vector<int64_t> rp_h((size_t)n + 1);
    std::vector<int32_t> col_h((size_t)nnz);
    std::vector<float> w_h(g->weighted ? (size_t)nnz : 0);
    if ((e = cudaMemcpyAsync(rp_h.data(), g->rp.p, sizeof(int64_t) * rp_h.size(), cudaMemcpyDeviceToHost,
                             ctx->stream)) != cudaSuccess ||
        (nnz && (e = cudaMemcpyAsync(col_h.data(), g->col.p, sizeof(int32_t) * col_h.size(), cudaMemcpyDeviceToHost,
                                     ctx->stream)) != cudaSuccess) ||
        (g->weighted && nnz &&
         (e = cudaMemcpyAsync(w_h.data(), g->w.p, sizeof(float) * w_h.size(), cudaMemcpyDeviceToHost, ctx->stream)) !=
             cudaSuccess) ||
        (e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
      return fail(cuda_err(ctx, e, "copy the CSR back for the pull CSR"));
    s = pull_csr_build(ctx, g, rp_h.data(), col_h.data(), g->weighted ? w_h.data() : nullptr);
    if (s != PPRVIZ_OK) return fail(s);
  }
  *out = g;
  return finish(ctx, PPRVIZ_OK);
}

void pprviz_graph_free(pprviz_graph *g) {
  if (!g) return;
  cudaSetDevice(g->device);  // the context may already be destroyed
  g->rp.release();
  g->col.release();
  g->w.release();
  g->deg.release();
  g->invdw_f.release();
  g->invdw_d.release();
  g->dwff.release();
  g->dense.release();
  g->comp.release();
  g->sp_items.release();
  g->sp_srow.release();
  g->prp.release();
  g->pcol.release();
  g->pw.release();
  delete g;
}

int pprviz_graph_degrees(pprviz_ctx *ctx, const pprviz_graph *g, double *deg_out, int64_t *n_out,
                         int64_t *nnz_out, double *m_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  if (!g) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph is NULL");
  PPRVIZ_TRY(begin(ctx));
  if (n_out) *n_out = g->n;
  if (nnz_out) *nnz_out = g->nnz;
  if (m_out) *m_out = g->m;
  if (deg_out) {
    const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(deg_out, g->deg.p, sizeof(double) * (size_t)g->n,
                                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, ctx->stream));
    if (!dev) PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_dppr(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view, int32_t k, double alpha, double eps,
                int precision, void *dppr_out, void *pdist_out, int64_t n_clamp, double *cert_out,
                uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!g || !view) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph or view is NULL");
  if (k < 1 || (int64_t)k > g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be in [1, n]");
  if (!(alpha > 0.0 && alpha < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(eps > 0.0) || !isfinite(eps)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "eps must be finite and > 0");
  if (precision < PPRVIZ_FP64 || precision > PPRVIZ_FP32_BF16TC)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG,
                   "precision must be PPRVIZ_FP64, PPRVIZ_FP32, PPRVIZ_FP32_CSR, PPRVIZ_FP32_TC or "
                   "PPRVIZ_FP32_BF16TC");
  if (n_clamp == 0) n_clamp = g->n;
  if (n_clamp < 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "n_clamp must be >= 2");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool out64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  const size_t kk = (size_t)k * (size_t)k;
  // view on both sides
  std::vector<int32_t> view_h((size_t)k);
  const int32_t *view_d = nullptr;
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(view_h.data(), view, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, ctx->stream));
    view_d = view;
  } else {
    memcpy(view_h.data(), view, sizeof(int32_t) * k);
    const void *p = nullptr;
    PPRVIZ_TRY(stage_in(ctx, view, sizeof(int32_t) * k, false, WS_VIEW, &p));
    view_d = (const int32_t *)p;
  }
  PPRVIZ_TRY(view_check(ctx, g, view_d, k));
  // DPPR is computed in FP64 for the FP64 path (and for FP64 outputs), else FP32
  const bool int64p = precision == PPRVIZ_FP64 || out64;
  const size_t ie = int64p ? sizeof(double) : sizeof(float);
  void *dppr_d = nullptr;
  if (dppr_out && dev && int64p == out64) dppr_d = dppr_out;
  else if (dppr_out || pdist_out) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_DPPR, ie * kk));
    dppr_d = ctx->ws[WS_DPPR].p;
  }
  std::vector<double> cert_tmp;
  double *cert_h = cert_out;
  int status = dppr_solve(ctx, g, view_d, view_h, k, alpha, eps, precision, dppr_d, int64p, cert_h);
  if (status != PPRVIZ_OK && status != PPRVIZ_E_NOT_CONVERGED) return finish(ctx, status);
  const std::string keep_err = ctx->err;
  void *pdist_d = nullptr;
  if (pdist_out) {
    if (dev && int64p == out64) pdist_d = pdist_out;
    else {
      PPRVIZ_TRY(ws_ensure(ctx, WS_PDIST, ie * kk));
      pdist_d = ctx->ws[WS_PDIST].p;
    }
    PPRVIZ_TRY(pdist_launch(ctx, dppr_d, k, n_clamp, pdist_d, int64p));
  }
  // deliver outputs in the requested type and memory space
  auto deliver = [&](void *src_d, void *dst, int tmp_slot) -> int {
    if (!dst || src_d == dst) return PPRVIZ_OK;
    const size_t ob = (out64 ? sizeof(double) : sizeof(float)) * kk;
    void *conv = src_d;
    if (int64p != out64) {
      // FP64 path with float outputs: narrow on the device
      void *target = dev ? dst : nullptr;
      if (!target) {
        PPRVIZ_TRY(ws_ensure(ctx, tmp_slot, ob));
        target = ctx->ws[tmp_slot].p;
      }
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_cast<double, float><<<(unsigned)((kk + 255) / 256), 256, 0, ctx->stream>>>((int64_t)kk, (const double *)src_d,
                                                                                 (float *)target); }
      PPRVIZ_LAUNCHED(ctx);
      conv = target;
      if (dev) return PPRVIZ_OK;
    }
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(dst, conv, ob, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                     ctx->stream));
    return PPRVIZ_OK;
  };
  PPRVIZ_TRY(deliver(dppr_d, dppr_out, WS_OUT0));
  PPRVIZ_TRY(deliver(pdist_d, pdist_out, WS_OUT1));
  if (!dev || cert_out) PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (status != PPRVIZ_OK) ctx->err = keep_err;
  return finish(ctx, status);
}

// Reads and checks a leaf-set CSR (host or device): lp / li get host copies,
// lp_d / li_d device pointers (the caller's, or staged copies).
static int leaf_sets_in(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr,
                        const int32_t *leaf_idx, bool dev, std::vector<int64_t> &lp, std::vector<int32_t> &li,
                        const int64_t **lp_d, const int32_t **li_d) {
  lp.assign((size_t)nsup + 1, 0);
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(lp.data(), leaf_ptr, sizeof(int64_t) * lp.size(), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    memcpy(lp.data(), leaf_ptr, sizeof(int64_t) * lp.size());
  }
  if (lp[0] != 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "leaf_ptr[0] must be 0");
  for (int32_t v = 0; v < nsup; ++v)
    if (lp[v + 1] <= lp[v]) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "every supernode needs at least one leaf");
  const int64_t nleaf = lp[nsup];
  if (nleaf > g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "more leaves than nodes: leaf sets must be disjoint");
  li.assign((size_t)nleaf, 0);
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(li.data(), leaf_idx, sizeof(int32_t) * li.size(), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    memcpy(li.data(), leaf_idx, sizeof(int32_t) * li.size());
  }
  std::vector<char> seen((size_t)g->n, 0);
  for (int32_t t : li) {
    if (t < 0 || (int64_t)t >= g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "leaf id out of range");
    if (seen[t]) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "leaf sets must be disjoint (a node is listed twice)");
    seen[t] = 1;
  }
  *lp_d = leaf_ptr;
  *li_d = leaf_idx;
  if (!dev) {
    const void *p = nullptr;
    PPRVIZ_TRY(stage_in(ctx, lp.data(), sizeof(int64_t) * lp.size(), false, WS_IN0, &p));
    *lp_d = (const int64_t *)p;
    PPRVIZ_TRY(stage_in(ctx, li.data(), sizeof(int32_t) * li.size(), false, WS_IN1, &p));
    *li_d = (const int32_t *)p;
  }
  return PPRVIZ_OK;
}

int pprviz_level_dppr(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr,
                      const int32_t *leaf_idx, double alpha, double eps, void *ldppr_out, void *pdist_out,
                      int64_t n_clamp, double *cert_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!g || !leaf_ptr || !leaf_idx) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph or leaf sets are NULL");
  if (nsup < 1 || (int64_t)nsup > g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "nsup must be in [1, n]");
  if (!(alpha > 0.0 && alpha < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(eps > 0.0) || !isfinite(eps)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "eps must be finite and > 0");
  if (n_clamp == 0) n_clamp = g->n;
  if (n_clamp < 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "n_clamp must be >= 2");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool out64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  std::vector<int64_t> lp;
  std::vector<int32_t> li;
  const int64_t *lp_d = nullptr;
  const int32_t *li_d = nullptr;
  PPRVIZ_TRY(leaf_sets_in(ctx, g, nsup, leaf_ptr, leaf_idx, dev, lp, li, &lp_d, &li_d));
  const size_t kk = (size_t)nsup * (size_t)nsup;
  const size_t ob = (out64 ? sizeof(double) : sizeof(float)) * kk;
  void *ld_d = nullptr;
  if (ldppr_out && dev) ld_d = ldppr_out;
  else {
    PPRVIZ_TRY(ws_ensure(ctx, WS_DPPR, ob));
    ld_d = ctx->ws[WS_DPPR].p;
  }
  int status = level_dppr_solve(ctx, g, nsup, lp_d, li_d, lp, li, alpha, eps, ld_d, out64, cert_out);
  if (status != PPRVIZ_OK && status != PPRVIZ_E_NOT_CONVERGED) return finish(ctx, status);
  const std::string keep_err = ctx->err;
  if (pdist_out) {
    void *pd_d = dev ? pdist_out : nullptr;
    if (!pd_d) {
      PPRVIZ_TRY(ws_ensure(ctx, WS_PDIST, ob));
      pd_d = ctx->ws[WS_PDIST].p;
    }
    PPRVIZ_TRY(pdist_launch(ctx, ld_d, nsup, n_clamp, pd_d, out64));
    if (!dev) PPRVIZ_CUDA(ctx, cudaMemcpyAsync(pdist_out, pd_d, ob, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (ldppr_out && !dev) PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ldppr_out, ld_d, ob, cudaMemcpyDeviceToHost, ctx->stream));
  if (!dev || cert_out) PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (status != PPRVIZ_OK) ctx->err = keep_err;
  return finish(ctx, status);
}

int pprviz_dpr(pprviz_ctx *ctx, const pprviz_graph *g, double alpha, double eps, double *dpr_out, double *cert_out,
               uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!g || !dpr_out) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph or output is NULL");
  if (!(alpha > 0.0 && alpha < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(eps > 0.0 && eps < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "eps must be in (0, 1)");
  if (!(g->m > 0.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "the DPR needs a graph with edges (m > 0)");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  double *out_d = dpr_out;
  if (!dev) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_OUT0, sizeof(double) * (size_t)g->n));
    out_d = ctx->ws[WS_OUT0].as<double>();
  }
  PPRVIZ_TRY(dpr_solve(ctx, g, alpha, eps, out_d, cert_out));
  if (!dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(dpr_out, out_d, sizeof(double) * (size_t)g->n, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_louvain_plus(pprviz_ctx *ctx, const pprviz_graph *g, int32_t k, int64_t *level_n, int32_t level_cap,
                        int32_t *parent, int64_t parent_cap, pprviz_louvain_info *info) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (info) memset(info, 0, sizeof(*info));
  if (!g || !level_n || !parent || !info) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph or an output is NULL");
  if (k < 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "Louvain+ needs k >= 2");
  if (level_cap < 0 || parent_cap < 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "negative capacity");
  if (g->directed)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "Louvain+ takes an undirected graph (symmetrise a directed one first)");
  if (g->nnz >= ((int64_t)1 << 31)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "Louvain+ takes graphs below 2^31 stored edges");
  std::vector<int32_t> par;
  std::vector<int64_t> ln;
  PPRVIZ_TRY(louvain_plus_solve(ctx, g, k, par, ln, info));
  if (info->levels > level_cap || info->parent_need > parent_cap)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "Louvain+: level_n or parent too short for the hierarchy (see info)");
  memcpy(level_n, ln.data(), sizeof(int64_t) * ln.size());
  if (!par.empty()) memcpy(parent, par.data(), sizeof(int32_t) * par.size());
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_tau_push(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr,
                    const int32_t *leaf_idx, const double *dpr, double alpha, double eps, double delta, double tau,
                    void *ldppr_out, void *pdist_out, int64_t n_clamp, pprviz_tau_info *info, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (info) memset(info, 0, sizeof(*info));
  if (!g || !leaf_ptr || !leaf_idx) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph or leaf sets are NULL");
  if (!dpr) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "the DPR index is NULL");
  if (nsup < 1 || (int64_t)nsup > g->n || nsup > 65535)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "nsup must be in [1, min(n, 65535)]");
  if ((int64_t)nsup * g->n >= ((int64_t)1 << 31))
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "nsup * n must stay below 2^31 (the residue entries are int32-indexed)");
  if (g->nnz >= ((int64_t)1 << 31))
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "Tau-Push takes graphs below 2^31 stored edges");
  if (!(alpha > 0.0 && alpha < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(eps > 0.0) || !isfinite(eps)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "eps must be finite and > 0");
  if (!(delta > 0.0) || !isfinite(delta)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "delta must be finite and > 0");
  if (!isfinite(tau)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "tau must be finite (<= 0 selects 1 / sqrt(k n))");
  if (n_clamp == 0) n_clamp = g->n;
  if (n_clamp < 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "n_clamp must be >= 2");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool out64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  std::vector<int64_t> lp;
  std::vector<int32_t> li;
  const int64_t *lp_d = nullptr;
  const int32_t *li_d = nullptr;
  PPRVIZ_TRY(leaf_sets_in(ctx, g, nsup, leaf_ptr, leaf_idx, dev, lp, li, &lp_d, &li_d));
  // the DPR index: checked on the host (a negative or non-finite entry is an error)
  std::vector<double> dh((size_t)g->n);
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(dh.data(), dpr, sizeof(double) * dh.size(), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    memcpy(dh.data(), dpr, sizeof(double) * dh.size());
  }
  for (double x : dh)
    if (!(x >= 0.0) || !isfinite(x)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "DPR entries must be finite and >= 0");
  const double *dpr_d = dpr;
  if (!dev) {
    const void *p = nullptr;
    PPRVIZ_TRY(stage_in(ctx, dh.data(), sizeof(double) * dh.size(), false, WS_OUT1, &p));
    dpr_d = (const double *)p;
  }
  const size_t kk = (size_t)nsup * (size_t)nsup;
  const size_t ob = (out64 ? sizeof(double) : sizeof(float)) * kk;
  void *ld_d = nullptr;
  if (ldppr_out && dev) ld_d = ldppr_out;
  else {
    PPRVIZ_TRY(ws_ensure(ctx, WS_DPPR, ob));
    ld_d = ctx->ws[WS_DPPR].p;
  }
  const int status = tau_push_solve(ctx, g, nsup, lp_d, li_d, lp, dpr_d, alpha, eps, delta, tau, ld_d, out64, info);
  if (status != PPRVIZ_OK) return finish(ctx, status);
  if (pdist_out) {
    void *pd_d = dev ? pdist_out : nullptr;
    if (!pd_d) {
      PPRVIZ_TRY(ws_ensure(ctx, WS_PDIST, ob));
      pd_d = ctx->ws[WS_PDIST].p;
    }
    PPRVIZ_TRY(pdist_launch(ctx, ld_d, nsup, n_clamp, pd_d, out64));
    if (!dev) PPRVIZ_CUDA(ctx, cudaMemcpyAsync(pdist_out, pd_d, ob, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (ldppr_out && !dev) PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ldppr_out, ld_d, ob, cudaMemcpyDeviceToHost, ctx->stream));
  if (!dev) PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_frontier_profile(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view, int32_t k, double alpha,
                            double eps, int32_t sweeps, int64_t *active_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!g || !view || !active_out) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "graph, view or output is NULL");
  if (k < 1 || (int64_t)k > g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be in [1, n]");
  if (sweeps < 1 || sweeps > 100000) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "sweeps must be in [1, 100000]");
  if (!(alpha > 0.0 && alpha < 1.0)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1)");
  if (!(eps > 0.0) || !isfinite(eps)) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "eps must be finite and > 0");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  std::vector<int32_t> view_h((size_t)k);
  const int32_t *view_d = nullptr;
  if (dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(view_h.data(), view, sizeof(int32_t) * k, cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    view_d = view;
  } else {
    memcpy(view_h.data(), view, sizeof(int32_t) * k);
    const void *p = nullptr;
    PPRVIZ_TRY(stage_in(ctx, view, sizeof(int32_t) * k, false, WS_VIEW, &p));
    view_d = (const int32_t *)p;
  }
  PPRVIZ_TRY(view_check(ctx, g, view_d, k));
  return finish(ctx, frontier_profile(ctx, g, view_d, view_h, k, alpha, eps, sweeps, active_out));
}

int pprviz_layout_metrics(pprviz_ctx *ctx, const void *x, int32_t k, const pprviz_graph *g, const int32_t *view,
                          double *nd_out, double *ulcv_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!x || k < 1) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "x is NULL or k < 1");
  if (ulcv_out && !g) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "ULCV needs the graph");
  if (g && !view && (int64_t)k != g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "without a view, k must be n");
  if (g && view && (int64_t)k > g->n) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be <= n");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool f64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  const void *xd = nullptr;
  PPRVIZ_TRY(stage_in(ctx, x, (f64 ? sizeof(double) : sizeof(float)) * 2 * (size_t)k, dev, WS_IN0, &xd));
  const int32_t *view_d = nullptr;
  if (g && view) {
    const void *p = nullptr;
    PPRVIZ_TRY(stage_in(ctx, view, sizeof(int32_t) * (size_t)k, dev, WS_VIEW, &p));
    view_d = (const int32_t *)p;
    PPRVIZ_TRY(view_check(ctx, g, view_d, k));
  }
  return finish(ctx, layout_metrics(ctx, xd, f64, k, g, view_d, nd_out, ulcv_out));
}

int pprviz_pdist(pprviz_ctx *ctx, const void *dppr, int32_t k, int64_t n_clamp, void *pdist_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!dppr || !pdist_out) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "NULL buffer");
  if (k < 1) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be >= 1");
  if (n_clamp < 2) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "n_clamp must be >= 2");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool f64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  const size_t bytes = (f64 ? sizeof(double) : sizeof(float)) * (size_t)k * k;
  const void *in_d = nullptr;
  PPRVIZ_TRY(stage_in(ctx, dppr, bytes, dev, WS_IN0, &in_d));
  void *out_d = pdist_out;
  if (!dev) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_OUT0, bytes));
    out_d = ctx->ws[WS_OUT0].p;
  }
  PPRVIZ_TRY(pdist_launch(ctx, in_d, k, n_clamp, out_d, f64));
  if (!dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(pdist_out, out_d, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_layout(pprviz_ctx *ctx, const void *pdist, int32_t k, const void *x0, int32_t iters, int precision,
                  void *x_out, double *stress_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!pdist || !x0 || !x_out) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "NULL buffer");
  if (k < 1 || iters < 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be >= 1 and iters >= 0");
  if (precision != PPRVIZ_FP64 && precision != PPRVIZ_FP32)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "precision must be PPRVIZ_FP64 or PPRVIZ_FP32");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool io64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  const size_t es = io64 ? sizeof(double) : sizeof(float);
  const void *pd = nullptr, *xd = nullptr;
  PPRVIZ_TRY(stage_in(ctx, pdist, es * (size_t)k * k, dev, WS_IN0, &pd));
  PPRVIZ_TRY(stage_in(ctx, x0, es * 2 * (size_t)k, dev, WS_IN1, &xd));
  void *xo = x_out;
  if (!dev) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_OUT0, es * 2 * (size_t)k));
    xo = ctx->ws[WS_OUT0].p;
  }
  int s = layout_run(ctx, pd, k, xd, iters, precision, io64, xo, stress_out);
  if (s != PPRVIZ_OK) return finish(ctx, s);
  if (!dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(x_out, xo, es * 2 * (size_t)k, cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_energy(pprviz_ctx *ctx, const void *pdist, int32_t k, const void *x, double grad_scale, double *e_out,
                  void *grad_x, void *grad_pdist, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (!pdist || !x) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "NULL buffer");
  if (k < 1) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "k must be >= 1");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  const bool f64 = (mem_flags & PPRVIZ_OUT_FP64) != 0;
  const size_t es = f64 ? sizeof(double) : sizeof(float);
  const void *pd = nullptr, *xd = nullptr;
  PPRVIZ_TRY(stage_in(ctx, pdist, es * (size_t)k * k, dev, WS_IN0, &pd));
  PPRVIZ_TRY(stage_in(ctx, x, es * 2 * (size_t)k, dev, WS_IN1, &xd));
  void *gx = grad_x, *gd = grad_pdist;
  if (!dev) {
    if (grad_x) {
      PPRVIZ_TRY(ws_ensure(ctx, WS_OUT0, es * 2 * (size_t)k));
      gx = ctx->ws[WS_OUT0].p;
    }
    if (grad_pdist) {
      PPRVIZ_TRY(ws_ensure(ctx, WS_PDIST, es * (size_t)k * k));
      gd = ctx->ws[WS_PDIST].p;
    }
  }
  int s = energy_run(ctx, pd, k, xd, grad_scale, f64, e_out, gx, gd);
  if (s != PPRVIZ_OK) return finish(ctx, s);
  if (!dev) {
    if (grad_x) PPRVIZ_CUDA(ctx, cudaMemcpyAsync(grad_x, gx, es * 2 * (size_t)k, cudaMemcpyDeviceToHost, ctx->stream));
    if (grad_pdist)
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(grad_pdist, gd, es * (size_t)k * k, cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return finish(ctx, PPRVIZ_OK);
}

int pprviz_views_batch(pprviz_ctx *ctx, int32_t nviews, const pprviz_graph *const *views, const int64_t *offsets,
                       double alpha, double eps, int32_t iters, const float *x0_packed, float *pdist_packed,
                       float *x_packed, double *stress_out, double *cert_out, uint32_t mem_flags) {
  if (!ctx) return PPRVIZ_E_INVALID_ARG;
  PPRVIZ_TRY(begin(ctx));
  if (nviews < 1 || !views || !offsets || !x0_packed || !x_packed)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "bad views arguments");
  if (iters < 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "iters must be >= 0");
  if (!(alpha > 0.0 && alpha < 1.0) || !(eps > 0.0))
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "alpha must be in (0, 1) and eps > 0");
  const bool dev = (mem_flags & PPRVIZ_DEVICE_PTRS) != 0;
  std::vector<int64_t> ks((size_t)nviews);
  int64_t sq_total = 0, maxk = 0;
  for (int32_t v = 0; v < nviews; ++v) {
    const pprviz_graph *g = views[v];
    if (!g) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "NULL view graph");
    const int64_t nv = offsets[v + 1] - offsets[v];
    if (nv != g->n || offsets[v] < 0) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "offsets do not match the view sizes");
    ks[v] = nv;
    sq_total += nv * nv;
    maxk = std::max(maxk, nv);
  }
  const int64_t ntot = offsets[nviews];
  // packed device buffers: all PDists, initial and final coordinates
  float *pdist_all = nullptr, *x0_all = nullptr, *x_all = nullptr;
  if (dev && pdist_packed) pdist_all = pdist_packed;
  else {
    PPRVIZ_TRY(ws_ensure(ctx, WS_BPD, sizeof(float) * (size_t)sq_total));
    pdist_all = ctx->ws[WS_BPD].as<float>();
  }
  const void *x0p = nullptr;
  PPRVIZ_TRY(stage_in(ctx, x0_packed, sizeof(float) * 2 * (size_t)ntot, dev, WS_BXIN, &x0p));
  x0_all = (float *)x0p;
  if (dev) x_all = x_packed;
  else {
    PPRVIZ_TRY(ws_ensure(ctx, WS_BXOUT, sizeof(float) * 2 * (size_t)ntot));
    x_all = ctx->ws[WS_BXOUT].as<float>();
  }
  // DPPR and PDist of all views: waves of similar-size views share every launch
  PPRVIZ_TRY(ws_ensure(ctx, WS_VIEW, sizeof(int32_t) * (size_t)maxk));
  int32_t *view_d = ctx->ws[WS_VIEW].as<int32_t>();
  std::vector<int32_t> iota((size_t)maxk);
  for (int64_t q = 0; q < maxk; ++q) iota[q] = (int32_t)q;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(view_d, iota.data(), sizeof(int32_t) * maxk, cudaMemcpyHostToDevice, ctx->stream));
  std::vector<int64_t> sq_off((size_t)nviews + 1, 0);
  for (int32_t v = 0; v < nviews; ++v) sq_off[v + 1] = sq_off[v] + ks[v] * ks[v];
  int status = dppr_views_solve(ctx, nviews, views, offsets, sq_off.data(), alpha, eps, view_d, pdist_all, cert_out);
  if (status != PPRVIZ_OK && status != PPRVIZ_E_NOT_CONVERGED) return finish(ctx, status);
  const std::string dppr_err = ctx->err;
  pprviz_stats acc = ctx->stats;
  // all layouts together: one launch per pass over every view's tiles
  int s = layout_batch_run(ctx, nviews, ks.data(), pdist_all, x0_all, iters, x_all, stress_out);
  if (s != PPRVIZ_OK) return finish(ctx, s);
  ctx->stats.groups = acc.groups;
  ctx->stats.sweeps_main = acc.sweeps_main;
  ctx->stats.sweeps_refine = acc.sweeps_refine;
  ctx->stats.refine_passes = acc.refine_passes;
  ctx->stats.residual_passes = acc.residual_passes;
  ctx->stats.max_cert = acc.max_cert;
  ctx->stats.bytes_sweep = acc.bytes_sweep;
  if (!dev) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(x_packed, x_all, sizeof(float) * 2 * (size_t)ntot, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    if (pdist_packed)
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(pdist_packed, pdist_all, sizeof(float) * (size_t)sq_total,
                                       cudaMemcpyDeviceToHost, ctx->stream));
  }
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (status != PPRVIZ_OK) ctx->err = dppr_err;
  return finish(ctx, status);
}

}  // extern "C"
