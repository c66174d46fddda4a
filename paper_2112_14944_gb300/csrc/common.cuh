// Internal declarations shared by the translation units of libpprviz.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "pprviz.h"

namespace pprviz {

// A grow-only device buffer owned by a context or a graph.
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
  template <class T>
  T *as() const { return reinterpret_cast<T *>(p); }
};

// Workspace slots of a context.
enum Slot {
  WS_VIEW = 0, WS_SRC, WS_Y0, WS_Y1, WS_Y2, WS_Y3, WS_RHS, WS_CERT, WS_FLAG,
  WS_DPPR, WS_PDIST, WS_IN0, WS_IN1, WS_OUT0, WS_OUT1, WS_W1, WS_M, WS_PIV,
  WS_B, WS_X, WS_E, WS_MISC,
  // batched views
  WS_BW1, WS_BM, WS_BX, WS_BPART, WS_BTAB, WS_BPD, WS_BXIN, WS_BXOUT,
  // deflated sweeps: spectral scratch, residual partials, per-source roots and coefficients
  WS_SPEC, WS_RPART, WS_CSRC, WS_KAPPA,
  // tensor maps of the layout pass matrices, row-block table of the reduce
  WS_TMAP, WS_TROWS, WS_TREC, WS_RUNP,
  // batched propagation: the union graph of the views and its tables
  WS_URP, WS_UCOL, WS_UW, WS_UDEG, WS_UINVD, WS_UINVF, WS_UDWFF, WS_ULIDX, WS_UNV, WS_UCOMP, WS_UKAP,
  WS_UDESC, WS_UBROWS, WS_UBPTR,
  // batched inverses: panels and pivot inverses of every view, job and step tables
  WS_FACB, WS_FACT,
  // split heavy rows of the FP32 sweeps: per-segment partial sums and arrival counters
  WS_SPART, WS_SCNT,
  // batched views: the waves' split work items and split rows
  WS_UITEMS, WS_USROW,
  // Tau-Push: residues, reserves, push records, (slot, share) pairs, dirty
  // marks, per-round counters, leaf maps and small per-supernode tables
  WS_TPR, WS_TPQ, WS_TPFA, WS_TPFB, WS_TPVAL, WS_TPCNT, WS_TPMAP, WS_TPTAB,
  // Louvain+: per-node round state, scan scratch, the level pair lists, the pair table
  WS_LPNODE, WS_LPSCAN, WS_LPEDGE, WS_LPHASH,
  WS_COUNT
};

}  // namespace pprviz

struct pprviz_ctx {
  // per-class device timing (pprviz_profile / pprviz_kernel_times)
  bool profiling = false;
  bool capturing = false;  // launches are being recorded into a CUDA graph
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev_pending;
  double class_ms[PPRVIZ_NKCLASS] = {0};
  int64_t class_launches[PPRVIZ_NKCLASS] = {0};
  int64_t class_timed[PPRVIZ_NKCLASS] = {0};  // launches whose device time is in class_ms
  int prof_every = 1;                         // sampling period of the hot classes
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  // second stream and events of the FP32 inverse's lookahead (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_t1 = nullptr, ev_dp = nullptr;
  std::string err;
  pprviz::DevBuf ws[pprviz::WS_COUNT];
  size_t ws_limit = 0;  // cap on the summed workspace capacity (0 = none); pprviz_set_workspace_limit
  bool test_expire_wait = false;  // pprviz_test_expire_wait: the next FP32 inverse withholds one copy
  bool scnt_clear = false;        // the split sweep's arrival counters are zero (set per call)
  pprviz_stats stats{};
  int launches = 0;  // kernels launched in the current call
  // source-group widths chosen by the sweep autotuner, by graph size class
  std::vector<std::pair<uint64_t, int64_t>> tuned_groups;
};

struct pprviz_graph {
  pprviz_ctx *ctx = nullptr;  // the uploading context; not used by pprviz_graph_free
  int device = 0;             // its device, for freeing after the context is gone
  int64_t n = 0, nnz = 0;
  bool weighted = false;
  uint32_t flags = 0;
  pprviz::DevBuf rp, col, w, deg, invdw_f, invdw_d;
  pprviz::DevBuf dwff;  // walk degree as a float pair (hi, lo), hi + lo = dw to ~2^-48
  double m = 0.0;
  std::vector<double> h_deg;  // host copy of d(v), for per-group decisions
  // dense weight matrix for the tensor-core sweeps, built on first use
  mutable pprviz::DevBuf dense;
  mutable int64_t dense_nw = 0;
  // component roots and spectral bound for the deflated sweeps, on first use
  mutable pprviz::DevBuf comp;             // root (smallest id) of each node's component
  mutable std::vector<int32_t> h_comp;     // host copy
  mutable std::vector<double> h_mc;        // m_C = sum of walk degrees, indexed by root
  mutable double spec_b = 1.0;             // |lambda| <= spec_b off the stationary modes (estimate + margin)
  mutable bool spec_deflate = false;       // components resolved
  mutable bool spec_ready = false;
  // sweep work items with heavy rows split into segments of at most 64 edges,
  // built on first use (sweep_plan in propagate.cu)
  mutable pprviz::DevBuf sp_items, sp_srow;
  mutable int64_t sp_nitems = 0, sp_nsplit = 0, sp_nslots = 0;
  mutable bool sp_ready = false;
  // directed graphs: the pull CSR (row j lists the in-neighbours i of j with
  // the weights w_ij, or 1; a dangling j has the entry (j, 1), a j without
  // in-edges the entry (j, 0)), so that no gather row is empty
  bool directed = false;
  pprviz::DevBuf prp, pcol, pw;
};

namespace pprviz {
// The CSR the pull-form kernels gather over: the graph itself when it is
// undirected, its pull CSR when it is directed (always weighted).
inline const int64_t *pull_rp(const pprviz_graph *g) { return g->directed ? g->prp.as<int64_t>() : g->rp.as<int64_t>(); }
inline const int32_t *pull_col(const pprviz_graph *g) {
  return g->directed ? g->pcol.as<int32_t>() : g->col.as<int32_t>();
}
inline const float *pull_w(const pprviz_graph *g) {
  return g->directed ? g->pw.as<float>() : (g->weighted ? g->w.as<float>() : nullptr);
}
inline bool pull_weighted(const pprviz_graph *g) { return g->directed || g->weighted; }
}  // namespace pprviz

namespace pprviz {

// ---- status helpers -------------------------------------------------------
int set_err(pprviz_ctx *ctx, int code, const std::string &msg);
int cuda_err(pprviz_ctx *ctx, cudaError_t e, const char *what);

#define PPRVIZ_CUDA(ctx, call)                                   \
  do {                                                           \
    cudaError_t e__ = (call);                                    \
    if (e__ != cudaSuccess) return ::pprviz::cuda_err(ctx, e__, #call); \
  } while (0)

#define PPRVIZ_LAUNCHED(ctx)                                             \
  do {                                                                   \
    (ctx)->launches++;                                                   \
    cudaError_t e__ = cudaGetLastError();                                \
    if (e__ != cudaSuccess) return ::pprviz::cuda_err(ctx, e__, "kernel launch"); \
  } while (0)

#define PPRVIZ_TRY(expr)        \
  do {                          \
    int s__ = (expr);           \
    if (s__ != PPRVIZ_OK) return s__; \
  } while (0)

int ws_ensure(pprviz_ctx *ctx, int slot, size_t bytes);

// Brackets the kernel launches of one scope with CUDA events on the context
// stream when profiling is on, and counts them per class either way.
struct ProfScope {
  pprviz_ctx *c;
  int cls;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(pprviz_ctx *ctx, int k);
  ~ProfScope();
};
#define PPRVIZ_PROF(ctx, cls) ::pprviz::ProfScope prof_scope__(ctx, cls)

// ---- graph (graph.cu) ---------------------------------------------------
int graph_build(pprviz_ctx *ctx, pprviz_graph *g, uint32_t flags);
// The pull CSR of a directed graph from host copies of its out-edge CSR;
// marks the graph directed.
int pull_csr_build(pprviz_ctx *ctx, pprviz_graph *g, const int64_t *rp, const int32_t *col, const float *w);
// Map view ids -> check range and duplicates on the device. `view_d` device.
int view_check(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d, int32_t k);

// ---- propagation (propagate.cu) ----------------------------------------
// Computes DPPR rows for all k view sources into dppr_d (k*k, double if
// out64 else float, row-major, ld k) and certificates into cert_h (host, k).
int dppr_solve(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d,
               const std::vector<int32_t> &view_h, int32_t k, double alpha, double eps,
               int precision, void *dppr_d, bool out64, double *cert_h);

// All-pairs DPPR and PDist of many views (each view: every node a source,
// n_clamp = its size) in shared launches. node_off: nviews + 1 prefix sums
// of the sizes (cert_h order); sq_off: prefix sums of the squared sizes
// (pdist_all order, device FP32); iota_d: 0 .. max n - 1 on the device.
int dppr_views_solve(pprviz_ctx *ctx, int32_t nviews, const pprviz_graph *const *views, const int64_t *node_off,
                     const int64_t *sq_off, double alpha, double eps, const int32_t *iota_d, float *pdist_all,
                     double *cert_h);

// Level-l DPPR between nsup supernodes with disjoint, non-empty leaf sets
// (CSR leaf_ptr / leaf_idx, on the device and the host); out_d: nsup x nsup
// row-major (source supernode = row), double if out64; cert_h: nsup
// certificates ||res||_1 / alpha.
int level_dppr_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr_d,
                     const int32_t *leaf_idx_d, const std::vector<int64_t> &leaf_ptr_h,
                     const std::vector<int32_t> &leaf_idx_h, double alpha, double eps, void *out_d, bool out64,
                     double *cert_h);

// Per power-iteration sweep t < sweeps, the number of (node, source) entries
// of the k view sources whose push residue exceeds d(v) eps / max_view d
// (active_h: host, sweeps entries).
int frontier_profile(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d,
                     const std::vector<int32_t> &view_h, int32_t k, double alpha, double eps, int32_t sweeps,
                     int64_t *active_h);

// ---- Tau-Push and its DPR index (taupush.cu) -------------------------------
// DPR of every node into dpr_d (device, n doubles); cert_h: (1 - alpha)^(T+1).
int dpr_solve(pprviz_ctx *ctx, const pprviz_graph *g, double alpha, double eps, double *dpr_d, double *cert_h);
// Tau-Push estimates (nsup x nsup, row = source) into out_d (double if out64);
// leaf sets on the device and the host (validated); dpr_d: device, n doubles.
int tau_push_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr_d,
                   const int32_t *leaf_idx_d, const std::vector<int64_t> &leaf_ptr_h, const double *dpr_d,
                   double alpha, double eps, double delta, double tau, void *out_d, bool out64,
                   pprviz_tau_info *info);

// ---- Louvain+ hierarchy (louvain.cu) ----------------------------------------
// The hierarchy of an undirected graph with at most k children per supernode:
// parents = the parent arrays of levels 1..L concatenated, level_n = n and the
// sizes of levels 1..L (host); info: filled (levels, parent_need, counters).
int louvain_plus_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t k, std::vector<int32_t> &parents,
                       std::vector<int64_t> &level_n, pprviz_louvain_info *info);

// ---- graph analysis for the deflated sweeps (spectral.cu) ------------------
// Fills g->comp / h_comp / h_mc / spec_b / spec_deflate once per graph.
int graph_spectral(pprviz_ctx *ctx, const pprviz_graph *g);

// ---- dense tensor-core sweeps (dense.cu) ----------------------------------
// True when the graph holds enough of all pairs for a dense contraction to
// beat the CSR gathers.
bool dense_eligible(const pprviz_graph *g);
// Source-group width of the dense path (multiple of 128).
int64_t dense_group(int32_t k);
// Builds g->dense (n x n weights, zero padded) if absent; E_OOM if it does not fit.
int dense_prepare(pprviz_ctx *ctx, const pprviz_graph *g);
// One Chebyshev sweep of a group with the semantics of the CSR sweep; yold is
// overwritten with the new iterate; err gets bit 0 if an MMA wait expired.
// bf16: BF16 operands (kind::f16) instead of the 3xTF32 split.
int dense_sweep(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src, const float *rhs,
                const float *ycur, float *yold, double alpha, double om, int *err, bool bf16);

// ---- layout quality metrics (metrics.cu) ----------------------------------
// ND and ULCV (Sec. 2) of k coordinates x_d (device, k x 2, double if f64);
// ULCV over the edges of g among the view's nodes (view_d: k node ids of g, or
// NULL when row i is node i). nd_h / ulcv_h: host outputs, either may be NULL.
int layout_metrics(pprviz_ctx *ctx, const void *x_d, bool f64, int32_t k, const pprviz_graph *g,
                   const int32_t *view_d, double *nd_h, double *ulcv_h);

// ---- pdist (pdist.cu) ------------------------------------------------------
int pdist_launch(pprviz_ctx *ctx, const void *dppr_d, int32_t k, int64_t n_clamp,
                 void *pdist_d, bool f64);

// ---- factor (factor.cu) ----------------------------------------------------
// In-place inverse of the SPD kp x kp matrix A (kp % 128 == 0); on return A
// holds A^-1 on its upper 64-block triangle and on the 128 x 128 diagonal tiles.
// `work` holds spd_inverse_work(kp) elements: two sets (the lookahead's
// parities) of panels (2 x 2 NB x kp: Ct and Ut split into high and low
// parts, NB = 128) and pivot inverse (NB x NB), and a status word. The FP32 version runs its trailing updates on the tensor cores and
// returns PPRVIZ_E_TIMEOUT if an MMA completion wait expires.
size_t spd_inverse_work(int32_t kp);  // elements of `work` for either type
int spd_inverse_f32(pprviz_ctx *ctx, int32_t kp, float *A, float *work);
// FP32 inverses of many SPD matrices at once (A[v]: kp[v] x kp[v] device,
// kp[v] % 128 == 0), in place as spd_inverse_f32; `work` holds
// spd_inverse_batch_work(nviews, kp) floats.
size_t spd_inverse_batch_work(int32_t nviews, const int32_t *kp);
int spd_inverse_batch_f32(pprviz_ctx *ctx, int32_t nviews, const int32_t *kp, float *const *A, float *work);
int spd_inverse_f64(pprviz_ctx *ctx, int32_t kp, double *A, double *work);

// ---- layout (layout.cu) ----------------------------------------------------
int layout_run(pprviz_ctx *ctx, const void *pdist_d, int32_t k, const void *x0_d, int32_t iters,
               int precision, bool io64, void *x_out_d, double *stress_h);
// FP32 layouts of many views: pdist_d packs the k_v x k_v matrices in order,
// x0_d / x_out_d the k_v x 2 coordinates; stress_h gets one value per view.
int layout_batch_run(pprviz_ctx *ctx, int32_t nviews, const int64_t *k_h, const float *pdist_d,
                     const float *x0_d, int32_t iters, float *x_out_d, double *stress_h);
int energy_run(pprviz_ctx *ctx, const void *pdist_d, int32_t k, const void *x_d, double scale,
               bool f64, double *e_h, void *grad_x_d, void *grad_pdist_d);

}  // namespace pprviz
