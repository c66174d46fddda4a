// Tau-Push (Sec. 4, Algorithms 1-3) as synchronous frontier pushes on the
// GPU, and the DPR index it reads (Eq. (dnpr-dnppr), Sec. 4.3).
//
// The paper's pushes are sequential: one node at a time, in no stated order.
// Here every (node, supernode) residue above its threshold is pushed in the
// same round. A round is two launches:
//   prepass  one thread per frontier entry: take the residue (atomic
//            exchange with 0), add the reserve share if the node is a leaf of
//            a child, and cut the node's edge list into push items of 32
//            edges;
//   push     one warp per item, one edge per lane: FP64 atomic add of the
//            share into the neighbour's residue; the lane whose add lifts the
//            residue over its threshold appends the neighbour to the next
//            frontier (so a residue is listed at most once per round).
// A residue taken in a round can grow again in the same round; the growth
// stays in the residue and, if it crosses the threshold, lists the node for
// the next round. No residue is lost and none above its threshold is left
// unlisted, so the rounds end exactly when Algorithm 2's (or 3's) loop
// condition fails, and the error bounds of Lemmas 2 and 3 hold as stated.
//
// Data layout: residues node-major (n x K doubles, K = sources or targets of
// the phase), so a hub reached by many supernodes keeps its K residues in a
// few cache lines; reserves only for the leaves of the children
// (leaves x K doubles, indexed by the leaf's position in leaf_idx).
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace pprviz {
namespace {

constexpr int TP_CH = 32;                  // edges per push item
constexpr int TP_TPB = 256;
constexpr int64_t TP_MAX_ROUNDS = 65535;   // a phase still active after this many rounds fails
constexpr int64_t DPR_HEAVY = 512;         // pull rows longer than this get a block of their own

struct TpEntry {
  int32_t v, s;  // node, source (forward) or target slot (backward)
};
struct TpItem {
  int32_t e, c;  // frontier entry, chunk of 32 edges
};

// Per-phase device counters: frontier size and item count of every round,
// the edges cut into items, and an overflow flag.
struct TpCounters {
  unsigned long long front[TP_MAX_ROUNDS + 2];
  unsigned long long items[TP_MAX_ROUNDS + 2];
  unsigned long long edges;
  int overflow;
};

__device__ __forceinline__ double take_residue(double *p) {
  return __longlong_as_double((long long)atomicExch(reinterpret_cast<unsigned long long *>(p), 0ull));
}

// pos_of[v] = position of v in leaf_idx (pos_of prefilled with -1)
__global__ void k_tp_pos(int64_t nleaf, const int32_t *__restrict__ leaf_idx, int32_t *__restrict__ pos_of) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < nleaf) pos_of[leaf_idx[p]] = (int32_t)p;
}

// psup[p] = the supernode whose leaf list holds position p (one block per supernode)
__global__ void k_tp_psup(const int64_t *__restrict__ leaf_ptr, int32_t *__restrict__ psup) {
  const int32_t j = blockIdx.x;
  for (int64_t p = leaf_ptr[j] + threadIdx.x; p < leaf_ptr[j + 1]; p += blockDim.x) psup[p] = j;
}

// Fixed-order block sum (deterministic for a given launch shape).
__device__ double block_sum(double v, double *sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;  // valid in thread 0
}

// Per supernode j: the mean leaf degree and the mean leaf DPR (tau_j of
// Eq. (dnpr-dnppr)); out[2 j] = mean d, out[2 j + 1] = tau_j.
__global__ void k_tp_means(const int64_t *__restrict__ leaf_ptr, const int32_t *__restrict__ leaf_idx,
                           const double *__restrict__ deg, const double *__restrict__ dpr, double *__restrict__ out) {
  __shared__ double sh[TP_TPB / 32];
  const int32_t j = blockIdx.x;
  const int64_t lo = leaf_ptr[j], hi = leaf_ptr[j + 1];
  double sd = 0.0, st = 0.0;
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) {
    const int32_t v = leaf_idx[p];
    sd += deg[v];
    st += dpr[v];
  }
  sd = block_sum(sd, sh);
  if (threadIdx.x == 0) out[2 * j] = sd / (double)(hi - lo);
  st = block_sum(st, sh);
  if (threadIdx.x == 0) out[2 * j + 1] = st / (double)(hi - lo);
}

// Forward start (Algorithm 2, initial residues): r(V_i, v) = d(v) / |F(V_i)|
// on the leaves of every source V_i; the ones above d(v) r_max form round 0.
__global__ void k_tp_fwd_init(int64_t nleaf, const int64_t *__restrict__ leaf_ptr,
                              const int32_t *__restrict__ leaf_idx, const int32_t *__restrict__ psup, int32_t K,
                              const double *__restrict__ deg, double r_max, double *__restrict__ R,
                              TpEntry *__restrict__ front, TpCounters *__restrict__ cnt) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nleaf) return;
  const int32_t i = psup[p], v = leaf_idx[p];
  const double r = deg[v] / (double)(leaf_ptr[i + 1] - leaf_ptr[i]);
  R[(size_t)v * K + i] = r;
  if (r > deg[v] * r_max) {
    const unsigned long long q = atomicAdd(&cnt->front[0], 1ull);
    front[q] = TpEntry{v, i};
  }
}

// Backward start (Algorithm 3, initial residues): r(v, V_j) = 1 / |F(V_j)| on
// the leaves of every refined target V_j (slot[j] >= 0); above thr_b form round 0.
__global__ void k_tp_bwd_init(int64_t nleaf, const int64_t *__restrict__ leaf_ptr,
                              const int32_t *__restrict__ leaf_idx, const int32_t *__restrict__ psup,
                              const int32_t *__restrict__ slot, int32_t K, const double *__restrict__ thr_b,
                              double *__restrict__ R, TpEntry *__restrict__ front, TpCounters *__restrict__ cnt) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nleaf) return;
  const int32_t j = psup[p], jb = slot[j];
  if (jb < 0) return;
  const int32_t v = leaf_idx[p];
  const double r = 1.0 / (double)(leaf_ptr[j + 1] - leaf_ptr[j]);
  R[(size_t)v * K + jb] = r;
  if (r > thr_b[jb]) {
    const unsigned long long q = atomicAdd(&cnt->front[0], 1ull);
    front[q] = TpEntry{v, jb};
  }
}

// Round prepass. Forward (Algorithm 2): the reserve of a leaf gains
// alpha r (the estimate's alpha r / |F(V_j)| is applied when the reserves are
// summed), and the share (1 - alpha) r / dw(v) waits for the push. Backward
// (Algorithm 3): the reserve gains alpha d(v) r and the share is (1 - alpha) r.
// A node without out-edges keeps the walk (a self-loop): the sum of its
// endless pushes is taken at once - forward, the whole residue is reserve and
// nothing moves; backward, the reserve gains d(v) r (= 0) and the other
// in-neighbours receive (1 - alpha) r / alpha times their walk probability.
template <bool BWD>
__global__ void __launch_bounds__(TP_TPB)
    k_tp_prepass(int64_t round, const TpEntry *__restrict__ front, int32_t K, double *__restrict__ R,
                 double *__restrict__ Q, const int32_t *__restrict__ pos_of, const int64_t *__restrict__ rp,
                 const int64_t *__restrict__ nrp, const double *__restrict__ deg,
                 const double *__restrict__ invdw, double alpha, double *__restrict__ val,
                 TpItem *__restrict__ items, int64_t item_cap, int64_t front_cap, TpCounters *__restrict__ cnt) {
  const int64_t F = min((int64_t)cnt->front[round], front_cap);  // beyond the cap only after an overflow
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < F; base += stride) {
    const int64_t e = base + lane;
    int32_t nch = 0;
    long long ne = 0;
    if (e < F) {
      const TpEntry en = front[e];
      const double r = take_residue(&R[(size_t)en.v * K + en.s]);
      const bool stays = rp[en.v + 1] == rp[en.v];
      const int32_t p = pos_of[en.v];
      if (!BWD) {
        if (p >= 0) Q[(size_t)p * K + en.s] += stays ? r : alpha * r;
        val[e] = stays ? 0.0 : (1.0 - alpha) * r * invdw[en.v];
        ne = stays ? 0 : (long long)(nrp[en.v + 1] - nrp[en.v]);
      } else {
        if (p >= 0) Q[(size_t)p * K + en.s] += (stays ? 1.0 : alpha) * deg[en.v] * r;
        val[e] = stays ? (1.0 - alpha) * r / alpha : (1.0 - alpha) * r;
        ne = (long long)(nrp[en.v + 1] - nrp[en.v]);
      }
      nch = (int32_t)((ne + TP_CH - 1) / TP_CH);
    }
    // warp prefix of the item counts; one atomic per warp
    int32_t incl = nch;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    long long ns = ne;
    for (int o = 16; o > 0; o >>= 1) ns += __shfl_down_sync(0xffffffffu, ns, o);
    const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long b0 = 0;
    if (lane == 31 && tot > 0) b0 = atomicAdd(&cnt->items[round], (unsigned long long)tot);
    b0 = __shfl_sync(0xffffffffu, b0, 31);
    if (lane == 0 && ns > 0) atomicAdd(&cnt->edges, (unsigned long long)ns);
    const int64_t first = (int64_t)b0 + incl - nch;
    if (first + nch > item_cap) {
      if (nch > 0) atomicOr(&cnt->overflow, 1);
    } else {
      for (int32_t c = 0; c < nch; ++c) items[first + c] = TpItem{(int32_t)e, c};
    }
  }
}

// Round push: one warp per item, one edge per lane. Forward shares go to the
// out-neighbours x with weight w(v, x) (1 unweighted) and threshold
// d(x) r_max; backward shares go to the in-neighbours x with the walk
// probability w(x, v) / dw(x) and the target's threshold thr_b.
template <bool BWD>
__global__ void __launch_bounds__(TP_TPB)
    k_tp_push(int64_t round, const TpItem *__restrict__ items, const TpEntry *__restrict__ front,
              const double *__restrict__ val, int32_t K, double *__restrict__ R, const int64_t *__restrict__ rp,
              const int64_t *__restrict__ nrp, const int32_t *__restrict__ ncol, const float *__restrict__ nw,
              const double *__restrict__ deg, const double *__restrict__ invdw, double r_max,
              const double *__restrict__ thr_b, TpEntry *__restrict__ next, int64_t next_cap, int64_t item_cap,
              TpCounters *__restrict__ cnt) {
  const int64_t I = min((int64_t)cnt->items[round], item_cap);  // beyond the cap only after an overflow
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < I; it += nwarps) {
    const TpItem im = items[it];
    const TpEntry en = front[im.e];
    const double share = val[im.e];
    const int64_t q = nrp[en.v] + (int64_t)im.c * TP_CH + lane;
    bool up = false;
    int32_t x = 0;
    if (q < nrp[en.v + 1]) {
      x = ncol[q];
      const double w = nw ? (double)nw[q] : 1.0;
      double add, thr;
      bool skip = false;
      if (!BWD) {
        add = share * w;
        thr = deg[x] * r_max;
      } else {
        skip = x == en.v && rp[en.v + 1] == rp[en.v];  // the walk's own self-loop, summed in the prepass
        add = share * w * invdw[x];
        thr = thr_b[en.s];
      }
      if (!skip && add > 0.0) {
        const double old = atomicAdd(&R[(size_t)x * K + en.s], add);
        up = old <= thr && old + add > thr;
      }
    }
    const unsigned b = __ballot_sync(0xffffffffu, up);
    if (b) {
      unsigned long long b0 = 0;
      const int leader = __ffs(b) - 1;
      if (lane == leader) b0 = atomicAdd(&cnt->front[round + 1], (unsigned long long)__popc(b));
      b0 = __shfl_sync(0xffffffffu, b0, leader);
      if (up) {
        const int64_t slot = (int64_t)b0 + __popc(b & ((1u << lane) - 1u));
        if (slot < next_cap) next[slot] = TpEntry{x, en.s};
        else atomicOr(&cnt->overflow, 2);
      }
    }
  }
}

// Estimates from the reserves. Forward: E[i][j] = sum_{p in F(V_j)} Q[p][i] / |F(V_j)|
// (block (j, i)). Backward: E[i][tsel[jb]] = sum_{p in F(V_i)} Q[p][jb] / |F(V_i)|
// (block (i, jb)). Fixed-order sums.
template <bool BWD>
__global__ void k_tp_collect(const int64_t *__restrict__ leaf_ptr, const double *__restrict__ Q, int32_t K,
                             int32_t nsup, const int32_t *__restrict__ tsel, double *__restrict__ E) {
  __shared__ double sh[TP_TPB / 32];
  const int32_t a = blockIdx.x, b = blockIdx.y;
  const int64_t lo = leaf_ptr[a], hi = leaf_ptr[a + 1];
  double s = 0.0;
  for (int64_t p = lo + threadIdx.x; p < hi; p += blockDim.x) s += Q[(size_t)p * K + b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) {
    const double est = s / (double)(hi - lo);
    if (!BWD) E[(size_t)b * nsup + a] = est;
    else E[(size_t)a * nsup + tsel[b]] = est;
  }
}

template <typename T>
__global__ void k_tp_out(int64_t cnt, const double *__restrict__ E, T *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (T)E[i];
}

// DPR power iteration, light rows: 8 lanes per pull row,
//   x_new(v) = alpha s(v) + (1 - alpha) sum_{u in pull(v)} w(u, v) x(u) / dw(u),
// s = d / m; an empty pull row (an isolated node of an undirected graph)
// keeps its own walk: x_new(v) = alpha s(v) + (1 - alpha) x(v).
__global__ void k_dpr_light(int64_t n, const int64_t *__restrict__ prp, const int32_t *__restrict__ pcol,
                            const float *__restrict__ pw, const double *__restrict__ invdw,
                            const double *__restrict__ deg, double inv_m, double alpha,
                            const double *__restrict__ x, double *__restrict__ y) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t v = t >> 3;
  const int sub = threadIdx.x & 7;
  if (v >= n) return;  // whole 8-lane groups leave together (n rows, 8 lanes each)
  const int64_t lo = prp[v], hi = prp[v + 1];
  if (hi - lo > DPR_HEAVY) return;  // done by k_dpr_heavy
  double acc = 0.0;
  for (int64_t q = lo + sub; q < hi; q += 8) {
    const int32_t u = pcol[q];
    acc += (pw ? (double)pw[q] : 1.0) * x[u] * invdw[u];
  }
  const unsigned gm = 0xffu << (threadIdx.x & 24);
  for (int o = 4; o > 0; o >>= 1) acc += __shfl_down_sync(gm, acc, o, 8);
  if (sub == 0) {
    if (hi == lo) acc = x[v];
    y[v] = alpha * deg[v] * inv_m + (1.0 - alpha) * acc;
  }
}

// DPR power iteration, heavy rows: one block per listed row.
__global__ void k_dpr_heavy(const int32_t *__restrict__ rows, const int64_t *__restrict__ prp,
                            const int32_t *__restrict__ pcol, const float *__restrict__ pw,
                            const double *__restrict__ invdw, const double *__restrict__ deg, double inv_m,
                            double alpha, const double *__restrict__ x, double *__restrict__ y) {
  __shared__ double sh[TP_TPB / 32];
  const int32_t v = rows[blockIdx.x];
  const int64_t lo = prp[v], hi = prp[v + 1];
  double acc = 0.0;
  for (int64_t q = lo + threadIdx.x; q < hi; q += blockDim.x) {
    const int32_t u = pcol[q];
    acc += (pw ? (double)pw[q] : 1.0) * x[u] * invdw[u];
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) y[v] = alpha * deg[v] * inv_m + (1.0 - alpha) * acc;
}

__global__ void k_dpr_heavy_list(int64_t n, const int64_t *__restrict__ prp, int32_t *__restrict__ rows,
                                 unsigned long long *__restrict__ cnt) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n && prp[v + 1] - prp[v] > DPR_HEAVY) rows[atomicAdd(cnt, 1ull)] = (int32_t)v;
}

__global__ void k_dpr_start(int64_t n, const double *__restrict__ deg, double inv_m, double alpha,
                            double *__restrict__ x) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < n) x[v] = alpha * deg[v] * inv_m;
}

unsigned blocks_for(int64_t cnt, int tpb) { return (unsigned)std::max<int64_t>(1, (cnt + tpb - 1) / tpb); }

}  // namespace

int dpr_solve(pprviz_ctx *ctx, const pprviz_graph *g, double alpha, double eps, double *dpr_d, double *cert_h) {
  const int64_t n = g->n;
  const double c = 1.0 - alpha;
  // after T iterations the walk mass not yet ended is c^(T+1)
  int64_t T = std::max<int64_t>(0, (int64_t)ceil(log(eps) / log(c)) - 1);
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPR, sizeof(double) * (size_t)n));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPMAP, sizeof(int32_t) * (size_t)n));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPTAB, 64));
  double *tmp = ctx->ws[WS_TPR].as<double>();
  int32_t *heavy = ctx->ws[WS_TPMAP].as<int32_t>();
  unsigned long long *hcnt = ctx->ws[WS_TPTAB].as<unsigned long long>();
  const int64_t *prp = pull_rp(g);
  const int32_t *pcol = pull_col(g);
  const float *pw = pull_w(g);
  const double *invdw = g->invdw_d.as<double>();
  const double *deg = g->deg.as<double>();
  const double inv_m = 1.0 / g->m;
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(hcnt, 0, sizeof(unsigned long long), ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_dpr_heavy_list<<<blocks_for(n, TP_TPB), TP_TPB, 0, ctx->stream>>>(n, prp, heavy, hcnt); }
  PPRVIZ_LAUNCHED(ctx);
  unsigned long long nheavy = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&nheavy, hcnt, sizeof(nheavy), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  // T iterations alternate between the caller's buffer and tmp so that the
  // last one lands in dpr_d
  double *a = (T % 2 == 0) ? dpr_d : tmp;
  double *b = (T % 2 == 0) ? tmp : dpr_d;
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_dpr_start<<<blocks_for(n, TP_TPB), TP_TPB, 0, ctx->stream>>>(n, deg, inv_m, alpha, a); }
  PPRVIZ_LAUNCHED(ctx);
  for (int64_t t = 0; t < T; ++t) {
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH);
      k_dpr_light<<<blocks_for(n * 8, TP_TPB), TP_TPB, 0, ctx->stream>>>(n, prp, pcol, pw, invdw, deg, inv_m, alpha,
                                                                        a, b);
    }
    PPRVIZ_LAUNCHED(ctx);
    if (nheavy) {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH); k_dpr_heavy<<<(unsigned)nheavy, TP_TPB, 0, ctx->stream>>>(heavy, prp, pcol, pw, invdw, deg, inv_m, alpha, a, b); }
      PPRVIZ_LAUNCHED(ctx);
    }
    std::swap(a, b);
  }
  ctx->stats.sweeps_main += T;
  if (cert_h) *cert_h = pow(c, (double)(T + 1));
  return PPRVIZ_OK;
}

namespace {

struct TpBufs {
  double *R, *Q, *val;
  TpEntry *fa, *fb;
  TpItem *items;
  TpCounters *cnt;
  int32_t *pos_of, *psup;
  int64_t front_cap, item_cap;
};

// Runs the rounds of one phase until a round starts with an empty frontier.
// Returns the number of rounds, the pushes (summed frontier sizes) and the
// edges cut into items.
template <bool BWD>
int tp_phase(pprviz_ctx *ctx, const pprviz_graph *g, const TpBufs &B, int32_t K, double alpha, double r_max,
             const double *thr_b, int64_t *rounds_out, int64_t *pushes_out, int64_t *edges_out) {
  const int64_t *rp = g->rp.as<int64_t>();
  const int64_t *nrp = BWD ? pull_rp(g) : g->rp.as<int64_t>();
  const int32_t *ncol = BWD ? pull_col(g) : g->col.as<int32_t>();
  const float *nw = BWD ? pull_w(g) : (g->weighted ? g->w.as<float>() : nullptr);
  const double *deg = g->deg.as<double>();
  const double *invdw = g->invdw_d.as<double>();
  const unsigned pre_grid = 152 * 4, push_grid = 152 * 8;
  int64_t r = 0;
  int batch = 4;
  unsigned long long head = 0;
  while (true) {
    for (int b = 0; b < batch && r < TP_MAX_ROUNDS; ++b, ++r) {
      TpEntry *cur = (r % 2 == 0) ? B.fa : B.fb;
      TpEntry *nxt = (r % 2 == 0) ? B.fb : B.fa;
      {
        PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH);
        k_tp_prepass<BWD><<<pre_grid, TP_TPB, 0, ctx->stream>>>(r, cur, K, B.R, B.Q, B.pos_of, rp, nrp, deg, invdw,
                                                                 alpha, B.val, B.items, B.item_cap, B.front_cap,
                                                                 B.cnt);
      }
      PPRVIZ_LAUNCHED(ctx);
      {
        PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH);
        k_tp_push<BWD><<<push_grid, TP_TPB, 0, ctx->stream>>>(r, B.items, cur, B.val, K, B.R, rp, nrp, ncol, nw, deg,
                                                              invdw, r_max, thr_b, nxt, B.front_cap, B.item_cap,
                                                              B.cnt);
      }
      PPRVIZ_LAUNCHED(ctx);
    }
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&head, &B.cnt->front[r], sizeof(head), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (head == 0 || r >= TP_MAX_ROUNDS) break;
    batch = std::min(batch * 2, 64);
  }
  std::vector<unsigned long long> fr((size_t)r + 1);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(fr.data(), B.cnt->front, sizeof(unsigned long long) * fr.size(),
                                   cudaMemcpyDeviceToHost, ctx->stream));
  unsigned long long edges = 0;
  int overflow = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&edges, &B.cnt->edges, sizeof(edges), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&overflow, &B.cnt->overflow, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (overflow) return set_err(ctx, PPRVIZ_E_CUDA, "Tau-Push: a frontier or item queue overflowed its bound");
  int64_t rounds = 0, pushes = 0;
  while (rounds <= r && fr[(size_t)rounds] > 0) pushes += (int64_t)fr[(size_t)rounds++];
  *rounds_out = rounds;
  *pushes_out = pushes;
  *edges_out = (int64_t)edges;
  if (head != 0)
    return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "Tau-Push: residues above the threshold after the round limit");
  return PPRVIZ_OK;
}

}  // namespace

int tau_push_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr_d,
                   const int32_t *leaf_idx_d, const std::vector<int64_t> &leaf_ptr_h, const double *dpr_d,
                   double alpha, double eps, double delta, double tau, void *out_d, bool out64,
                   pprviz_tau_info *info) {
  const int64_t n = g->n;
  const int64_t nleaf = leaf_ptr_h[(size_t)nsup];
  const size_t kk = (size_t)nsup * (size_t)nsup;
  // queue and item bounds: a (node, supernode) pair is listed at most once per
  // round, and the items of a round number at most entries + K nnz / 32
  int64_t pull_nnz = g->nnz;
  if (g->directed) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&pull_nnz, g->prp.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  const int64_t K = nsup;
  const int64_t front_cap = n * K;
  const int64_t item_cap = front_cap + (K * std::max(g->nnz, pull_nnz) + TP_CH - 1) / TP_CH + 1;
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPR, sizeof(double) * (size_t)(n * K)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPQ, sizeof(double) * (size_t)(nleaf * K)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPFA, sizeof(TpEntry) * (size_t)front_cap));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPFB, sizeof(TpEntry) * (size_t)front_cap));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPVAL, sizeof(double) * (size_t)front_cap));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPITEM, sizeof(TpItem) * (size_t)item_cap));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPCNT, sizeof(TpCounters)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPMAP, sizeof(int32_t) * (size_t)(n + nleaf)));
  // table: E (kk doubles), means (2 nsup), thr_b (nsup), slot (nsup int32), tsel (nsup int32)
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPTAB, sizeof(double) * (kk + 3 * (size_t)nsup) + 2 * sizeof(int32_t) * nsup + 64));
  TpBufs B;
  B.R = ctx->ws[WS_TPR].as<double>();
  B.Q = ctx->ws[WS_TPQ].as<double>();
  B.fa = ctx->ws[WS_TPFA].as<TpEntry>();
  B.fb = ctx->ws[WS_TPFB].as<TpEntry>();
  B.val = ctx->ws[WS_TPVAL].as<double>();
  B.items = ctx->ws[WS_TPITEM].as<TpItem>();
  B.cnt = ctx->ws[WS_TPCNT].as<TpCounters>();
  B.pos_of = ctx->ws[WS_TPMAP].as<int32_t>();
  B.psup = B.pos_of + n;
  B.front_cap = front_cap;
  B.item_cap = item_cap;
  double *E = ctx->ws[WS_TPTAB].as<double>();
  double *means = E + kk;
  double *thr_b = means + 2 * (size_t)nsup;
  int32_t *slot = reinterpret_cast<int32_t *>(thr_b + nsup);
  int32_t *tsel = slot + nsup;
  const double *deg = g->deg.as<double>();

  // leaf maps and the per-supernode means
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.pos_of, 0xFF, sizeof(int32_t) * (size_t)n, ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_tp_pos<<<blocks_for(nleaf, TP_TPB), TP_TPB, 0, ctx->stream>>>(nleaf, leaf_idx_d, B.pos_of); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_tp_psup<<<(unsigned)nsup, TP_TPB, 0, ctx->stream>>>(leaf_ptr_d, B.psup); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH); k_tp_means<<<(unsigned)nsup, TP_TPB, 0, ctx->stream>>>(leaf_ptr_d, leaf_idx_d, deg, dpr_d, means); }
  PPRVIZ_LAUNCHED(ctx);
  std::vector<double> mh((size_t)2 * nsup);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(mh.data(), means, sizeof(double) * mh.size(), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));

  // Algorithm 1: thresholds
  if (!(tau > 0.0)) tau = 1.0 / sqrt((double)nsup * (double)n);
  const double r_max = g->m > 0.0 ? eps * delta / (g->m * tau) : INFINITY;
  std::vector<int32_t> slot_h((size_t)nsup, -1), tsel_h;
  std::vector<double> thr_h;
  for (int32_t j = 0; j < nsup; ++j) {
    if (!(mh[2 * (size_t)j + 1] > tau)) continue;
    double dmax = -1.0;
    for (int32_t i = 0; i < nsup; ++i)
      if (i != j) dmax = std::max(dmax, mh[2 * (size_t)i]);
    if (nsup == 1) dmax = mh[0];
    slot_h[(size_t)j] = (int32_t)tsel_h.size();
    tsel_h.push_back(j);
    thr_h.push_back(dmax > 0.0 ? eps * delta / dmax : INFINITY);
  }
  const int32_t Kb = (int32_t)tsel_h.size();
  pprviz_tau_info inf;
  memset(&inf, 0, sizeof(inf));
  inf.tau = tau;
  inf.r_max = r_max;
  inf.backward_targets = Kb;

  // forward phase (GFP from every child)
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.R, 0, sizeof(double) * (size_t)(n * K), ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.Q, 0, sizeof(double) * (size_t)(nleaf * K), ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(TpCounters), ctx->stream));
  if (std::isfinite(r_max)) {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH); k_tp_fwd_init<<<blocks_for(nleaf, TP_TPB), TP_TPB, 0, ctx->stream>>>(nleaf, leaf_ptr_d, leaf_idx_d, B.psup, (int32_t)K, deg, r_max, B.R, B.fa, B.cnt); }
    PPRVIZ_LAUNCHED(ctx);
    int64_t rounds = 0, pushes = 0, edges = 0;
    const int st = tp_phase<false>(ctx, g, B, (int32_t)K, alpha, r_max, nullptr, &rounds, &pushes, &edges);
    inf.fwd_rounds = (int32_t)rounds;
    inf.fwd_pushes = pushes;
    inf.fwd_edges = edges;
    if (st != PPRVIZ_OK) {
      if (info) *info = inf;
      return st;
    }
  }
  {
    PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT);
    k_tp_collect<false><<<dim3((unsigned)nsup, (unsigned)nsup), TP_TPB, 0, ctx->stream>>>(leaf_ptr_d, B.Q, (int32_t)K,
                                                                                       nsup, nullptr, E);
  }
  PPRVIZ_LAUNCHED(ctx);

  // backward phase (GBP towards every target above the DPR threshold)
  if (Kb > 0) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(thr_b, thr_h.data(), sizeof(double) * (size_t)Kb, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(slot, slot_h.data(), sizeof(int32_t) * (size_t)nsup, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(tsel, tsel_h.data(), sizeof(int32_t) * (size_t)Kb, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.R, 0, sizeof(double) * (size_t)(n * Kb), ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.Q, 0, sizeof(double) * (size_t)(nleaf * Kb), ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(TpCounters), ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH); k_tp_bwd_init<<<blocks_for(nleaf, TP_TPB), TP_TPB, 0, ctx->stream>>>(nleaf, leaf_ptr_d, leaf_idx_d, B.psup, slot, Kb, thr_b, B.R, B.fa, B.cnt); }
    PPRVIZ_LAUNCHED(ctx);
    int64_t rounds = 0, pushes = 0, edges = 0;
    const int st = tp_phase<true>(ctx, g, B, Kb, alpha, 0.0, thr_b, &rounds, &pushes, &edges);
    inf.bwd_rounds = (int32_t)rounds;
    inf.bwd_pushes = pushes;
    inf.bwd_edges = edges;
    if (st != PPRVIZ_OK) {
      if (info) *info = inf;
      return st;
    }
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT);
      k_tp_collect<true><<<dim3((unsigned)nsup, (unsigned)Kb), TP_TPB, 0, ctx->stream>>>(leaf_ptr_d, B.Q, Kb, nsup,
                                                                                       tsel, E);
    }
    PPRVIZ_LAUNCHED(ctx);
  }
  if (out64) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(out_d, E, sizeof(double) * kk, cudaMemcpyDeviceToDevice, ctx->stream));
  } else {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_tp_out<float><<<blocks_for((int64_t)kk, TP_TPB), TP_TPB, 0, ctx->stream>>>((int64_t)kk, E, (float *)out_d); }
    PPRVIZ_LAUNCHED(ctx);
  }
  if (info) *info = inf;
  return PPRVIZ_OK;
}

}  // namespace pprviz
