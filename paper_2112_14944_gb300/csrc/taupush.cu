// Tau-Push (Sec. 4, Algorithms 1-3) as synchronous frontier pushes on the
// GPU, and the DPR index it reads (Eq. (dnpr-dnppr), Sec. 4.3).
//
// The paper's pushes are sequential: one node at a time, in no stated order.
// Here every (node, supernode) residue above its threshold is pushed in the
// same round. A round is two launches:
//   collect  one thread per node, dirty nodes only: it takes (sets to 0)
//            every residue of the node above its threshold, books its
//            reserve share and lists the node for the push: its taken
//            residues' (supernode slot, share) pairs, and either one small
//            record (at most TP_SMALL units of work; unit = one edge times
//            one taken residue) or pieces of at most TP_PIECE units; the
//            lists of a warp are placed with one atomic each;
//   push     one warp per task of at most TP_PIECE units: 32 small records
//            (a lane finds its record by a 5-step search over the warp's
//            prefix sums) or one piece; a lane's unit o of a record is its
//            edge o / c and taken residue o % c; TP_CPW units in flight per
//            lane; the share is added with a fire-and-forget FP64 atomic
//            reduction and the neighbour marked dirty.
// One record serves all of a node's taken residues, so an edge's column
// index is read once for all of them and their adds land in the same few
// cache lines of the neighbour. No push reads a residue back, so the adds of
// a round overlap freely; the residues are read only when no push is in
// flight. Every residue above its threshold belongs to a node touched since
// it was last taken, so the rounds end exactly when Algorithm 2's (or 3's)
// loop condition fails, and the error bounds of Lemmas 2 and 3 hold as stated.
//
// Data layout: residues node-major (n x K doubles, K = sources or targets of
// the phase), so the K residues of a node sit in a few cache lines and the
// collect pass reads them together; reserves only for the leaves of the
// children (leaves x K doubles, indexed by the leaf's position in leaf_idx).
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace pprviz {
namespace {

constexpr int TP_TPB = 256;
constexpr int64_t TP_MAX_ROUNDS = 65535;   // a phase still active after this many rounds fails
constexpr int64_t DPR_HEAVY = 512;         // pull rows longer than this get a block of their own

// A listed node: its first edge (out-edges forward, in-edges backward), edge
// count, number of taken residues and where their (slot, share) pairs start.
struct TpRec {
  int64_t q0;
  int64_t pb;
  int32_t v, ne, c, pad;
};
struct TpPair {
  int32_t s, pad;
  double share;  // per unit walk weight
};

// Per-phase device counters, per round: small records, pieces and
// (slot, share) pairs;
// and the residues taken, the edge relaxations listed and an overflow flag.
struct TpCounters {
  unsigned long long small[TP_MAX_ROUNDS + 2];
  unsigned long long big[TP_MAX_ROUNDS + 2];
  unsigned long long pairs[TP_MAX_ROUNDS + 2];
  unsigned long long takes;
  unsigned long long edges;
  int overflow;
};

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
// on the leaves of every source V_i; the leaves are marked for the collect pass.
__global__ void k_tp_fwd_init(int64_t nleaf, const int64_t *__restrict__ leaf_ptr,
                              const int32_t *__restrict__ leaf_idx, const int32_t *__restrict__ psup, int32_t KR,
                              const double *__restrict__ deg, double *__restrict__ R, uint8_t *__restrict__ dirty) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nleaf) return;
  const int32_t i = psup[p], v = leaf_idx[p];
  R[(size_t)v * KR + i] = deg[v] / (double)(leaf_ptr[i + 1] - leaf_ptr[i]);
  dirty[v] = 1;
}

// Backward start (Algorithm 3, initial residues): r(v, V_j) = 1 / |F(V_j)| on
// the leaves of every refined target V_j (slot[j] >= 0).
__global__ void k_tp_bwd_init(int64_t nleaf, const int64_t *__restrict__ leaf_ptr,
                              const int32_t *__restrict__ leaf_idx, const int32_t *__restrict__ psup,
                              const int32_t *__restrict__ slot, int32_t KR, double *__restrict__ R,
                              uint8_t *__restrict__ dirty) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nleaf) return;
  const int32_t j = psup[p], jb = slot[j];
  if (jb < 0) return;
  const int32_t v = leaf_idx[p];
  R[(size_t)v * KR + jb] = 1.0 / (double)(leaf_ptr[j + 1] - leaf_ptr[j]);
  dirty[v] = 1;
}

// One unit of a push: the share sent along edge q lands in the residue
// (slot sl) of neighbour x = ncol[q], which is marked dirty. Forward: weight
// w(v, x) (1 unweighted). Backward: walk probability w(x, v) / dw(x); the
// walk's own self-loop at a node without out-edges was summed when its
// residue was taken. The add is a reduction (no value read back).
template <bool BWD>
__device__ __forceinline__ void push_unit(int64_t q, int32_t v, const TpPair &pr, int32_t KR,
                                          double *__restrict__ R, const int64_t *__restrict__ rp,
                                          const int32_t *__restrict__ ncol, const float *__restrict__ nw,
                                          const double *__restrict__ invdw, uint8_t *__restrict__ dirty) {
  const int32_t x = ncol[q];
  double add = pr.share;  // FP64 arithmetic is scarce on this GPU: no multiply by a unit weight
  if (nw) add *= (double)nw[q];
  if (BWD) {
    if (x == v && rp[v + 1] == rp[v]) return;
    add *= invdw[x];
  }
  if (__double_as_longlong(add) <= 0) return;  // add >= 0: skip the zero weights by the bits
  atomicAdd(&R[(size_t)x * KR + pr.s], add);
  dirty[x] = 1;
}

// Number of the 32 inclusive prefix sums (one per lane) that are <= t
// (32 when t is past the last one).
__device__ __forceinline__ int32_t prefix_count(int32_t incl, int64_t t) {
  int32_t j = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    const int32_t v = __shfl_sync(0xffffffffu, incl, j + step - 1);
    if ((int64_t)v <= t) j += step;
  }
  if (t >= (int64_t)__shfl_sync(0xffffffffu, incl, 31)) j = 32;
  return j;
}

constexpr int TP_CPW = 4;          // units in flight per lane
constexpr int32_t TP_SMALL = 32;    // records of at most this much work are packed 32 to a warp
constexpr int32_t TP_PIECE = 1024;  // larger work is cut into pieces of at most this much, one warp each

// Push of a round. Tasks [0, ceil(S / 32)) take 32 consecutive small records
// each (one unit per lane: a 5-step search over the warp's prefix sums finds
// the record); the next B tasks take one piece each (unit o of the piece:
// edge o / c, residue o % c). Every task is at most TP_PIECE units.
template <bool BWD>
__global__ void __launch_bounds__(TP_TPB, 4)
    k_tp_push(int64_t round, const TpRec *__restrict__ small, const TpRec *__restrict__ big,
              const TpPair *__restrict__ pairs, int32_t KR, double *__restrict__ R, const int64_t *__restrict__ rp,
              const int32_t *__restrict__ ncol, const float *__restrict__ nw, const double *__restrict__ invdw,
              uint8_t *__restrict__ dirty, int64_t small_cap, int64_t big_cap, const TpCounters *__restrict__ cnt) {
  const int64_t S = min((int64_t)cnt->small[round], small_cap);  // beyond the caps only after an overflow
  const int64_t Bn = min((int64_t)cnt->big[round], big_cap);
  const int64_t ntask = (S + 31) / 32 + Bn;
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t task = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; task < ntask; task += nwarps) {
    if (task < (S + 31) / 32) {
      const int64_t e = task * 32 + lane;
      TpRec me{0, 0, 0, 0, 1, 0};
      int32_t work = 0;
      if (e < S) {
        me = small[e];
        work = me.ne * me.c;
      }
      int32_t incl = work;
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t a = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += a;
      }
      const int32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      for (int64_t t0 = 0; t0 < tot; t0 += 32 * TP_CPW) {
#pragma unroll
        for (int u = 0; u < TP_CPW; ++u) {
          const int64_t t = t0 + 32 * u + lane;
          const int32_t j = prefix_count(incl, t);
          const int32_t jj = j < 32 ? j : 31;
          const int32_t prev = __shfl_sync(0xffffffffu, incl, jj > 0 ? jj - 1 : 0);
          const int64_t q0 = __shfl_sync(0xffffffffu, me.q0, jj);
          const int64_t pb = __shfl_sync(0xffffffffu, me.pb, jj);
          const int32_t v = __shfl_sync(0xffffffffu, me.v, jj);
          const int32_t c = __shfl_sync(0xffffffffu, me.c, jj);
          if (j < 32) {
            const int32_t o = (int32_t)(t - (j > 0 ? prev : 0));
            const int32_t ed = o / c;
            push_unit<BWD>(q0 + ed, v, pairs[pb + (o - ed * c)], KR, R, rp, ncol, nw, invdw, dirty);
          }
        }
      }
    } else {
      const TpRec r = big[task - (S + 31) / 32];
      const int32_t work = r.ne * r.c;
      for (int32_t o0 = 0; o0 < work; o0 += 32 * TP_CPW) {
#pragma unroll
        for (int u = 0; u < TP_CPW; ++u) {
          const int32_t o = o0 + 32 * u + lane;
          if (o < work) {
            const int32_t ed = o / r.c;
            push_unit<BWD>(r.q0 + ed, r.v, pairs[r.pb + (o - ed * r.c)], KR, R, rp, ncol, nw, invdw, dirty);
          }
        }
      }
    }
  }
}

// Inclusive warp prefix sum.
template <typename T>
__device__ __forceinline__ T warp_incl(T v, int lane) {
  for (int o = 1; o < 32; o <<= 1) {
    const T a = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += a;
  }
  return v;
}

// r > thr for non-negative doubles (residues and thresholds are >= 0, NaN
// never occurs, INFINITY orders last) by their bit patterns: the ordering of
// non-negative IEEE doubles is that of their bits as integers, and the
// integer compare keeps the comparisons off this GPU's narrow FP64 pipe.
__device__ __forceinline__ bool above(double r, double thr) {
  return __double_as_longlong(r) > __double_as_longlong(thr);
}

// Collect pass (builds round `round`): one thread per node x; a dirty x has
// its mark cleared and each residue above its threshold (forward
// d(x) r_max, backward the target's thr_b) taken. Forward (Algorithm 2): the
// reserve of a leaf gains alpha r (the estimate's alpha r / |F(V_j)| is
// applied when the reserves are summed) and the share is (1 - alpha) r / dw(x).
// Backward (Algorithm 3): the reserve gains alpha d(x) r and the share is
// (1 - alpha) r. A node without out-edges keeps the walk (a self-loop): the
// sum of its endless pushes is taken at once - forward, the whole residue is
// reserve and nothing is listed; backward, the reserve gains d(x) r (= 0) and
// the other in-neighbours receive (1 - alpha) r / alpha times their walk
// probability.
template <bool BWD>
__global__ void __launch_bounds__(TP_TPB)
    k_tp_collect_front(int64_t round, int64_t n, int32_t K, int32_t KR, double *__restrict__ R, double *__restrict__ Q,
                       uint8_t *__restrict__ dirty, const int32_t *__restrict__ pos_of,
                       const int64_t *__restrict__ rp, const int64_t *__restrict__ nrp,
                       const double *__restrict__ deg, const double *__restrict__ invdw, double alpha, double r_max,
                       const double *__restrict__ thr_b, TpRec *__restrict__ small, TpRec *__restrict__ big,
                       TpPair *__restrict__ pairs, int64_t small_cap, int64_t big_cap, int64_t pair_cap,
                       TpCounters *__restrict__ cnt) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t x0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); x0 < n; x0 += stride) {
    const int64_t x = x0 + lane;
    const bool mine = x < n && dirty[x];
    if (!__any_sync(0xffffffffu, mine)) continue;
    int32_t c = 0, ne = 0, p = -1;
    int64_t q0 = 0;
    bool stays = false;
    double thr = 0.0, dx = 0.0;
    double *Rx = R + (size_t)x * KR;  // KR even: 16-byte aligned pairs
    if (mine) {
      dirty[x] = 0;
      stays = rp[x + 1] == rp[x];
      q0 = nrp[x];
      ne = (!BWD && stays) ? 0 : (int32_t)(nrp[x + 1] - q0);
      p = pos_of[x];
      dx = deg[x];
      thr = dx * r_max;
      // how many residues of x are above their thresholds
#pragma unroll 4
      for (int32_t sl = 0; sl < K; sl += 2) {
        const double2 r2 = *reinterpret_cast<const double2 *>(Rx + sl);
        c += above(r2.x, BWD ? thr_b[sl] : thr);
        if (sl + 1 < K) c += above(r2.y, BWD ? thr_b[sl + 1] : thr);
      }
    }
    const bool listed = ne > 0 && c > 0;
    const int64_t work = (int64_t)ne * c;
    const bool is_small = listed && work <= TP_SMALL;
    const int32_t epr = c > 0 ? max(1, TP_PIECE / c) : 1;  // edges per piece
    const int32_t nsm = is_small ? 1 : 0;
    const int32_t npc = (listed && !is_small) ? (ne + epr - 1) / epr : 0;
    // warp placement of the pairs, small records and pieces, one atomic each
    const int32_t pc = listed ? c : 0;
    const int32_t pin = warp_incl(pc, lane), sin_ = warp_incl(nsm, lane), bin = warp_incl(npc, lane);
    const int32_t ptot = __shfl_sync(0xffffffffu, pin, 31), stot = __shfl_sync(0xffffffffu, sin_, 31);
    const int32_t btot = __shfl_sync(0xffffffffu, bin, 31);
    unsigned long long pb0 = 0, sb0 = 0, bb0 = 0;
    if (lane == 31) {
      if (ptot) pb0 = atomicAdd(&cnt->pairs[round], (unsigned long long)ptot);
      if (stot) sb0 = atomicAdd(&cnt->small[round], (unsigned long long)stot);
      if (btot) bb0 = atomicAdd(&cnt->big[round], (unsigned long long)btot);
    }
    pb0 = __shfl_sync(0xffffffffu, pb0, 31);
    sb0 = __shfl_sync(0xffffffffu, sb0, 31);
    bb0 = __shfl_sync(0xffffffffu, bb0, 31);
    const long long tk = warp_incl((long long)c, lane);
    const long long ed = warp_incl(listed ? (long long)ne * c : 0ll, lane);
    if (lane == 31) {
      if (tk) atomicAdd(&cnt->takes, (unsigned long long)tk);
      if (ed) atomicAdd(&cnt->edges, (unsigned long long)ed);
    }
    if (c == 0) continue;
    const int64_t pb = (int64_t)pb0 + pin - pc, sb = (int64_t)sb0 + sin_ - nsm, bb = (int64_t)bb0 + bin - npc;
    const bool fits = pb + pc <= pair_cap && sb + nsm <= small_cap && bb + npc <= big_cap;
    if (!fits) atomicOr(&cnt->overflow, 1);
    double rnext = 0.0;
    int32_t k = 0;
    const double inv = invdw[x];
    for (int32_t sl = 0; sl < K; ++sl) {
      double r;
      if ((sl & 1) == 0) {
        const double2 r2 = *reinterpret_cast<const double2 *>(Rx + sl);
        r = r2.x;
        rnext = r2.y;
      } else {
        r = rnext;
      }
      if (!above(r, BWD ? thr_b[sl] : thr)) continue;
      Rx[sl] = 0.0;
      double share;
      if (!BWD) {
        if (p >= 0) Q[(size_t)p * K + sl] += stays ? r : alpha * r;
        share = (1.0 - alpha) * r * inv;
      } else {
        if (p >= 0) Q[(size_t)p * K + sl] += (stays ? 1.0 : alpha) * dx * r;
        share = stays ? (1.0 - alpha) * r / alpha : (1.0 - alpha) * r;
      }
      if (listed && fits) pairs[pb + k] = TpPair{sl, 0, share};
      ++k;
    }
    if (listed && fits) {
      if (is_small) small[sb] = TpRec{q0, pb, (int32_t)x, ne, c, 0};
      for (int32_t i = 0; i < npc; ++i)
        big[bb + i] = TpRec{q0 + (int64_t)i * epr, pb, (int32_t)x, min(epr, ne - i * epr), c, 0};
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
  double *R, *Q;
  uint8_t *dirty;
  TpRec *small, *big;
  TpPair *pairs;
  TpCounters *cnt;
  int32_t *pos_of, *psup;
  int64_t small_cap, big_cap, pair_cap;
};

// Runs the rounds of one phase (the start residues set and their nodes
// marked) until a collect pass lists nothing. Returns the number of rounds,
// the residues taken and the edges of the listed records.
template <bool BWD>
int tp_phase(pprviz_ctx *ctx, const pprviz_graph *g, const TpBufs &B, int32_t K, double alpha, double r_max,
             const double *thr_b, int64_t *rounds_out, int64_t *takes_out, int64_t *edges_out) {
  const int64_t n = g->n;
  const int64_t *rp = g->rp.as<int64_t>();
  const int64_t *nrp = BWD ? pull_rp(g) : g->rp.as<int64_t>();
  const int32_t *ncol = BWD ? pull_col(g) : g->col.as<int32_t>();
  const float *nw = BWD ? pull_w(g) : (g->weighted ? g->w.as<float>() : nullptr);
  const double *deg = g->deg.as<double>();
  const double *invdw = g->invdw_d.as<double>();
  const int32_t KR = (K + 1) & ~1;  // residue row stride (even)
  const unsigned grid = 152 * 8;
  auto collect = [&](int64_t r) -> int {
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH);
      k_tp_collect_front<BWD><<<grid, TP_TPB, 0, ctx->stream>>>(r, n, K, KR, B.R, B.Q, B.dirty, B.pos_of, rp, nrp, deg,
                                                                invdw, alpha, r_max, thr_b, B.small, B.big, B.pairs,
                                                                B.small_cap, B.big_cap, B.pair_cap, B.cnt);
    }
    PPRVIZ_LAUNCHED(ctx);
    return PPRVIZ_OK;
  };
  PPRVIZ_TRY(collect(0));
  int64_t r = 0;  // rounds pushed so far; round r's lists are built
  int batch = 4;
  unsigned long long head = 0;
  while (true) {
    for (int b = 0; b < batch && r < TP_MAX_ROUNDS; ++b, ++r) {
      {
        PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH);
        k_tp_push<BWD><<<grid, TP_TPB, 0, ctx->stream>>>(r, B.small, B.big, B.pairs, KR, B.R, rp, ncol, nw, invdw,
                                                         B.dirty, B.small_cap, B.big_cap, B.cnt);
      }
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_TRY(collect(r + 1));
    }
    unsigned long long hb = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&head, &B.cnt->small[r], sizeof(head), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hb, &B.cnt->big[r], sizeof(hb), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    head += hb;
    if (head == 0 || r >= TP_MAX_ROUNDS) break;
    batch = std::min(batch * 2, 64);
  }
  std::vector<unsigned long long> rc((size_t)r + 1), rb((size_t)r + 1);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(rc.data(), B.cnt->small, sizeof(unsigned long long) * rc.size(),
                                   cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(rb.data(), B.cnt->big, sizeof(unsigned long long) * rb.size(),
                                   cudaMemcpyDeviceToHost, ctx->stream));
  unsigned long long takes = 0, edges = 0;
  int overflow = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&takes, &B.cnt->takes, sizeof(takes), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&edges, &B.cnt->edges, sizeof(edges), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&overflow, &B.cnt->overflow, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (overflow) return set_err(ctx, PPRVIZ_E_CUDA, "Tau-Push: a record list overflowed its bound");
  int64_t rounds = 0;
  while (rounds <= r && rc[(size_t)rounds] + rb[(size_t)rounds] > 0) ++rounds;
  *rounds_out = rounds;
  *takes_out = (int64_t)takes;
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
  // list bounds: a node is listed at most once per round and a residue at
  // most once (one pair)
  int64_t pull_nnz = g->nnz;
  if (g->directed) {
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&pull_nnz, g->prp.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  const int64_t K = nsup;
  const int64_t nnz_max = std::max(g->nnz, pull_nnz);
  // records: one small record per node, or pieces of at least
  // max(1, TP_PIECE / K) edges each (the last piece of a node may be shorter)
  const int64_t small_cap = n;
  const int64_t big_cap = n + nnz_max / std::max<int64_t>(1, TP_PIECE / K) + 1;
  const int64_t pair_cap = n * K;
  const int64_t KR = (K + 1) & ~(int64_t)1;  // residue row stride: even, so that rows are 16-byte aligned
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPR, sizeof(double) * (size_t)(n * KR)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPQ, sizeof(double) * (size_t)(nleaf * K)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPFA, sizeof(TpRec) * (size_t)(small_cap + big_cap)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPFB, sizeof(TpPair) * (size_t)pair_cap));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPVAL, (size_t)n));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPCNT, sizeof(TpCounters)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPMAP, sizeof(int32_t) * (size_t)(n + nleaf)));
  // table: E (kk doubles), means (2 nsup), thr_b (nsup), slot (nsup int32), tsel (nsup int32)
  PPRVIZ_TRY(ws_ensure(ctx, WS_TPTAB, sizeof(double) * (kk + 3 * (size_t)nsup) + 2 * sizeof(int32_t) * nsup + 64));
  TpBufs B;
  B.R = ctx->ws[WS_TPR].as<double>();
  B.Q = ctx->ws[WS_TPQ].as<double>();
  B.small = ctx->ws[WS_TPFA].as<TpRec>();
  B.big = B.small + small_cap;
  B.pairs = ctx->ws[WS_TPFB].as<TpPair>();
  B.dirty = ctx->ws[WS_TPVAL].as<uint8_t>();
  B.cnt = ctx->ws[WS_TPCNT].as<TpCounters>();
  B.pos_of = ctx->ws[WS_TPMAP].as<int32_t>();
  B.psup = B.pos_of + n;
  B.small_cap = small_cap;
  B.big_cap = big_cap;
  B.pair_cap = pair_cap;
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
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.R, 0, sizeof(double) * (size_t)(n * KR), ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.Q, 0, sizeof(double) * (size_t)(nleaf * K), ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(TpCounters), ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.dirty, 0, (size_t)n, ctx->stream));
  if (std::isfinite(r_max)) {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH); k_tp_fwd_init<<<blocks_for(nleaf, TP_TPB), TP_TPB, 0, ctx->stream>>>(nleaf, leaf_ptr_d, leaf_idx_d, B.psup, (int32_t)KR, deg, B.R, B.dirty); }
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
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.R, 0, sizeof(double) * (size_t)(n * ((Kb + 1) & ~1)), ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.Q, 0, sizeof(double) * (size_t)(nleaf * Kb), ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.cnt, 0, sizeof(TpCounters), ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(B.dirty, 0, (size_t)n, ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PUSH); k_tp_bwd_init<<<blocks_for(nleaf, TP_TPB), TP_TPB, 0, ctx->stream>>>(nleaf, leaf_ptr_d, leaf_idx_d, B.psup, slot, (Kb + 1) & ~1, B.R, B.dirty); }
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
