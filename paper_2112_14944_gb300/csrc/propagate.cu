// P1/P2 - multi-source PPR propagation with an FP64 residual certificate.
//
// What is computed (Sec. 3.1): for every view source s, the PPR row
//   pi(s, .) = alpha * sum_t (1 - alpha)^t e_s P^t,
// i.e. the solution x of x (I - c P) = alpha e_s with c = 1 - alpha, and the
// DPPR pi_d(s, t) = d(s) pi(s, t) (Definition 1).
//
// How (GB300 design, not the paper's sequential push):
//  * Sources are processed in groups of G columns. The state of a group is a
//    node-major [n][G] matrix so that one warp gathers a neighbour's 128
//    (FP32) or 64 (FP64) source values with one 512-byte coalesced load. G is
//    chosen so that the group's live buffers stay resident in the 126 MB L2;
//    each sweep then re-reads the CSR and the gathered rows from L2.
//  * The state is degree-scaled, y_v = x_v / dw(v) (dw = walk degree), so a
//    pull over the symmetric CSR needs no per-edge weight on unit graphs:
//    (x P)_j = sum_{i in N(j)} x_i / dw(i) = sum_{i in N(j)} y_i.
//  * FP64 plain path: power iteration x <- alpha e_s + c x P for the a-priori
//    sweep count T with d(s) c^(T+1) <= eps / 2.
//  * FP32 path: Chebyshev semi-iteration. The walk matrix of an undirected
//    graph is reversible, so the spectrum of I - cP lies in [1 - c, 1 + c]
//    and the three-term Chebyshev recurrence converges with rate
//    rho = (1 - sqrt(1 - c^2)) / c (0.557 at alpha = 0.15, vs 0.85 for the
//    power iteration), needing no inner products.
//  * Deflated start: the coefficient of a row on the stationary vector of its
//    source's component is known exactly (1 for x (I - cP) = alpha e_s, and
//    sum_j r_j / alpha for a correction system with right-hand side r), so
//    every solve starts from that multiple of the stationary vector (uniform
//    in y) and only the remaining modes, with |lambda| <= b (estimated per
//    graph), are iterated: Chebyshev on [1 - cb, 1 + cb], rate
//    (1 - sqrt(1 - (cb)^2)) / (cb), e.g. 0.21 instead of 0.557 at b = 0.48.
//  * The certificate (Eq. (3)): with res = alpha e_s - x (I - cP) computed in
//    FP64, the exact row is x + res Pi / alpha, so every DPPR entry of the row
//    is within d(s) ||res||_1 / alpha. FP32 rows are refined: the FP32
//    correction system delta (I - cP) = res is solved with the same sweeps
//    and kept as a second FP32 array (x = x_hi + x_lo), until the FP64
//    certificate is at most eps.
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <cstring>

#include "common.cuh"

namespace pprviz {

constexpr int kWarps = 8;         // warps per block in the residual kernels
constexpr int kSweepWarps = 1;    // warps per block in k_sweep: one-warp blocks retire with their own
                                  // row, so a hub row does not hold seven finished warps' slots
constexpr int kChunk = 128;       // group width granule (sources)
constexpr int kMaxRefine = 6;     // refinement passes before E_NOT_CONVERGED
constexpr int kMaxRefineBf16 = 16;  // the same with BF16 tensor-core sweeps
constexpr int kMaxRefineSweeps = 32;  // Chebyshev sweeps per refinement pass

template <typename T>
struct Vec;  // 16-byte vector of T
template <>
struct Vec<float> {
  static constexpr int N = 4;
  using V = float4;
  __device__ static void load(const float *p, float (&v)[4]) {
    float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ static void store(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct Vec<double> {
  static constexpr int N = 2;
  __device__ static void load(const double *p, double (&v)[2]) {
    double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = t.x; v[1] = t.y;
  }
  __device__ static void store(double *p, const double (&v)[2]) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  }
};

// y[v_q][q] = alpha / dw(v_q) (the first iterate x_1 = alpha e_s, y-scaled);
// all other entries are zeroed beforehand by a memset.
template <typename T>
__global__ void k_init_delta(int32_t gcount, const int32_t *__restrict__ src, int64_t ld,
                             const T *__restrict__ invdw, T alpha, T *__restrict__ y) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= gcount) return;
  int32_t s = src[q];
  if (s >= 0) y[(int64_t)s * ld + q] = alpha * invdw[s];
}

// y = rhs / dw (the first iterate of the correction system, x_1 = rhs).
__global__ void k_init_rhs(int64_t n, int64_t ld, const float *__restrict__ rhs,
                           const float *__restrict__ invdw, float *__restrict__ y) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ld) return;
  y[idx] = rhs[idx] * invdw[idx / ld];
}

// Deflated start of a solve for the sources of a group: on the component of
// source q (root csrc[q], -1 for a padded column) y_0 = kappa[q], the
// coefficient on the stationary vector (uniform in y); y_1 = c y_0 + b / dw,
// the first Chebyshev step from y_0 (P fixes the stationary vector), with
// b = alpha e_s, or the rhs of a correction system.
__global__ void k_init_defl(int64_t n, int64_t ld, const int32_t *__restrict__ comp,
                            const int32_t *__restrict__ csrc, const double *__restrict__ kappa,
                            const int32_t *__restrict__ src, const float *__restrict__ rhs,
                            const float *__restrict__ invdw, float alpha, float c, float *__restrict__ y0,
                            float *__restrict__ y1) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ld) return;
  const int64_t j = idx / ld, q = idx - j * ld;
  const int32_t cs = csrc[q];
  const float v0 = (cs >= 0 && comp[j] == cs) ? (float)kappa[q] : 0.0f;
  const float b = rhs ? rhs[idx] : ((src[q] == (int32_t)j) ? alpha : 0.0f);
  y0[idx] = v0;
  y1[idx] = c * v0 + b * invdw[j];
}

__global__ void k_axpy(int64_t count, const float *__restrict__ x, float *__restrict__ y) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx < count) y[idx] += x[idx];
}

// Exact renormalisation of the two-float state: hi + lo is replaced by
// s = fl(hi + lo) and the exact remainder lo - (s - hi) (Fast2Sum, Dekker
// 1971; |hi| >= |lo| holds since lo is a correction of hi). Afterwards
// |lo| <= ulp(hi) / 2, so later corrections keep ~48 significant bits.
__global__ void k_renorm(int64_t count, float *__restrict__ hi, float *__restrict__ lo) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count) return;
  const float h = hi[idx], l = lo[idx];
  const float s = h + l;
  hi[idx] = s;
  lo[idx] = l - (s - h);
}

// One sweep for the rows of a group.  For each node j and source column q:
//   acc  = sum_{i in N(j)} w_ij y_cur[i][q]   (+ y_cur[j][q] if j has no edges)
//   xnew = (b_jq + c * acc) / dw(j)           (y-scaled next iterate)
//   CHEB: y_out = om1 * y_old + om * xnew     (three-term recurrence, in place over y_old)
//   else: y_out = xnew                         (power iteration)
// b_jq = alpha [j == src[q]] unless RHS, then b_jq = rhs[j][q].
// One warp per (row j, 32*VEC-source chunk); lanes own VEC consecutive sources.
// Batched views (BATCH): the graph is the disjoint union of the views and the
// state covers its rows [row0, row0 + n); column q is, for every row, the
// source g0 + q of that row's own view, and src holds each node's index within
// its view, so b_jq = alpha [src[row0 + j] == g0 + q]. Neighbours stay inside
// their view, hence inside the state's row range.
template <typename T, bool WEIGHTED, bool CHEB, bool RHS, bool BATCH>
__global__ void __launch_bounds__(kSweepWarps * 32)
k_sweep(int64_t n, int64_t ld, int nchunks, const int64_t *__restrict__ rp,
        const int32_t *__restrict__ col, const float *__restrict__ w, const T *__restrict__ invdw,
        const int32_t *__restrict__ src, const float *__restrict__ rhs, const T *__restrict__ ycur,
        const T *yold, T *yout, T alpha, T c, T om, T om1, int64_t row0, int32_t g0) {
  constexpr int VEC = Vec<T>::N;
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * kSweepWarps + (threadIdx.x >> 5);
  if (item >= n * nchunks) return;
  const int64_t chunk = item / n;
  const int64_t j = item - chunk * n;  // row within the state
  const int64_t jg = j + row0;         // row of the graph
  const int64_t off = chunk * (32 * VEC) + lane * VEC;
  const int64_t rb = BATCH ? row0 : 0;  // state row of graph node i: i - rb
  T acc[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) acc[u] = T(0);
  const int64_t b = rp[jg], e = rp[jg + 1];
  for (int64_t base = b; base < e; base += 32) {
    const int cnt = (int)min((int64_t)32, e - base);
    int32_t myc = lane < cnt ? col[base + lane] : 0;
    float myw = 1.0f;
    if (WEIGHTED) myw = lane < cnt ? w[base + lane] : 0.0f;
    int t = 0;
    for (; t + 8 <= cnt; t += 8) {
      T v[8][VEC];
      float wv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int32_t iq = __shfl_sync(0xffffffffu, myc, t + q);
        if (WEIGHTED) wv[q] = __shfl_sync(0xffffffffu, myw, t + q);
        Vec<T>::load(ycur + ((int64_t)iq - rb) * ld + off, v[q]);
      }
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        if (WEIGHTED) {
          T s = T(0);
#pragma unroll
          for (int q = 0; q < 8; ++q) s += (T)wv[q] * v[q][u];
          acc[u] += s;
        } else {
          acc[u] += ((v[0][u] + v[1][u]) + (v[2][u] + v[3][u])) + ((v[4][u] + v[5][u]) + (v[6][u] + v[7][u]));
        }
      }
    }
    for (; t + 4 <= cnt; t += 4) {
      T v0[VEC], v1[VEC], v2[VEC], v3[VEC];
      const int32_t i0 = __shfl_sync(0xffffffffu, myc, t);
      const int32_t i1 = __shfl_sync(0xffffffffu, myc, t + 1);
      const int32_t i2 = __shfl_sync(0xffffffffu, myc, t + 2);
      const int32_t i3 = __shfl_sync(0xffffffffu, myc, t + 3);
      Vec<T>::load(ycur + ((int64_t)i0 - rb) * ld + off, v0);
      Vec<T>::load(ycur + ((int64_t)i1 - rb) * ld + off, v1);
      Vec<T>::load(ycur + ((int64_t)i2 - rb) * ld + off, v2);
      Vec<T>::load(ycur + ((int64_t)i3 - rb) * ld + off, v3);
      if (WEIGHTED) {
        const T w0 = (T)__shfl_sync(0xffffffffu, myw, t);
        const T w1 = (T)__shfl_sync(0xffffffffu, myw, t + 1);
        const T w2 = (T)__shfl_sync(0xffffffffu, myw, t + 2);
        const T w3 = (T)__shfl_sync(0xffffffffu, myw, t + 3);
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u] += w0 * v0[u] + w1 * v1[u] + w2 * v2[u] + w3 * v3[u];
      } else {
#pragma unroll
        for (int u = 0; u < VEC; ++u) acc[u] += (v0[u] + v1[u]) + (v2[u] + v3[u]);
      }
    }
    for (; t < cnt; ++t) {
      T v0[VEC];
      const int32_t i0 = __shfl_sync(0xffffffffu, myc, t);
      Vec<T>::load(ycur + ((int64_t)i0 - rb) * ld + off, v0);
      const T w0 = WEIGHTED ? (T)__shfl_sync(0xffffffffu, myw, t) : T(1);
#pragma unroll
      for (int u = 0; u < VEC; ++u) acc[u] += w0 * v0[u];
    }
  }
  const int64_t rowoff = j * ld + off;
  if (e == b) {  // no edges: the walk stays on j (self-loop of weight 1)
    T v0[VEC];
    Vec<T>::load(ycur + rowoff, v0);
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[u] += v0[u];
  }
  const T invd = invdw[jg];
  T bq[VEC];
  if (RHS) {
#pragma unroll
    for (int u = 0; u < VEC; ++u) bq[u] = (T)rhs[rowoff + u];
  } else if (BATCH) {
    const int32_t lj = src[jg] - g0 - (int32_t)off;
#pragma unroll
    for (int u = 0; u < VEC; ++u) bq[u] = (lj == u) ? alpha : T(0);
  } else {
#pragma unroll
    for (int u = 0; u < VEC; ++u) bq[u] = (src[off + u] == (int32_t)jg) ? alpha : T(0);
  }
  T out[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) out[u] = (bq[u] + c * acc[u]) * invd;
  if (CHEB) {
    T old[VEC];
    Vec<T>::load(yold + rowoff, old);
#pragma unroll
    for (int u = 0; u < VEC; ++u) out[u] = om1 * old[u] + om * out[u];
  }
  Vec<T>::store(yout + rowoff, out);
}

// The FP32 Chebyshev sweep with heavy rows split (same result up to the
// order of the additions). One warp per (work item, 128-source chunk); a
// work item is a whole row, or a segment of at most kSegEdges edges of a row
// with more. A row's work then ends within a few round trips to L2 however
// high its degree (in one piece, a degree-477 hub of the power-law graphs
// is a chain of ~60 dependent gather rounds, as long as the whole sweep).
// A segment writes its partial neighbour sum to its slot; the warp that
// arrives last at the row (per-row, per-chunk counter) adds the row's slots
// in slot order, so the result does not depend on the arrival order, applies
// the update and resets the counter for the next sweep.
// items[t] = {row, first edge within the row, edge count, split row or -1};
// srow[s] = {first slot, segments} of split row s.
constexpr int kSegEdges = 64;

// BATCH: a wave of views (see k_sweep): item rows are union-graph rows, the
// state covers rows [row0, row0 + nrows) and column q is source g0 + q of
// every row's view (src = each node's index within its view).
template <bool WEIGHTED, bool RHS, bool BATCH>
__global__ void __launch_bounds__(32)
k_sweep_sp(int64_t nitems, int64_t ld, int nchunks, const int4 *__restrict__ items, const int2 *__restrict__ srow,
           const int64_t *__restrict__ rp, const int32_t *__restrict__ col, const float *__restrict__ w,
           const float *__restrict__ invdw, const int32_t *__restrict__ src, const float *__restrict__ rhs,
           const float *__restrict__ ycur, const float *yold, float *yout, float alpha, float c, float om, float om1,
           float *__restrict__ part, int *__restrict__ cnt, int64_t row0, int32_t g0) {
  const int lane = threadIdx.x & 31;
  const int64_t gid = blockIdx.x;
  if (gid >= nitems * nchunks) return;
  const int64_t chunk = gid / nitems;
  const int4 it = items[gid - chunk * nitems];
  const int64_t jg = it.x;                  // row of the graph
  const int64_t rb = BATCH ? row0 : 0;      // state row of graph node i: i - rb
  const int64_t j = jg - rb;                // row of the state
  const int64_t off = chunk * 128 + lane * 4;
  float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  const int64_t b = rp[jg] + it.y, e = b + it.z;
  for (int64_t base = b; base < e; base += 32) {
    const int cnt_e = (int)min((int64_t)32, e - base);
    const int32_t myc = lane < cnt_e ? col[base + lane] : 0;
    float myw = 1.0f;
    if (WEIGHTED) myw = lane < cnt_e ? w[base + lane] : 0.0f;
    int t = 0;
    for (; t + 8 <= cnt_e; t += 8) {
      float v[8][4], wv[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int32_t iq = __shfl_sync(0xffffffffu, myc, t + q);
        if (WEIGHTED) wv[q] = __shfl_sync(0xffffffffu, myw, t + q);
        Vec<float>::load(ycur + ((int64_t)iq - rb) * ld + off, v[q]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (WEIGHTED) {
          float s2 = 0.0f;
#pragma unroll
          for (int q = 0; q < 8; ++q) s2 += wv[q] * v[q][u];
          acc[u] += s2;
        } else {
          acc[u] += ((v[0][u] + v[1][u]) + (v[2][u] + v[3][u])) + ((v[4][u] + v[5][u]) + (v[6][u] + v[7][u]));
        }
      }
    }
    for (; t < cnt_e; ++t) {
      float v0[4];
      const int32_t i0 = __shfl_sync(0xffffffffu, myc, t);
      Vec<float>::load(ycur + ((int64_t)i0 - rb) * ld + off, v0);
      const float w0 = WEIGHTED ? __shfl_sync(0xffffffffu, myw, t) : 1.0f;
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += w0 * v0[u];
    }
  }
  if (it.w >= 0) {
    const int2 s = srow[it.w];
    float *mine = part + (int64_t)(s.x + it.y / kSegEdges) * ld + off;
    Vec<float>::store(mine, acc);
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(&cnt[(int64_t)it.w * nchunks + chunk], 1) == s.y - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = 0.0f;
    for (int k2 = 0; k2 < s.y; ++k2) {
      const float4 p4 = __ldcg(reinterpret_cast<const float4 *>(part + (int64_t)(s.x + k2) * ld + off));
      acc[0] += p4.x; acc[1] += p4.y; acc[2] += p4.z; acc[3] += p4.w;
    }
    if (lane == 0) cnt[(int64_t)it.w * nchunks + chunk] = 0;
  }
  const int64_t rowoff = j * ld + off;
  if (it.z == 0) {  // no edges: the walk stays on j (self-loop of weight 1)
    float v0[4];
    Vec<float>::load(ycur + rowoff, v0);
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += v0[u];
  }
  const float invd = invdw[jg];
  float bq[4];
  if (RHS) {
#pragma unroll
    for (int u = 0; u < 4; ++u) bq[u] = rhs[rowoff + u];
  } else if (BATCH) {
    const int32_t lj = src[jg] - g0 - (int32_t)off;
#pragma unroll
    for (int u = 0; u < 4; ++u) bq[u] = (lj == u) ? alpha : 0.0f;
  } else {
#pragma unroll
    for (int u = 0; u < 4; ++u) bq[u] = (src[off + u] == (int32_t)jg) ? alpha : 0.0f;
  }
  float old[4], out[4];
  Vec<float>::load(yold + rowoff, old);
#pragma unroll
  for (int u = 0; u < 4; ++u) out[u] = om1 * old[u] + om * ((bq[u] + c * acc[u]) * invd);
  Vec<float>::store(yout + rowoff, out);
}

// v[u] = (double)(y_hi[u] + y_lo[u]), u < 4, with 16-byte loads (p is 4-aligned).
__device__ __forceinline__ void load4(const float *hi, const float *lo, double (&v)[4]) {
  float a[4];
  Vec<float>::load(hi, a);
#pragma unroll
  for (int u = 0; u < 4; ++u) v[u] = (double)a[u];
  if (lo) {
    float b[4];
    Vec<float>::load(lo, b);
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] += (double)b[u];
  }
}
__device__ __forceinline__ void load4(const double *hi, const float *lo, double (&v)[4]) {
  double a[2], b[2];
  Vec<double>::load(hi, a);
  Vec<double>::load(hi + 2, b);
  v[0] = a[0]; v[1] = a[1]; v[2] = b[0]; v[3] = b[1];
  (void)lo;  // the FP64 path keeps no low part
}

// FP64 residual of the computed rows x = dw * (y_hi + y_lo) against the
// original system x (I - cP) = alpha e_s:
//   res_jq = alpha [j == src[q]] - x_jq + c * sum_{i in N(j)} w_ij (y_hi + y_lo)[i][q]
// written (rounded to FP32) into rhs_out for the refinement; the block's
// sums of |res_jq| and res_jq per source go to part[blockIdx.x][0 / 1][q]
// (FP64), which k_res_reduce sums in a fixed order.
// Grid: (row blocks, nchunks), row blocks fastest, so that the 128-source
// chunks are processed roughly one after another and the state columns being
// gathered stay resident in L2 even when the whole group does not fit; each
// warp walks rows with a stride so its per-source partial sums are reduced
// once per block.
// Batched views (BATCH, see k_sweep): block b covers the state rows
// brows[b] = [x, y), all of one view, so its partial sums belong to that view;
// graph node i is state row i - row0 and the source test is src[i] == g0 + q.
// Level-l DPPR (LEVEL): column q is the group start of supernode g0 + q
// (Sec. 3.2, Eq. (2)): b_jq = alpha d(j) / |F(V_q)| for the leaves j of V_q,
// given per node by src[j] = its supernode (-1 for none) and bscale[j] =
// d(j) / |F(V_src[j])| in FP64, so the residual is exact for that b.
template <typename T, bool WEIGHTED, bool EXACT, bool BATCH, bool LEVEL, bool LO = true>
__global__ void __launch_bounds__(kWarps * 32)
k_residual(int64_t n, int64_t ld, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
           const float *__restrict__ w, const double *__restrict__ invdw, const float2 *__restrict__ dwff,
           const int32_t *__restrict__ src, const T *__restrict__ yhi, const float *__restrict__ ylo,
           float *__restrict__ rhs_out, double *__restrict__ part_out, double alpha, double c,
           const int2 *__restrict__ brows, int64_t row0, int32_t g0, const double *__restrict__ bscale) {
  constexpr int VEC = 4;  // 128 sources per warp chunk for both state types
  __shared__ double red[kWarps][32 * VEC];
  __shared__ double reds[kWarps][32 * VEC];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int64_t chunk = blockIdx.y;
  const int64_t off = chunk * (32 * VEC) + lane * VEC;
  int32_t sq[VEC];
#pragma unroll
  for (int u = 0; u < VEC; ++u) sq[u] = (BATCH || LEVEL) ? 0 : src[off + u];
  const int64_t rb = BATCH ? row0 : 0;  // state row of graph node i: i - rb
  // alpha and c as float-float pairs (float-float residual of the FP32 path)
  const float alh = (float)alpha, all = (float)(alpha - (double)alh);
  const float ch = (float)c, cl = (float)(c - (double)ch);
  double part[VEC], psig[VEC];
  float fpart[VEC], fpsig[VEC];  // the float-float path's per-lane sums
#pragma unroll
  for (int u = 0; u < VEC; ++u) {
    part[u] = psig[u] = 0.0;
    fpart[u] = fpsig[u] = 0.0f;
  }
  int64_t jfirst, jend, stride;
  if (BATCH) {
    const int2 br = brows[blockIdx.x];
    jfirst = br.x + warp;
    jend = br.y;
    stride = kWarps;
  } else {
    jfirst = (int64_t)blockIdx.x * kWarps + warp;
    jend = n;
    stride = (int64_t)gridDim.x * kWarps;
  }
  for (int64_t j = jfirst; j < jend; j += stride) {
    const int64_t jg = j + row0;  // row of the graph
    if (BATCH || LEVEL) {
      const int32_t lj = src[jg] - g0 - (int32_t)off;
#pragma unroll
      for (int u = 0; u < VEC; ++u) sq[u] = (lj == u) ? (int32_t)jg : -1;
    }
    const double bval = LEVEL ? alpha * bscale[jg] : alpha;  // b_jq where q is j's column
    double acc[VEC];
#pragma unroll
    for (int u = 0; u < VEC; ++u) acc[u] = 0.0;
    const int64_t b = rp[jg], e = rp[jg + 1];
    if constexpr (std::is_same<T, float>::value && !EXACT) {
      // Error-free FP32 accumulation of sum_i w_ij (y_hi + y_lo)_i: TwoSum
      // (Knuth) keeps the exact rounding error of every addition of the high
      // parts, FMA the exact error of every weighted product; the
      // compensation is flushed into a float-float accumulator (ah, al) after
      // every 32 edges. The residual is then formed in float-float arithmetic
      // (TwoProd by FMA, TwoSum), ~2^-48 relative to the row: GB300's FP64
      // rate is too low to spend FP64 operations per (node, source).
      float shi[VEC], sc[VEC], slo[VEC], ah[VEC], al[VEC];
#pragma unroll
      for (int u = 0; u < VEC; ++u) shi[u] = sc[u] = slo[u] = ah[u] = al[u] = 0.0f;
      for (int64_t base = b; base < e; base += 32) {
        const int cnt = (int)min((int64_t)32, e - base);
        int32_t myc = lane < cnt ? col[base + lane] : 0;
        float myw = 1.0f;
        if (WEIGHTED) myw = lane < cnt ? w[base + lane] : 0.0f;
        // GB neighbour rows in flight, then accumulated in edge order
        constexpr int GB = WEIGHTED ? 4 : 8;
        for (int t0 = 0; t0 < cnt; t0 += GB) {
          float h[GB][VEC], l[GB][VEC], wv[GB];
#pragma unroll
          for (int q = 0; q < GB; ++q) {
            const int32_t i = __shfl_sync(0xffffffffu, myc, (t0 + q) & 31);
            wv[q] = WEIGHTED ? __shfl_sync(0xffffffffu, myw, (t0 + q) & 31) : 1.0f;
            if (t0 + q < cnt) {
              const int64_t p = ((int64_t)i - rb) * ld + off;
              Vec<float>::load(reinterpret_cast<const float *>(yhi) + p, h[q]);
              if (LO && ylo) Vec<float>::load(ylo + p, l[q]);
            }
          }
#pragma unroll
          for (int q = 0; q < GB; ++q) {
            if (t0 + q >= cnt) break;
            const float wi = wv[q];
#pragma unroll
            for (int u = 0; u < VEC; ++u) {
              float a = h[q][u], pe = 0.0f;
              if (WEIGHTED) {
                a = wi * h[q][u];
                pe = fmaf(wi, h[q][u], -a);
              }
              const float s = shi[u] + a;
              const float bb = s - shi[u];
              sc[u] += ((shi[u] - (s - bb)) + (a - bb)) + pe;
              shi[u] = s;
              if (LO && ylo) slo[u] = fmaf(wi, l[q][u], slo[u]);
            }
          }
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u) {
          const float t = ah[u] + sc[u];
          const float bb = t - ah[u];
          al[u] += (ah[u] - (t - bb)) + (sc[u] - bb);
          ah[u] = t;
          sc[u] = 0.0f;
        }
      }
      const int64_t rowoff = j * ld + off;
      const float2 dwp = dwff[jg];
      const float dwh = dwp.x, dwl = dwp.y;
      float hrow[VEC], lrow[VEC];
      Vec<float>::load(reinterpret_cast<const float *>(yhi) + rowoff, hrow);
      if (LO && ylo) Vec<float>::load(ylo + rowoff, lrow);
#pragma unroll
      for (int u = 0; u < VEC; ++u) {
        if (!(LO && ylo)) lrow[u] = 0.0f;
        // S = shi + ah + al + slo (the neighbour sum), as float-float
        float Sh = shi[u] + ah[u];
        const float bb = Sh - shi[u];
        float Sl = ((shi[u] - (Sh - bb)) + (ah[u] - bb)) + (al[u] + slo[u]);
        if (e == b) {  // no edges: the walk stays on j
          Sh = hrow[u];
          Sl = lrow[u];
        }
        // X = dw y and C = c S as unevaluated sums (TwoProd by FMA)
        const float p1 = dwh * hrow[u];
        const float t1 = fmaf(dwh, lrow[u], fmaf(dwl, hrow[u], fmaf(dwh, hrow[u], -p1)));
        const float p2 = ch * Sh;
        const float t2 = fmaf(ch, Sl, fmaf(cl, Sh, fmaf(ch, Sh, -p2)));
        // r = b - X + C with the large terms combined by TwoSum
        const float s1 = p2 - p1;
        const float b1 = s1 - p2;
        const float e1 = (p2 - (s1 - b1)) + (-p1 - b1);
        const bool src_here = sq[u] == (int32_t)jg;
        float bh = src_here ? alh : 0.0f, bl = src_here ? all : 0.0f;
        if (LEVEL) {
          const float bvh = (float)bval;
          bh = src_here ? bvh : 0.0f;
          bl = src_here ? (float)(bval - (double)bvh) : 0.0f;
        }
        const float s2 = s1 + bh;
        const float b2 = s2 - s1;
        const float e2 = (s1 - (s2 - b2)) + (bh - b2);
        const float r = s2 + (((e1 + e2) + (t2 - t1)) + bl);
        if (rhs_out) rhs_out[rowoff + u] = r;
        fpart[u] += fabsf(r);
        fpsig[u] += r;
      }
      continue;
    } else {
      for (int64_t base = b; base < e; base += 32) {
        const int cnt = (int)min((int64_t)32, e - base);
        int32_t myc = lane < cnt ? col[base + lane] : 0;
        float myw = 1.0f;
        if (WEIGHTED) myw = lane < cnt ? w[base + lane] : 0.0f;
        // 4 neighbour rows in flight, then accumulated in edge order
        for (int t0 = 0; t0 < cnt; t0 += 4) {
          double v[4][VEC], wv[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int32_t i = __shfl_sync(0xffffffffu, myc, (t0 + q) & 31);
            wv[q] = WEIGHTED ? (double)__shfl_sync(0xffffffffu, myw, (t0 + q) & 31) : 1.0;
            if (t0 + q < cnt) {
              const int64_t p = ((int64_t)i - rb) * ld + off;
              load4(yhi + p, ylo ? ylo + p : nullptr, v[q]);
            }
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (t0 + q >= cnt) break;
#pragma unroll
            for (int u = 0; u < VEC; ++u) acc[u] += wv[q] * v[q][u];
          }
        }
      }
    }
    const int64_t rowoff = j * ld + off;
    const double dw = 1.0 / invdw[jg];
    double yrow[VEC];
    load4(yhi + rowoff, ylo ? ylo + rowoff : nullptr, yrow);
#pragma unroll
    for (int u = 0; u < VEC; ++u) {
      const double y = yrow[u];
      if (e == b) acc[u] += y;
      const double bq = (sq[u] == (int32_t)jg) ? bval : 0.0;
      const double r = bq - dw * y + c * acc[u];
      if (rhs_out) rhs_out[rowoff + u] = (float)r;
      part[u] += fabs(r);
      psig[u] += r;
    }
  }
#pragma unroll
  for (int u = 0; u < VEC; ++u) {
    red[warp][lane * VEC + u] = part[u] + (double)fpart[u];
    reds[warp][lane * VEC + u] = psig[u] + (double)fpsig[u];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 32 * VEC; t += blockDim.x) {
    double s = 0.0, ss = 0.0;
#pragma unroll
    for (int wv = 0; wv < kWarps; ++wv) {
      s += red[wv][t];
      ss += reds[wv][t];
    }
    part_out[((int64_t)blockIdx.x * 2 + 0) * ld + chunk * (32 * VEC) + t] = s;
    part_out[((int64_t)blockIdx.x * 2 + 1) * ld + chunk * (32 * VEC) + t] = ss;
  }
}

// l1[q] = sum_b part[b][0][q], sig[q] = sum_b part[b][1][q] in a fixed order:
// one warp per source, lane l sums blocks l, l + 32, ... in turn, then a
// fixed butterfly over the lanes.
__global__ void k_res_reduce(int64_t ld, int nblocks, const double *__restrict__ part, double *__restrict__ l1,
                             double *__restrict__ sig) {
  const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (q >= ld) return;
  double s = 0.0, ss = 0.0;
  for (int b = lane; b < nblocks; b += 32) {
    s += part[((int64_t)b * 2 + 0) * ld + q];
    ss += part[((int64_t)b * 2 + 1) * ld + q];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) {
    l1[q] = s;
    sig[q] = ss;
  }
}

// Batched views: out[w][0][q] = sum over the blocks b of view w (bptr[w] <=
// b < bptr[w + 1]) of part[b][0][q], out[w][1][q] likewise, in the fixed
// order of k_res_reduce. One warp per (view, source).
__global__ void k_res_reduce_batch(int64_t ld, int nviews, const int *__restrict__ bptr,
                                   const double *__restrict__ part, double *__restrict__ out) {
  const int64_t wq = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wq >= (int64_t)nviews * ld) return;
  const int64_t v = wq / ld, q = wq - v * ld;
  double s = 0.0, ss = 0.0;
  for (int b = bptr[v] + lane; b < bptr[v + 1]; b += 32) {
    s += part[((int64_t)b * 2 + 0) * ld + q];
    ss += part[((int64_t)b * 2 + 1) * ld + q];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    ss += __shfl_xor_sync(0xffffffffu, ss, o);
  }
  if (lane == 0) {
    out[(v * 2 + 0) * ld + q] = s;
    out[(v * 2 + 1) * ld + q] = ss;
  }
}

// Batched views: the deflated start of k_init_defl for a wave. The source of
// column q for state row j (graph node jg = row0 + j) is node
// s = jg - lidx[jg] + g0 + q of the same view when g0 + q < nv[jg] (nv: the
// size of the node's view); kap[s] is that source's stationary coefficient
// (NULL: no deflation, y_0 = 0).
__global__ void k_init_defl_batch(int64_t nrows, int64_t ld, int64_t row0, int32_t g0, const int32_t *__restrict__ lidx,
                                  const int32_t *__restrict__ nv, const int32_t *__restrict__ comp,
                                  const double *__restrict__ kap, const float *__restrict__ rhs,
                                  const float *__restrict__ invdw, float alpha, float c, float *__restrict__ y0,
                                  float *__restrict__ y1) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nrows * ld) return;
  const int64_t j = idx / ld, q = idx - j * ld;
  const int64_t jg = row0 + j;
  const int32_t lj = lidx[jg];
  const int64_t colq = (int64_t)g0 + q;
  float v0 = 0.0f;
  if (kap && colq < nv[jg]) {
    const int64_t s = jg - lj + colq;
    if (comp[jg] == comp[s]) v0 = (float)kap[s];
  }
  const float b = rhs ? rhs[idx] : ((colq == lj) ? alpha : 0.0f);
  y0[idx] = v0;
  y1[idx] = c * v0 + b * invdw[jg];
}

// out[(g0 + q) * k + r] = d(view[g0+q]) * dw(view[r]) * (y_hi + y_lo)[view[r]][q]
// for q < gvalid, r < k: DPPR rows of the group, transposed through shared
// memory so that both the state reads and the output writes are coalesced.
// FP32 state: the products in float-float arithmetic (TwoProd by FMA) with dw
// as its float pair, ~2^-46 relative: GB300's FP64 rate is too low to spend a
// division per entry. FP64 state: FP64 arithmetic.
template <typename T, typename TO>
__global__ void k_extract(int32_t k, int32_t g0, int32_t gvalid, int64_t ld,
                          const int32_t *__restrict__ view, const double *__restrict__ deg,
                          const double *__restrict__ invdw, const float2 *__restrict__ dwff,
                          const T *__restrict__ yhi, const float *__restrict__ ylo, TO *__restrict__ out) {
  const int q0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  if constexpr (std::is_same<T, float>::value) {
    __shared__ float2 tile[32][33];
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr, q = q0 + tx;
      float2 v = make_float2(0.0f, 0.0f);
      if (r < k && q < gvalid) {
        const int32_t t = view[r];
        const int64_t p = (int64_t)t * ld + q;
        const float yh = yhi[p], yl = ylo ? ylo[p] : 0.0f;
        const float2 dw = dwff[t];
        const float ph = yh * dw.x;
        v = make_float2(ph, fmaf(yh, dw.x, -ph) + fmaf(yh, dw.y, yl * dw.x));
      }
      tile[rr][tx] = v;
    }
    __syncthreads();
    for (int qq = ty; qq < 32; qq += 8) {
      const int q = q0 + qq, r = r0 + tx;
      if (q < gvalid && r < k) {
        const double ds = deg[view[g0 + q]];
        const float sh = (float)ds, sl = (float)(ds - (double)sh);
        const float2 v = tile[tx][qq];
        const float oh = sh * v.x;
        const float ol = fmaf(sh, v.x, -oh) + fmaf(sh, v.y, sl * v.x);
        if constexpr (std::is_same<TO, float>::value) out[(int64_t)(g0 + q) * k + r] = oh + ol;
        else out[(int64_t)(g0 + q) * k + r] = (double)oh + (double)ol;
      }
    }
  } else {
    __shared__ double tile[32][33];
    for (int rr = ty; rr < 32; rr += 8) {
      const int r = r0 + rr, q = q0 + tx;
      double v = 0.0;
      if (r < k && q < gvalid) {
        const int32_t t = view[r];
        const int64_t p = (int64_t)t * ld + q;
        double y = (double)yhi[p];
        if (ylo) y += (double)ylo[p];
        v = y / invdw[t];
      }
      tile[rr][tx] = v;
    }
    __syncthreads();
    for (int qq = ty; qq < 32; qq += 8) {
      const int q = q0 + qq, r = r0 + tx;
      if (q < gvalid && r < k) {
        const double ds = deg[view[g0 + q]];
        out[(int64_t)(g0 + q) * k + r] = (TO)(ds * tile[tx][qq]);
      }
    }
  }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
namespace {

struct GroupPlan {
  int64_t ld;    // group width (multiple of kChunk)
};

int64_t choose_group(int64_t n, int32_t k, size_t elem) {
  // keep ~3 live [n][G] buffers within ~64 MB of L2
  const double budget = 64.0 * 1024 * 1024;
  int64_t g = (int64_t)(budget / (3.0 * (double)n * (double)elem));
  g = (g / kChunk) * kChunk;
  const int64_t kk = ((int64_t)k + kChunk - 1) / kChunk * kChunk;
  g = std::max<int64_t>(g, kChunk);
  g = std::min<int64_t>(g, kk);
  g = std::min<int64_t>(g, 4096);
  return g;
}

// A wave of batched views (see k_sweep): the state covers the union-graph
// rows [row0, row0 + nrows), column q is source g0 + q of every row's view;
// lidx[i] is node i's index within its view. The residual's blocks each cover
// the state rows brows[b] of one view; the blocks of the wave's view w are
// [bptr[w], bptr[w + 1]).
struct Wave {
  const int32_t *lidx = nullptr;
  int64_t row0 = 0, nrows = 0;
  int32_t g0 = 0;
  const int2 *brows = nullptr;
  const int *bptr = nullptr;
  const int32_t *nv = nullptr;  // size of each node's view
  int nblocks = 0, nviews = 0;
  // split work items of the wave's rows (k_sweep_sp), or none
  const int4 *items = nullptr;
  const int2 *srow = nullptr;
  int64_t nitems = 0, nsplit = 0, nslots = 0;
};

// Work items of the split sweep (k_sweep_sp) for the rows [r0, r1) of a CSR
// (host row_ptr): the hub rows, with more than max(kSegEdges, 4 x the mean
// degree of the range) edges, in kSegEdges-edge segments, the others whole
// (rows of uniformly high degree gain less from splitting than the partial
// sums cost); split rows and slots numbered from 0. Returns the number of
// slots.
int64_t split_items(const std::vector<int64_t> &rp, int64_t r0, int64_t r1, std::vector<int4> &items,
                    std::vector<int2> &srow) {
  int64_t slots = 0;
  const double mean = r1 > r0 ? (double)(rp[r1] - rp[r0]) / (double)(r1 - r0) : 0.0;
  const int64_t thr = std::max<int64_t>(kSegEdges, (int64_t)(4.0 * mean));
  for (int64_t j = r0; j < r1; ++j) {
    const int64_t len = rp[j + 1] - rp[j];
    if (len <= thr) {
      items.push_back(make_int4((int)j, 0, (int)len, -1));
      continue;
    }
    const int nseg = (int)((len + kSegEdges - 1) / kSegEdges);
    const int sr = (int)srow.size();
    srow.push_back(make_int2((int)slots, nseg));
    for (int q = 0; q < nseg; ++q) {
      const int64_t a = (int64_t)q * kSegEdges;
      items.push_back(make_int4((int)j, (int)a, (int)std::min<int64_t>(kSegEdges, len - a), sr));
    }
    slots += nseg;
  }
  return slots;
}

// The split plan of a whole graph, built once and kept with it.
int sweep_plan(pprviz_ctx *ctx, const pprviz_graph *g) {
  if (g->sp_ready) return PPRVIZ_OK;
  const int64_t n = g->n;
  std::vector<int64_t> rp((size_t)n + 1);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(rp.data(), pull_rp(g), sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int4> items;
  std::vector<int2> srow;
  items.reserve((size_t)n);
  const int64_t slots = split_items(rp, 0, n, items, srow);
  cudaError_t e = g->sp_items.ensure(sizeof(int4) * items.size());
  if (e == cudaSuccess) e = g->sp_srow.ensure(sizeof(int2) * std::max<size_t>(1, srow.size()));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(ctx, PPRVIZ_E_OOM, "sweep work items: allocation failed");
  }
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->sp_items.p, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  if (!srow.empty())
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(g->sp_srow.p, srow.data(), sizeof(int2) * srow.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  g->sp_nitems = (int64_t)items.size();
  g->sp_nsplit = (int64_t)srow.size();
  g->sp_nslots = slots;
  g->sp_ready = true;
  return PPRVIZ_OK;
}

template <typename T>
int launch_sweep(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, bool cheb, bool rhs,
                 const int32_t *src, const float *rhsbuf, const T *ycur, const T *yold, T *yout,
                 double alpha, double om, const Wave *wv = nullptr) {
  constexpr int VEC = Vec<T>::N;
  if constexpr (std::is_same<T, float>::value) {
    if (cheb && (wv ? wv->nsplit > 0 : true)) {
      // FP32 Chebyshev sweep: heavy rows split into segments
      if (!wv) PPRVIZ_TRY(sweep_plan(ctx, g));
      const int64_t nitems = wv ? wv->nitems : g->sp_nitems;
      const int64_t nsplit = wv ? wv->nsplit : g->sp_nsplit;
      const int64_t nslots = wv ? wv->nslots : g->sp_nslots;
      const int4 *items = wv ? wv->items : g->sp_items.as<int4>();
      const int2 *srowp = wv ? wv->srow : g->sp_srow.as<int2>();
      if (nsplit > 0) {
        const int nchunks = (int)(ld / 128);
        PPRVIZ_TRY(ws_ensure(ctx, WS_SPART, sizeof(float) * (size_t)std::max<int64_t>(1, nslots) * (size_t)ld));
        const size_t cbytes = sizeof(int) * (size_t)nsplit * (size_t)nchunks;
        const bool fresh = ctx->ws[WS_SCNT].cap < cbytes || !ctx->ws[WS_SCNT].p;
        PPRVIZ_TRY(ws_ensure(ctx, WS_SCNT, cbytes));
        // the counters return to zero after every sweep; clear them once per call
        if (fresh || !ctx->scnt_clear) {
          PPRVIZ_CUDA(ctx, cudaMemsetAsync(ctx->ws[WS_SCNT].p, 0, ctx->ws[WS_SCNT].cap, ctx->stream));
          ctx->scnt_clear = true;
        }
        const int64_t blocks = nitems * nchunks;
        const float *w = pull_w(g);
        const float a = (float)alpha, c = (float)(1.0 - alpha), o = (float)om, o1 = (float)(1.0 - om);
        const int32_t *srcp = wv ? wv->lidx : src;
        const int64_t row0 = wv ? wv->row0 : 0;
        const int32_t g0 = wv ? wv->g0 : 0;
        PPRVIZ_PROF(ctx, PPRVIZ_K_SWEEP);
#define PPRVIZ_SWEEP_SP(W, R, B)                                                                               \
  k_sweep_sp<W, R, B><<<(unsigned)blocks, 32, 0, ctx->stream>>>(                                                \
      nitems, ld, nchunks, items, srowp, pull_rp(g), pull_col(g), w, g->invdw_f.as<float>(),                    \
      srcp, rhsbuf, (const float *)ycur, (const float *)yold, (float *)yout, a, c, o, o1,                       \
      ctx->ws[WS_SPART].as<float>(), ctx->ws[WS_SCNT].as<int>(), row0, g0)
        if (wv) {
          if (pull_weighted(g)) { if (rhs) PPRVIZ_SWEEP_SP(true, true, true); else PPRVIZ_SWEEP_SP(true, false, true); }
          else { if (rhs) PPRVIZ_SWEEP_SP(false, true, true); else PPRVIZ_SWEEP_SP(false, false, true); }
        } else {
          if (pull_weighted(g)) { if (rhs) PPRVIZ_SWEEP_SP(true, true, false); else PPRVIZ_SWEEP_SP(true, false, false); }
          else { if (rhs) PPRVIZ_SWEEP_SP(false, true, false); else PPRVIZ_SWEEP_SP(false, false, false); }
        }
#undef PPRVIZ_SWEEP_SP
        PPRVIZ_LAUNCHED(ctx);
        return PPRVIZ_OK;
      }
    }
  }
  const int nchunks = (int)(ld / (32 * VEC));
  const int64_t nrows = wv ? wv->nrows : g->n;
  const int64_t items = nrows * nchunks;
  const unsigned blocks = (unsigned)((items + kSweepWarps - 1) / kSweepWarps);
  const T *invdw = std::is_same<T, float>::value ? (const T *)g->invdw_f.p : (const T *)g->invdw_d.p;
  const T a = (T)alpha, c = (T)(1.0 - alpha), o = (T)om, o1 = (T)(1.0 - om);
  const float *w = pull_w(g);
  const int64_t *rp = pull_rp(g);
  const int32_t *col = pull_col(g);
  const int64_t row0 = wv ? wv->row0 : 0;
  const int32_t g0 = wv ? wv->g0 : 0;
  if (wv) src = wv->lidx;
  PPRVIZ_PROF(ctx, PPRVIZ_K_SWEEP);
#define PPRVIZ_SWEEP(W, C, R, B)                                                                   \
  k_sweep<T, W, C, R, B><<<blocks, kSweepWarps * 32, 0, ctx->stream>>>(nrows, ld, nchunks, rp, col, w, invdw, \
                                                                  src, rhsbuf, ycur, yold, yout, a, c, o, o1, row0, g0)
  if (wv) {
    if constexpr (std::is_same<T, float>::value) {
      if (!cheb) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "batched sweeps are Chebyshev sweeps");
      if (pull_weighted(g)) { if (rhs) PPRVIZ_SWEEP(true, true, true, true); else PPRVIZ_SWEEP(true, true, false, true); }
      else { if (rhs) PPRVIZ_SWEEP(false, true, true, true); else PPRVIZ_SWEEP(false, true, false, true); }
    } else {
      return set_err(ctx, PPRVIZ_E_INVALID_ARG, "batched sweeps are FP32");
    }
  } else if (pull_weighted(g)) {
    if (cheb) { if (rhs) PPRVIZ_SWEEP(true, true, true, false); else PPRVIZ_SWEEP(true, true, false, false); }
    else { if (rhs) PPRVIZ_SWEEP(true, false, true, false); else PPRVIZ_SWEEP(true, false, false, false); }
  } else {
    if (cheb) { if (rhs) PPRVIZ_SWEEP(false, true, true, false); else PPRVIZ_SWEEP(false, true, false, false); }
    else { if (rhs) PPRVIZ_SWEEP(false, false, true, false); else PPRVIZ_SWEEP(false, false, false, false); }
  }
#undef PPRVIZ_SWEEP
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

// EXACT selects FP64 accumulation of the neighbour sums; otherwise the FP32
// path uses the error-free compensated sums (certificate floor ~1e-9 at the
// largest degrees, so tighter eps needs EXACT).
// l1 receives, per view of the group (one view unless batched), 2 * ld
// doubles: sum |res| per source, then sum res per source.
template <typename T, bool EXACT>
int launch_residual(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src,
                    const T *yhi, const float *ylo, float *rhs_out, double *l1, double alpha,
                    const Wave *wv = nullptr, int total_blocks = 1216, const double *bscale = nullptr,
                    int32_t level_g0 = 0) {
  const int nchunks = (int)(ld / 128);
  int rows_blocks;
  if (wv) {
    rows_blocks = wv->nblocks;
  } else {
    // `total_blocks` CTAs in all when the group's state fits in L2 (1,216
    // unless tuned); otherwise ~608 per chunk (about the resident CTAs of the
    // GPU), so that the chunks run one after another and only ~one chunk's
    // columns are gathered at a time
    const bool fits_l2 = (double)g->n * (double)ld * 8.0 <= 64.0 * 1024 * 1024;
    rows_blocks = (int)std::min<int64_t>((g->n + kWarps - 1) / kWarps,
                                         fits_l2 ? std::max(1, total_blocks / nchunks) : 608);
  }
  dim3 grid(rows_blocks, nchunks);
  PPRVIZ_TRY(ws_ensure(ctx, WS_RPART, sizeof(double) * 2 * (size_t)rows_blocks * (size_t)ld));
  double *part = ctx->ws[WS_RPART].as<double>();
  const float *w = pull_w(g);
  const int64_t n = wv ? wv->nrows : g->n;
  const int2 *brows = wv ? wv->brows : nullptr;
  const int64_t row0 = wv ? wv->row0 : 0;
  const int32_t g0 = wv ? wv->g0 : level_g0;
  if (wv) src = wv->lidx;
#define PPRVIZ_RES(W, B, L, LOW)                                                                             \
  k_residual<T, W, EXACT, B, L, LOW><<<grid, kWarps * 32, 0, ctx->stream>>>(                                   \
      n, ld, pull_rp(g), pull_col(g), w, g->invdw_d.as<double>(), g->dwff.as<float2>(), src,                   \
      yhi, ylo, rhs_out, part, alpha, 1.0 - alpha, brows, row0, g0, bscale)
  {
    PPRVIZ_PROF(ctx, PPRVIZ_K_RESIDUAL);
    if (wv) { if (pull_weighted(g)) PPRVIZ_RES(true, true, false, true); else PPRVIZ_RES(false, true, false, true); }
    else if (bscale) { if (pull_weighted(g)) PPRVIZ_RES(true, false, true, true); else PPRVIZ_RES(false, false, true, true); }
    else if (pull_weighted(g)) PPRVIZ_RES(true, false, false, true);
    else if (ylo) PPRVIZ_RES(false, false, false, true);
    else PPRVIZ_RES(false, false, false, false);  // no low parts: a lighter instance (fewer registers)
  }
#undef PPRVIZ_RES
  PPRVIZ_LAUNCHED(ctx);
  if (wv) {
    const int64_t warps = (int64_t)wv->nviews * ld;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_RESIDUAL); k_res_reduce_batch<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, ctx->stream>>>(
        ld, wv->nviews, wv->bptr, part, l1); }
  } else {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_RESIDUAL); k_res_reduce<<<(unsigned)((ld * 32 + 255) / 256), 256, 0, ctx->stream>>>(ld, rows_blocks, part, l1, l1 + ld); }
  }
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

// Autotuner of the FP32 CSR path's launch shapes, per size class (bit
// lengths of n, nnz and k, weighted or not), kept in the context so that its
// cost (a few milliseconds) is paid on the first call of each class:
//  * the source-group width G: candidates 128, 256, ... up to the width whose
//    ~3 live [n][G] buffers fill ~64 MB of L2 (choose_group); each runs three
//    timed Chebyshev sweeps on the graph (after one untimed), and the width
//    with the least time per source and sweep wins;
//  * then, at that width, the residual's CTA count (608 .. 4,864 in all): three
//    timed residual passes with a low part each, the fastest wins.
// The values of the state do not change the work of either kernel, so both
// are timed on zeroed buffers.
struct TunedShape {
  int64_t group;
  int res_blocks;
};

TunedShape tuned_shape(pprviz_ctx *ctx, const pprviz_graph *g, int32_t k, int *status) {
  *status = PPRVIZ_OK;
  auto bits = [](uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return (uint64_t)b; };
  const uint64_t key = (bits((uint64_t)g->n) << 40) | (bits((uint64_t)g->nnz) << 32) | (bits((uint64_t)k) << 8) |
                       (g->weighted ? 1u : 0u) | (g->directed ? 2u : 0u);
  for (const auto &e : ctx->tuned_groups)
    if (e.first == key) return TunedShape{e.second >> 16, (int)(e.second & 0xFFFF)};
  const int64_t gmax = choose_group(g->n, k, sizeof(float));
  std::vector<int64_t> cands;
  for (int64_t c = kChunk; c < gmax; c *= 2) cands.push_back(c);
  cands.push_back(gmax);
  int64_t best = gmax;
  int best_res = 1216;
  {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      cudaGetLastError();
      if (e0) cudaEventDestroy(e0);
      *status = set_err(ctx, PPRVIZ_E_CUDA, "autotuner: event creation failed");
      return TunedShape{gmax, 1216};
    }
    double best_score = 0.0;
    int st = PPRVIZ_OK;
    for (int64_t G : cands) {
      if (cands.size() == 1) break;
      const size_t bytes = sizeof(float) * (size_t)(g->n * G);
      if ((st = ws_ensure(ctx, WS_Y0, bytes)) != PPRVIZ_OK) break;
      if ((st = ws_ensure(ctx, WS_Y1, bytes)) != PPRVIZ_OK) break;
      if ((st = ws_ensure(ctx, WS_SRC, sizeof(int32_t) * (size_t)G)) != PPRVIZ_OK) break;
      float *ya = ctx->ws[WS_Y0].as<float>(), *yb = ctx->ws[WS_Y1].as<float>();
      const int32_t *src = ctx->ws[WS_SRC].as<int32_t>();
      cudaError_t ce = cudaMemsetAsync(ya, 0, bytes, ctx->stream);
      if (ce == cudaSuccess) ce = cudaMemsetAsync(yb, 0, bytes, ctx->stream);
      if (ce == cudaSuccess) ce = cudaMemsetAsync(ctx->ws[WS_SRC].p, 0xFF, sizeof(int32_t) * (size_t)G, ctx->stream);
      if (ce != cudaSuccess) { st = cuda_err(ctx, ce, "autotuner"); break; }
      float ms = 0.0f;
      for (int rep = 0; rep < 4 && st == PPRVIZ_OK; ++rep) {
        if (rep == 1) cudaEventRecord(e0, ctx->stream);
        st = launch_sweep<float>(ctx, g, G, true, false, src, nullptr, (rep & 1) ? yb : ya, (rep & 1) ? ya : yb,
                                 (rep & 1) ? ya : yb, 0.15, 1.0);
      }
      if (st != PPRVIZ_OK) break;
      cudaEventRecord(e1, ctx->stream);
      if ((ce = cudaEventSynchronize(e1)) != cudaSuccess || (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
        st = cuda_err(ctx, ce, "autotuner timing");
        break;
      }
      const double score = (double)ms / (double)G;
      if (best_score == 0.0 || score < best_score) {
        best_score = score;
        best = G;
      }
    }
    // the residual's CTA count at the chosen width (only where its state fits in L2)
    const bool fits_l2 = (double)g->n * (double)best * 8.0 <= 64.0 * 1024 * 1024;
    if (st == PPRVIZ_OK && fits_l2 && g->n >= 8 * 608) {
      const size_t bytes = sizeof(float) * (size_t)(g->n * best);
      if (st == PPRVIZ_OK) st = ws_ensure(ctx, WS_Y0, bytes);
      if (st == PPRVIZ_OK) st = ws_ensure(ctx, WS_Y1, bytes);
      if (st == PPRVIZ_OK) st = ws_ensure(ctx, WS_RHS, bytes);
      if (st == PPRVIZ_OK) st = ws_ensure(ctx, WS_SRC, sizeof(int32_t) * (size_t)best);
      if (st == PPRVIZ_OK) st = ws_ensure(ctx, WS_CERT, 2 * sizeof(double) * (size_t)best);
      cudaError_t ce = cudaSuccess;
      if (st == PPRVIZ_OK) ce = cudaMemsetAsync(ctx->ws[WS_Y0].p, 0, bytes, ctx->stream);
      if (st == PPRVIZ_OK && ce == cudaSuccess) ce = cudaMemsetAsync(ctx->ws[WS_Y1].p, 0, bytes, ctx->stream);
      if (st == PPRVIZ_OK && ce == cudaSuccess)
        ce = cudaMemsetAsync(ctx->ws[WS_SRC].p, 0xFF, sizeof(int32_t) * (size_t)best, ctx->stream);
      if (st == PPRVIZ_OK && ce != cudaSuccess) st = cuda_err(ctx, ce, "autotuner");
      double best_t = 0.0;
      for (int total : {608, 1216, 2432, 4864}) {
        if (st != PPRVIZ_OK) break;
        float ms = 0.0f;
        for (int rep = 0; rep < 4 && st == PPRVIZ_OK; ++rep) {
          if (rep == 1) cudaEventRecord(e0, ctx->stream);
          st = launch_residual<float, false>(ctx, g, best, ctx->ws[WS_SRC].as<int32_t>(), ctx->ws[WS_Y0].as<float>(),
                                             ctx->ws[WS_Y1].as<float>(), ctx->ws[WS_RHS].as<float>(),
                                             ctx->ws[WS_CERT].as<double>(), 0.15, nullptr, total);
        }
        if (st != PPRVIZ_OK) break;
        cudaEventRecord(e1, ctx->stream);
        if ((ce = cudaEventSynchronize(e1)) != cudaSuccess || (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
          st = cuda_err(ctx, ce, "autotuner timing");
          break;
        }
        if (best_t == 0.0 || ms < best_t) {
          best_t = ms;
          best_res = total;
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PPRVIZ_OK) {
      *status = st;
      return TunedShape{gmax, 1216};
    }
  }
  ctx->tuned_groups.push_back({key, (best << 16) | best_res});
  return TunedShape{best, best_res};
}

// certificates of the group's sources: d(s) * ||res_s||_1 / alpha
// (and the signed residual sums sigma_q = sum_j res_jq, which fix the
// stationary coefficient of the next correction)
int read_certs(pprviz_ctx *ctx, const pprviz_graph *g, const std::vector<int32_t> &view_h, int32_t g0,
               int32_t gvalid, int64_t ld, const double *l1_d, double alpha, std::vector<double> &cert,
               std::vector<double> &sigma) {
  std::vector<double> l1((size_t)2 * ld);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(l1.data(), l1_d, sizeof(double) * 2 * (size_t)ld,
                                   cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  cert.resize((size_t)gvalid);
  sigma.assign((size_t)ld, 0.0);
  for (int32_t q = 0; q < gvalid; ++q) {
    cert[q] = g->h_deg[view_h[g0 + q]] * l1[q] / alpha;
    sigma[q] = l1[(size_t)ld + q];
  }
  return PPRVIZ_OK;
}

double chebyshev_rate(double c) { return (1.0 - sqrt(1.0 - c * c)) / c; }

// Runs `sweeps` Chebyshev steps of x (I - cP) = b for the interval
// [1 - delta, 1 + delta] of the iterated modes. Without deflation (csrc ==
// nullptr, delta = c) from x_0 = 0, x_1 = b; with it from the stationary
// multiple x_0 = kappa (in y) and x_1 = c x_0 + b.
// On entry ya, yb are the two state buffers; returns the buffer holding the
// last iterate.  b is the source delta (rhs == nullptr) or the dense rhs.
// `tcerr` non-null selects the dense tensor-core sweeps (it receives their
// error word); otherwise the CSR gather sweeps run.
int chebyshev_solve(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src,
                    int32_t gcount, const float *rhs, float *ya, float *yb, int sweeps,
                    double alpha, int *tcerr, const int32_t *csrc, const double *kappa, double delta,
                    float **result, const Wave *wv = nullptr, bool bf16 = false) {
  const size_t bytes = sizeof(float) * (size_t)(g->n * ld);
  const double c = 1.0 - alpha;
  if (wv) {
    // kappa: the sources' stationary coefficients by graph node, or NULL
    const int64_t cnt = wv->nrows * ld;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_defl_batch<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(
        wv->nrows, ld, wv->row0, wv->g0, wv->lidx, wv->nv, g->comp.as<int32_t>(), kappa, rhs, g->invdw_f.as<float>(),
        (float)alpha, (float)c, ya, yb); }
    PPRVIZ_LAUNCHED(ctx);
  } else if (csrc) {
    const int64_t cnt = g->n * ld;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_defl<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(
        g->n, ld, g->comp.as<int32_t>(), csrc, kappa, src, rhs, g->invdw_f.as<float>(), (float)alpha, (float)c, ya, yb); }
    PPRVIZ_LAUNCHED(ctx);
  } else {
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(ya, 0, bytes, ctx->stream));
  if (rhs) {
    const int64_t cnt = g->n * ld;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_rhs<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(g->n, ld, rhs, g->invdw_f.as<float>(), yb); }
    PPRVIZ_LAUNCHED(ctx);
  } else {
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(yb, 0, bytes, ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_delta<float><<<(gcount + 255) / 256, 256, 0, ctx->stream>>>(gcount, src, ld, g->invdw_f.as<float>(),
                                                                      (float)alpha, yb); }
    PPRVIZ_LAUNCHED(ctx);
  }
  }
  // theta = 1: omega_2 = 1 / (1 - delta^2 / 2), omega_{k+1} = 1 / (1 - delta^2 omega_k / 4)
  double om = 1.0;
  float *cur = yb, *old = ya;
  const double d2 = delta * delta;
  for (int s = 1; s < sweeps; ++s) {
    om = (s == 1) ? 1.0 / (1.0 - d2 / 2.0) : 1.0 / (1.0 - d2 * om / 4.0);
    if (tcerr)
      PPRVIZ_TRY(dense_sweep(ctx, g, ld, src, rhs, cur, old, alpha, om, tcerr, bf16));
    else
      PPRVIZ_TRY(launch_sweep<float>(ctx, g, ld, true, rhs != nullptr, src, rhs, cur, old, old, alpha, om, wv));
    std::swap(cur, old);
  }
  *result = cur;
  return PPRVIZ_OK;
}

}  // namespace

int dppr_solve(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d,
               const std::vector<int32_t> &view_h, int32_t k, double alpha, double eps,
               int precision, void *dppr_d, bool out64, double *cert_h) {
  const bool fp64 = precision == PPRVIZ_FP64;
  const size_t elem = fp64 ? sizeof(double) : sizeof(float);
  // sweep kernel: dense tensor-core contraction (forced, or chosen by density
  // when the n x n matrix fits) or CSR gathers
  bool dense = false;
  // BF16 operands on the tensor cores; a BF16 solve resolves ~2^-8 of its
  // correction, so its sweeps stop there and more refinement passes follow
  const bool bf16 = precision == PPRVIZ_FP32_BF16TC;
  if ((precision == PPRVIZ_FP32_TC || bf16) && g->directed)
    return set_err(ctx, PPRVIZ_E_INVALID_ARG, "the tensor-core sweeps take undirected graphs");
  if (precision == PPRVIZ_FP32_TC || bf16) {
    PPRVIZ_TRY(dense_prepare(ctx, g));
    dense = true;
  } else if (precision == PPRVIZ_FP32 && !g->directed && dense_eligible(g)) {
    dense = dense_prepare(ctx, g) == PPRVIZ_OK;
    if (!dense) ctx->err.clear();
  }
  int64_t ld = 0;
  int res_blocks = 1216;
  if (dense) {
    ld = dense_group(k);
  } else if (fp64) {
    ld = choose_group(g->n, k, elem);
  } else {
    int ts = PPRVIZ_OK;
    const TunedShape sh = tuned_shape(ctx, g, k, &ts);
    PPRVIZ_TRY(ts);
    ld = sh.group;
    res_blocks = sh.res_blocks;
  }
  const size_t sbytes = elem * (size_t)(g->n * ld);
  const double c = 1.0 - alpha;
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y0, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y1, sbytes));
  if (!fp64) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_Y2, sbytes));
    PPRVIZ_TRY(ws_ensure(ctx, WS_Y3, sbytes));
    PPRVIZ_TRY(ws_ensure(ctx, WS_RHS, sbytes));
  }
  PPRVIZ_TRY(ws_ensure(ctx, WS_SRC, sizeof(int32_t) * (size_t)ld));
  PPRVIZ_TRY(ws_ensure(ctx, WS_CERT, 2 * sizeof(double) * (size_t)ld));
  int32_t *src = ctx->ws[WS_SRC].as<int32_t>();
  double *l1 = ctx->ws[WS_CERT].as<double>();
  // deflated sweeps (FP32): component roots and the spectral bound of the graph
  bool defl = false;
  double bsp = 1.0;
  int32_t *csrc = nullptr;
  double *kappa = nullptr;
  // a directed walk is not reversible: its spectrum is complex, so the FP32
  // path runs power sweeps (the Chebyshev weights with an interval of width 0)
  // from the plain start instead of deflated Chebyshev sweeps
  const bool power = g->directed;
  if (!fp64 && !power) {
    PPRVIZ_TRY(graph_spectral(ctx, g));
    defl = g->spec_deflate;
    bsp = defl ? g->spec_b : 1.0;
  }
  if (!fp64) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_CSRC, sizeof(int32_t) * (size_t)ld));
    PPRVIZ_TRY(ws_ensure(ctx, WS_KAPPA, sizeof(double) * (size_t)ld));
    csrc = ctx->ws[WS_CSRC].as<int32_t>();
    kappa = ctx->ws[WS_KAPPA].as<double>();
  }
  std::vector<int32_t> csrc_h((size_t)ld, -1);
  std::vector<double> kappa_h((size_t)ld, 0.0), sigma;
  int *tcerr = nullptr;
  if (dense) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
    tcerr = ctx->ws[WS_FLAG].as<int>();
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(tcerr, 0, sizeof(int), ctx->stream));
  }
  pprviz_stats &st = ctx->stats;
  st.source_group = (int32_t)ld;
  std::vector<int32_t> srch((size_t)ld);
  std::vector<double> cert;
  bool not_converged = false;
  // rate of the iterated modes on [1 - delta, 1 + delta] (power sweeps: c)
  auto rate = [power, c](double delta) { return power ? c : (delta > 1e-12 ? chebyshev_rate(delta) : 0.0); };
  auto sweeps_for = [](double factor, double r) {  // K with 2 r^K <= factor
    return r > 0.0 ? (int)ceil(log(0.5 * factor) / log(r)) : 1;
  };
  // the compensated FP32 residual resolves certificates down to ~1e-9; below
  // that the neighbour sums are accumulated in FP64
  const bool exact_res = eps < 1e-9;

  for (int32_t g0 = 0; g0 < k; g0 += (int32_t)ld) {
    const int32_t gvalid = (int32_t)std::min<int64_t>(ld, (int64_t)k - g0);
    for (int64_t q = 0; q < ld; ++q) srch[q] = q < gvalid ? view_h[g0 + q] : -1;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(src, srch.data(), sizeof(int32_t) * (size_t)ld,
                                     cudaMemcpyHostToDevice, ctx->stream));
    double dmax = 0.0;
    for (int32_t q = 0; q < gvalid; ++q) dmax = std::max(dmax, g->h_deg[view_h[g0 + q]]);
    st.groups++;
    const void *yhi = nullptr;
    const float *ylo = nullptr;
    if (fp64) {
      // power iteration for T sweeps: d(s) c^(T+1) <= eps / 2 for every source of the group
      int T = 0;
      if (dmax > 0.0) T = std::max(0, (int)ceil(log(0.5 * eps / dmax) / log(c)) - 1);
      double *ya = ctx->ws[WS_Y0].as<double>(), *yb = ctx->ws[WS_Y1].as<double>();
      PPRVIZ_CUDA(ctx, cudaMemsetAsync(ya, 0, sbytes, ctx->stream));
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_delta<double><<<(unsigned)((ld + 255) / 256), 256, 0, ctx->stream>>>(
          (int32_t)ld, src, ld, g->invdw_d.as<double>(), alpha, ya); }
      PPRVIZ_LAUNCHED(ctx);
      double *cur = ya, *nxt = yb;
      for (int s = 0; s < T; ++s) {
        PPRVIZ_TRY(launch_sweep<double>(ctx, g, ld, false, false, src, nullptr, cur, nullptr, nxt, alpha, 1.0));
        std::swap(cur, nxt);
      }
      st.sweeps_main += T;
      st.bytes_sweep += 16.0 * (double)g->n * gvalid * T;
      PPRVIZ_TRY((launch_residual<double, true>(ctx, g, ld, src, cur, nullptr, nullptr, l1, alpha)));
      st.residual_passes++;
      PPRVIZ_TRY(read_certs(ctx, g, view_h, g0, gvalid, ld, l1, alpha, cert, sigma));
      yhi = cur;
    } else {
      float *bufs[4] = {ctx->ws[WS_Y0].as<float>(), ctx->ws[WS_Y1].as<float>(), ctx->ws[WS_Y2].as<float>(),
                        ctx->ws[WS_Y3].as<float>()};
      float *rhs = ctx->ws[WS_RHS].as<float>();
      // deflated start: the source's component root per column, and the
      // stationary coefficient 1 / m_C of the main system
      if (defl) {
        for (int64_t q = 0; q < ld; ++q) {
          csrc_h[q] = q < gvalid ? g->h_comp[view_h[g0 + q]] : -1;
          kappa_h[q] = q < gvalid ? 1.0 / g->h_mc[(size_t)csrc_h[q]] : 0.0;
        }
        PPRVIZ_CUDA(ctx, cudaMemcpyAsync(csrc, csrc_h.data(), sizeof(int32_t) * (size_t)ld, cudaMemcpyHostToDevice,
                                         ctx->stream));
        PPRVIZ_CUDA(ctx, cudaMemcpyAsync(kappa, kappa_h.data(), sizeof(double) * (size_t)ld,
                                         cudaMemcpyHostToDevice, ctx->stream));
      }
      double delta_c = power ? 0.0 : c * bsp;
      // main solve to a Chebyshev error bound 2 rho^K <= 1e-5: every further
      // sweep here would only save one refinement sweep, and the refinement
      // (driven by the exact FP64 residual) finishes the job
      // (BF16: to 2 rho^K <= 1e-3, about what BF16 products resolve)
      const int K1 = std::max(2, sweeps_for(bf16 ? 1e-3 : 1e-5, rate(delta_c)));
      float *hi = nullptr;
      PPRVIZ_TRY(chebyshev_solve(ctx, g, ld, src, (int32_t)ld, nullptr, bufs[0], bufs[1], K1, alpha, tcerr,
                                 defl ? csrc : nullptr, kappa, delta_c, &hi, nullptr, bf16));
      st.sweeps_main += K1;
      if (dense) st.flops_dense += 2.0 * (double)g->n * (double)g->n * gvalid * (K1 - 1);
      else st.bytes_sweep += 12.0 * (double)g->n * gvalid * (K1 - 1);
      // free buffers for the correction solves; the first correction becomes x_lo
      float *fa = hi == bufs[0] ? bufs[1] : bufs[0], *fb = bufs[2], *fc = bufs[3];
      float *lo = nullptr;
      PPRVIZ_TRY((exact_res ? launch_residual<float, true>(ctx, g, ld, src, hi, nullptr, rhs, l1, alpha, nullptr, res_blocks)
                            : launch_residual<float, false>(ctx, g, ld, src, hi, nullptr, rhs, l1, alpha, nullptr, res_blocks)));
      st.residual_passes++;
      PPRVIZ_TRY(read_certs(ctx, g, view_h, g0, gvalid, ld, l1, alpha, cert, sigma));
      double cprev = 0.0;
      for (int pass = 0; pass < (bf16 ? kMaxRefineBf16 : kMaxRefine); ++pass) {
        double cmax = 0.0;
        for (double v : cert) cmax = std::max(cmax, v);
        if (cmax <= eps) break;
        // a pass that gained less than 10x (BF16: 2x) means modes outside the
        // estimated interval: iterate the full interval [1 - c, 1 + c] from here on
        if (!power && pass > 0 && cmax > (bf16 ? 0.5 : 0.1) * cprev) delta_c = c;
        cprev = cmax;
        // correction's stationary coefficient: sum_j res_jq / alpha over m_C
        if (defl) {
          for (int64_t q = 0; q < gvalid; ++q) kappa_h[q] = sigma[q] / (alpha * g->h_mc[(size_t)csrc_h[q]]);
          PPRVIZ_CUDA(ctx, cudaMemcpyAsync(kappa, kappa_h.data(), sizeof(double) * (size_t)ld,
                                           cudaMemcpyHostToDevice, ctx->stream));
        }
        // sweeps for the correction: its Chebyshev error must fall by eps / (4 cmax),
        // but an FP32 correction resolves only ~1e-7 of itself per pass, so
        // sweeps past 2 rho^K ~ 3e-8 are left to the next pass
        int K2 = sweeps_for(0.5 * eps / cmax, rate(delta_c)) + 2;
        K2 = std::min(std::max(K2, 4), power ? 4 * kMaxRefineSweeps : kMaxRefineSweeps);
        if (bf16) K2 = std::min(K2, sweeps_for(1e-3, rate(delta_c)) + 1);
        float *delta = nullptr;
        PPRVIZ_TRY(chebyshev_solve(ctx, g, ld, src, (int32_t)ld, rhs, fa, fb, K2, alpha, tcerr,
                                   defl ? csrc : nullptr, kappa, delta_c, &delta, nullptr, bf16));
        st.sweeps_refine += K2;
        if (dense) st.flops_dense += 2.0 * (double)g->n * (double)g->n * gvalid * (K2 - 1);
        else st.bytes_sweep += 16.0 * (double)g->n * gvalid * (K2 - 1);
        st.refine_passes++;
        if (!lo) {
          lo = delta;
          fa = (delta == fa) ? fb : fa;
          fb = fc;
        } else {
          const int64_t cnt = g->n * ld;
          { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_axpy<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, delta, lo); }
          PPRVIZ_LAUNCHED(ctx);
        }
        {
          const int64_t cnt = g->n * ld;
          { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_renorm<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, hi, lo); }
          PPRVIZ_LAUNCHED(ctx);
        }
        PPRVIZ_TRY((exact_res ? launch_residual<float, true>(ctx, g, ld, src, hi, lo, rhs, l1, alpha, nullptr, res_blocks)
                              : launch_residual<float, false>(ctx, g, ld, src, hi, lo, rhs, l1, alpha, nullptr, res_blocks)));
        st.residual_passes++;
        PPRVIZ_TRY(read_certs(ctx, g, view_h, g0, gvalid, ld, l1, alpha, cert, sigma));
      }
      yhi = hi;
      ylo = lo;
    }
    for (int32_t q = 0; q < gvalid; ++q) {
      st.max_cert = std::max(st.max_cert, cert[q]);
      if (cert[q] > eps) not_converged = true;
      if (cert_h) cert_h[g0 + q] = cert[q];
    }
    if (dppr_d) {
      dim3 grid((unsigned)((gvalid + 31) / 32), (unsigned)((k + 31) / 32));
      dim3 block(32, 8);
      if (fp64) {
        if (out64)
          { PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT); k_extract<double, double><<<grid, block, 0, ctx->stream>>>(k, g0, gvalid, ld, view_d, g->deg.as<double>(),
              g->invdw_d.as<double>(), g->dwff.as<float2>(), (const double *)yhi, nullptr, (double *)dppr_d); }
        else
          { PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT); k_extract<double, float><<<grid, block, 0, ctx->stream>>>(k, g0, gvalid, ld, view_d, g->deg.as<double>(),
              g->invdw_d.as<double>(), g->dwff.as<float2>(), (const double *)yhi, nullptr, (float *)dppr_d); }
      } else {
        if (out64)
          { PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT); k_extract<float, double><<<grid, block, 0, ctx->stream>>>(k, g0, gvalid, ld, view_d, g->deg.as<double>(),
              g->invdw_d.as<double>(), g->dwff.as<float2>(), (const float *)yhi, ylo, (double *)dppr_d); }
        else
          { PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT); k_extract<float, float><<<grid, block, 0, ctx->stream>>>(k, g0, gvalid, ld, view_d, g->deg.as<double>(),
              g->invdw_d.as<double>(), g->dwff.as<float2>(), (const float *)yhi, ylo, (float *)dppr_d); }
      }
      PPRVIZ_LAUNCHED(ctx);
    }
  }
  if (tcerr) {
    int herr = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, tcerr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "tensor-core sweep: an MMA completion wait expired");
  }
  if (not_converged)
    return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "certificate above eps after the refinement cap");
  return PPRVIZ_OK;
}


// --------------------------------------------------------------------------
// Level-l DPPR between supernodes (Sec. 3.2, Definition 2, Eq. (2)):
//   pi_d(V_i, V_j) = sum_{s in F(V_i), t in F(V_j)} pi_d(s, t) / (|F(V_i)| |F(V_j)|).
// By linearity the inner sum over s is one PPR solve from the group start
// b_i = alpha sum_{s in F(V_i)} d(s) / |F(V_i)| e_s (the initial residues of
// GFP, Algorithm 2): rho_i = b_i (I - cP)^-1 = sum_s d(s) / |F(V_i)| pi(s, .),
// and pi_d(V_i, V_j) is the average of rho_i over F(V_j). One source column per
// supernode runs the FP32 Chebyshev sweeps with a dense right-hand side; the
// FP64 residual (LEVEL mode, exact b) and FP32 refinement certify every entry
// of rho_i to ||res_i||_1 / alpha, which bounds each average as well.
// --------------------------------------------------------------------------
namespace {

// rhs[j][q] = alpha * bscale[j] if node j is a leaf of supernode g0 + q, else 0
__global__ void k_level_rhs(int64_t n, int64_t ld, int32_t g0, const int32_t *__restrict__ owner,
                            const double *__restrict__ bscale, double alpha, float *__restrict__ rhs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * ld) return;
  const int64_t j = idx / ld, q = idx - j * ld;
  rhs[idx] = (owner[j] == g0 + (int32_t)q) ? (float)(alpha * bscale[j]) : 0.0f;
}

// out[(g0 + q) * nsup + r] = sum_{t in F(V_r)} x_q(t) / |F(V_r)|, x = dw (y_hi + y_lo),
// in FP64; block (chunk of 128 columns, target supernode r), thread = column.
template <typename TO>
__global__ void __launch_bounds__(128)
k_level_extract(int32_t nsup, int32_t g0, int32_t gvalid, int64_t ld, const int64_t *__restrict__ leaf_ptr,
                const int32_t *__restrict__ leaf_idx, const double *__restrict__ invdw, const float *__restrict__ yhi,
                const float *__restrict__ ylo, TO *__restrict__ out) {
  const int32_t r = blockIdx.y;
  const int32_t q = blockIdx.x * 128 + threadIdx.x;
  if (q >= gvalid) return;
  const int64_t a = leaf_ptr[r], e = leaf_ptr[r + 1];
  double acc = 0.0;
  for (int64_t p = a; p < e; ++p) {
    const int64_t t = leaf_idx[p];
    const double y = (double)yhi[t * ld + q] + (ylo ? (double)ylo[t * ld + q] : 0.0);
    acc += y / invdw[t];
  }
  out[(int64_t)(g0 + q) * nsup + r] = (TO)(acc / (double)(e - a));
}

}  // namespace

int level_dppr_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr_d,
                     const int32_t *leaf_idx_d, const std::vector<int64_t> &leaf_ptr_h,
                     const std::vector<int32_t> &leaf_idx_h, double alpha, double eps, void *out_d, bool out64,
                     double *cert_h) {
  const int64_t n = g->n;
  // owner of each node and the FP64 right-hand-side scale d(j) / |F(V_owner)|
  std::vector<int32_t> owner((size_t)n, -1);
  std::vector<double> bscale((size_t)n, 0.0);
  for (int32_t v = 0; v < nsup; ++v) {
    const double sz = (double)(leaf_ptr_h[v + 1] - leaf_ptr_h[v]);
    for (int64_t p = leaf_ptr_h[v]; p < leaf_ptr_h[v + 1]; ++p) {
      const int32_t t = leaf_idx_h[p];
      owner[t] = v;
      bscale[t] = g->h_deg[t] / sz;
    }
  }
  const int64_t ld = choose_group(n, nsup, sizeof(float));
  const size_t sbytes = sizeof(float) * (size_t)(n * ld);
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y0, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y1, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y2, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y3, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_RHS, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_SRC, sizeof(int32_t) * (size_t)std::max<int64_t>(n, ld)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_CERT, 2 * sizeof(double) * (size_t)ld));
  PPRVIZ_TRY(ws_ensure(ctx, WS_KAPPA, sizeof(double) * (size_t)n));
  int32_t *owner_d = ctx->ws[WS_SRC].as<int32_t>();
  double *bscale_d = ctx->ws[WS_KAPPA].as<double>();
  double *l1 = ctx->ws[WS_CERT].as<double>();
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(owner_d, owner.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(bscale_d, bscale.data(), sizeof(double) * (size_t)n, cudaMemcpyHostToDevice,
                                   ctx->stream));
  pprviz_stats &st = ctx->stats;
  st.source_group = (int32_t)ld;
  const double c = 1.0 - alpha;
  const bool power = g->directed;
  auto rate = [power, c](double delta) { return power ? c : (delta > 1e-12 ? chebyshev_rate(delta) : 0.0); };
  auto sweeps_for = [](double factor, double r) { return r > 0.0 ? (int)ceil(log(0.5 * factor) / log(r)) : 1; };
  const bool exact_res = eps < 1e-9;
  bool not_converged = false;
  std::vector<double> l1h((size_t)2 * ld);
  for (int32_t g0 = 0; g0 < nsup; g0 += (int32_t)ld) {
    const int32_t gvalid = (int32_t)std::min<int64_t>(ld, (int64_t)nsup - g0);
    st.groups++;
    float *bufs[4] = {ctx->ws[WS_Y0].as<float>(), ctx->ws[WS_Y1].as<float>(), ctx->ws[WS_Y2].as<float>(),
                      ctx->ws[WS_Y3].as<float>()};
    float *rhs = ctx->ws[WS_RHS].as<float>();
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER);
      k_level_rhs<<<(unsigned)((n * ld + 255) / 256), 256, 0, ctx->stream>>>(n, ld, g0, owner_d, bscale_d, alpha, rhs);
    }
    PPRVIZ_LAUNCHED(ctx);
    // undeflated Chebyshev on the whole interval [1 - c, 1 + c] (a leaf set
    // may span several components); power sweeps on a directed graph
    const double delta_c = g->directed ? 0.0 : c;
    const int K1 = std::max(2, sweeps_for(1e-5, rate(delta_c)));
    float *hi = nullptr;
    PPRVIZ_TRY(chebyshev_solve(ctx, g, ld, owner_d, (int32_t)ld, rhs, bufs[0], bufs[1], K1, alpha, nullptr, nullptr,
                               nullptr, delta_c, &hi));
    st.sweeps_main += K1;
    st.bytes_sweep += 16.0 * (double)n * gvalid * (K1 - 1);
    float *fa = hi == bufs[0] ? bufs[1] : bufs[0], *fb = bufs[2], *fc = bufs[3];
    float *lo = nullptr;
    std::vector<double> cert((size_t)gvalid);
    auto certs = [&](const float *yh, const float *yl) -> int {
      PPRVIZ_TRY((exact_res ? launch_residual<float, true>(ctx, g, ld, owner_d, yh, yl, rhs, l1, alpha, nullptr, 1216,
                                                            bscale_d, g0)
                            : launch_residual<float, false>(ctx, g, ld, owner_d, yh, yl, rhs, l1, alpha, nullptr, 1216,
                                                             bscale_d, g0)));
      st.residual_passes++;
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(l1h.data(), l1, sizeof(double) * 2 * (size_t)ld, cudaMemcpyDeviceToHost,
                                       ctx->stream));
      PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      for (int32_t q = 0; q < gvalid; ++q) cert[q] = l1h[q] / alpha;
      return PPRVIZ_OK;
    };
    PPRVIZ_TRY(certs(hi, nullptr));
    for (int pass = 0; pass < kMaxRefine; ++pass) {
      double cmax = 0.0;
      for (double v : cert) cmax = std::max(cmax, v);
      if (cmax <= eps) break;
      int K2 = sweeps_for(0.5 * eps / cmax, rate(delta_c)) + 2;
      K2 = std::min(std::max(K2, 4), power ? 4 * kMaxRefineSweeps : kMaxRefineSweeps);
      float *delta = nullptr;
      PPRVIZ_TRY(chebyshev_solve(ctx, g, ld, owner_d, (int32_t)ld, rhs, fa, fb, K2, alpha, nullptr, nullptr, nullptr,
                                 delta_c, &delta));
      st.sweeps_refine += K2;
      st.bytes_sweep += 16.0 * (double)n * gvalid * (K2 - 1);
      st.refine_passes++;
      const int64_t cnt = n * ld;
      if (!lo) {
        lo = delta;
        fa = (delta == fa) ? fb : fa;
        fb = fc;
      } else {
        { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_axpy<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, delta, lo); }
        PPRVIZ_LAUNCHED(ctx);
      }
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_renorm<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, hi, lo); }
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_TRY(certs(hi, lo));
    }
    for (int32_t q = 0; q < gvalid; ++q) {
      st.max_cert = std::max(st.max_cert, cert[q]);
      if (cert[q] > eps) not_converged = true;
      if (cert_h) cert_h[g0 + q] = cert[q];
    }
    {
      PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT);
      const dim3 grid((unsigned)((gvalid + 127) / 128), (unsigned)nsup);
      if (out64)
        k_level_extract<double><<<grid, 128, 0, ctx->stream>>>(nsup, g0, gvalid, ld, leaf_ptr_d, leaf_idx_d,
                                                                g->invdw_d.as<double>(), hi, lo, (double *)out_d);
      else
        k_level_extract<float><<<grid, 128, 0, ctx->stream>>>(nsup, g0, gvalid, ld, leaf_ptr_d, leaf_idx_d,
                                                               g->invdw_d.as<double>(), hi, lo, (float *)out_d);
    }
    PPRVIZ_LAUNCHED(ctx);
  }
  if (not_converged)
    return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "certificate above eps after the refinement cap");
  return PPRVIZ_OK;
}

// --------------------------------------------------------------------------
// Frontier profile (diagnostic for Algorithm 2's threshold). Power iteration
// x_{t+1} = alpha e_s + c x_t P is Forward-Push with every node pushed once
// per sweep: after sweep t the push residue of node v is, in DPPR units,
// r_v = d(s) (x_{t+1} - x_t)_v / alpha (Eq. (3)). GFP pushes only nodes with
// r_v > d(v) r_max; r_max = eps / max_{t in view} d(t) bounds every DPPR
// entry of the view by eps (sum_v r_v pi(v, t) <= r_max d(t) on an undirected
// graph). This counts, per sweep, the (node, source) entries above it.
// --------------------------------------------------------------------------
namespace {

__global__ void k_frontier_count(int64_t n, int64_t ld, int32_t gvalid, const double *__restrict__ ycur,
                                 const double *__restrict__ ynext, const double *__restrict__ invdw,
                                 const double *__restrict__ deg, const double *__restrict__ dsrc, double alpha,
                                 double rmax, unsigned long long *__restrict__ count) {
  __shared__ unsigned int blk;
  if (threadIdx.x == 0) blk = 0;
  __syncthreads();
  unsigned int mine = 0;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n * ld;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = idx / ld, q = idx - v * ld;
    if (q >= gvalid) continue;
    const double r = dsrc[q] * fabs(ynext[idx] - ycur[idx]) / invdw[v] / alpha;
    if (r > deg[v] * rmax) ++mine;
  }
  atomicAdd(&blk, mine);
  __syncthreads();
  if (threadIdx.x == 0 && blk) atomicAdd(count, (unsigned long long)blk);
}

}  // namespace

int frontier_profile(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view_d,
                     const std::vector<int32_t> &view_h, int32_t k, double alpha, double eps, int32_t sweeps,
                     int64_t *active_h) {
  const int64_t n = g->n;
  const int64_t ld = choose_group(n, k, sizeof(double));
  const size_t sbytes = sizeof(double) * (size_t)(n * ld);
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y0, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y1, sbytes));
  PPRVIZ_TRY(ws_ensure(ctx, WS_SRC, sizeof(int32_t) * (size_t)ld));
  PPRVIZ_TRY(ws_ensure(ctx, WS_KAPPA, sizeof(double) * (size_t)ld));
  PPRVIZ_TRY(ws_ensure(ctx, WS_MISC, sizeof(unsigned long long) * (size_t)sweeps));
  int32_t *src = ctx->ws[WS_SRC].as<int32_t>();
  double *dsrc = ctx->ws[WS_KAPPA].as<double>();
  unsigned long long *cnt = ctx->ws[WS_MISC].as<unsigned long long>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)sweeps, ctx->stream));
  double dmax = 0.0;
  for (int32_t q = 0; q < k; ++q) dmax = std::max(dmax, g->h_deg[view_h[q]]);
  const double rmax = dmax > 0.0 ? eps / dmax : eps;
  std::vector<int32_t> srch((size_t)ld);
  std::vector<double> dsh((size_t)ld);
  const double c = 1.0 - alpha;
  (void)c;
  for (int32_t g0 = 0; g0 < k; g0 += (int32_t)ld) {
    const int32_t gvalid = (int32_t)std::min<int64_t>(ld, (int64_t)k - g0);
    for (int64_t q = 0; q < ld; ++q) {
      srch[q] = q < gvalid ? view_h[g0 + q] : -1;
      dsh[q] = q < gvalid ? g->h_deg[view_h[g0 + q]] : 0.0;
    }
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(src, srch.data(), sizeof(int32_t) * (size_t)ld, cudaMemcpyHostToDevice,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(dsrc, dsh.data(), sizeof(double) * (size_t)ld, cudaMemcpyHostToDevice,
                                     ctx->stream));
    double *ya = ctx->ws[WS_Y0].as<double>(), *yb = ctx->ws[WS_Y1].as<double>();
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(ya, 0, sbytes, ctx->stream));
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_init_delta<double><<<(unsigned)((ld + 255) / 256), 256, 0, ctx->stream>>>(
        (int32_t)ld, src, ld, g->invdw_d.as<double>(), alpha, ya); }
    PPRVIZ_LAUNCHED(ctx);
    double *cur = ya, *nxt = yb;
    for (int32_t t = 0; t < sweeps; ++t) {
      PPRVIZ_TRY(launch_sweep<double>(ctx, g, ld, false, false, src, nullptr, cur, nullptr, nxt, alpha, 1.0));
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_frontier_count<<<1216, 256, 0, ctx->stream>>>(
          n, ld, gvalid, cur, nxt, g->invdw_d.as<double>(), g->deg.as<double>(), dsrc, alpha, rmax, cnt + t); }
      PPRVIZ_LAUNCHED(ctx);
      std::swap(cur, nxt);
    }
  }
  std::vector<unsigned long long> h((size_t)sweeps);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(h.data(), cnt, sizeof(unsigned long long) * (size_t)sweeps,
                                   cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  for (int32_t t = 0; t < sweeps; ++t) active_h[t] = (int64_t)h[t];
  return PPRVIZ_OK;
}

// --------------------------------------------------------------------------
// Batched views (P7): many views of uneven size in shared launches.
//
// The views are laid out, largest first, as the disjoint union of their
// graphs (node ids offset, CSR concatenated; lidx = index within the view,
// nv = the view's size). Consecutive views of similar size form a wave, a
// contiguous row range of the union; column q of a wave's state is source q
// of every view in it at once (k_sweep, BATCH), so one sweep launch advances
// all sources of all views of the wave. Each wave iterates its Chebyshev
// sweeps on the largest spectral bound of its views. Per-view results
// (certificates, DPPR rows, PDist) are separated again by row range.
// --------------------------------------------------------------------------
namespace {

struct UnionDesc {
  const int64_t *rp;
  const int32_t *col;
  const float *w;
  const double *deg, *invd;
  const float *invf;
  const float2 *dwff;
  int64_t n, off, nnzoff;
};

__global__ void k_union_build(const UnionDesc *__restrict__ d, int64_t *__restrict__ rp, int32_t *__restrict__ col,
                              float *__restrict__ w, double *__restrict__ deg, float *__restrict__ invf,
                              double *__restrict__ invd, float2 *__restrict__ dwff, int32_t *__restrict__ lidx,
                              int32_t *__restrict__ nv) {
  const UnionDesc v = d[blockIdx.y];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= v.n) return;
  const int64_t gi = v.off + i;
  const int64_t b = v.rp[i], e = v.rp[i + 1];
  rp[gi] = b + v.nnzoff;
  if (i == v.n - 1) rp[gi + 1] = e + v.nnzoff;  // equals the next view's first entry
  for (int64_t k = b; k < e; ++k) {
    col[v.nnzoff + k] = v.col[k] + (int32_t)v.off;
    if (w) w[v.nnzoff + k] = v.w ? v.w[k] : 1.0f;
  }
  deg[gi] = v.deg[i];
  invf[gi] = v.invf[i];
  invd[gi] = v.invd[i];
  dwff[gi] = v.dwff[i];
  lidx[gi] = (int32_t)i;
  nv[gi] = (int32_t)v.n;
}

// a workspace slot seen as a graph buffer (released with the context)
pprviz::DevBuf slot_view(pprviz_ctx *ctx, int slot) { return ctx->ws[slot]; }

}  // namespace

// Source-group width of a wave of the batched propagation, tuned on first
// use per size class (bit lengths of the wave's rows, edges and width): the
// candidates 128, 256, ... up to the budget's width each run three timed
// Chebyshev sweeps of the wave (after one untimed) on zeroed buffers, and
// the width with the least time per source and sweep wins.
int64_t tuned_wave_group(pprviz_ctx *ctx, const pprviz_graph *U, const Wave &wv0, int64_t width, int64_t ldmax,
                         int64_t nnz, int *status) {
  *status = PPRVIZ_OK;
  if (ldmax <= kChunk) return ldmax;
  auto bits = [](uint64_t x) { int b = 0; while (x) { ++b; x >>= 1; } return (uint64_t)b; };
  const uint64_t key = (1ull << 63) | (bits((uint64_t)wv0.nrows) << 40) | (bits((uint64_t)nnz) << 32) |
                       (bits((uint64_t)width) << 8) | (U->weighted ? 1u : 0u);
  for (const auto &e : ctx->tuned_groups)
    if (e.first == key) return std::min<int64_t>(e.second, ldmax);
  std::vector<int64_t> cands;
  for (int64_t c = kChunk; c < ldmax; c *= 2) cands.push_back(c);
  cands.push_back(ldmax);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    *status = set_err(ctx, PPRVIZ_E_CUDA, "wave autotuner: event creation failed");
    return ldmax;
  }
  int64_t best = ldmax;
  double best_score = 0.0;
  float *ya = ctx->ws[WS_Y0].as<float>(), *yb = ctx->ws[WS_Y1].as<float>();
  for (int64_t G : cands) {
    const size_t bytes = sizeof(float) * (size_t)(wv0.nrows * G);
    cudaError_t ce = cudaMemsetAsync(ya, 0, bytes, ctx->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(yb, 0, bytes, ctx->stream);
    if (ce != cudaSuccess) {
      *status = cuda_err(ctx, ce, "wave autotuner");
      break;
    }
    Wave wv = wv0;
    wv.g0 = 0;
    float ms = 0.0f;
    int st = PPRVIZ_OK;
    for (int rep = 0; rep < 4 && st == PPRVIZ_OK; ++rep) {
      if (rep == 1) cudaEventRecord(e0, ctx->stream);
      st = launch_sweep<float>(ctx, U, G, true, false, nullptr, nullptr, (rep & 1) ? yb : ya, (rep & 1) ? ya : yb,
                               (rep & 1) ? ya : yb, 0.15, 1.0, &wv);
    }
    if (st != PPRVIZ_OK) {
      *status = st;
      break;
    }
    cudaEventRecord(e1, ctx->stream);
    if ((ce = cudaEventSynchronize(e1)) != cudaSuccess || (ce = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) {
      *status = cuda_err(ctx, ce, "wave autotuner timing");
      break;
    }
    const double score = (double)ms / (double)G;
    if (best_score == 0.0 || score < best_score) {
      best_score = score;
      best = G;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (*status == PPRVIZ_OK) ctx->tuned_groups.push_back({key, best});
  return best;
}

int dppr_views_solve(pprviz_ctx *ctx, int32_t nviews, const pprviz_graph *const *views, const int64_t *node_off,
                     const int64_t *sq_off, double alpha, double eps, const int32_t *iota_d, float *pdist_all,
                     double *cert_h) {
  const double c = 1.0 - alpha;
  // processing order: largest view first (stable)
  std::vector<int32_t> order((size_t)nviews);
  for (int32_t v = 0; v < nviews; ++v) order[v] = v;
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return views[a]->n > views[b]->n; });
  std::vector<int64_t> uoff((size_t)nviews), unnz((size_t)nviews);
  int64_t N = 0, NNZ = 0, maxn = 0;
  bool weighted = false;
  for (int32_t v = 0; v < nviews; ++v)
    if (views[v]->directed) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "batched views take undirected graphs");
  for (int32_t i = 0; i < nviews; ++i) {
    const pprviz_graph *g = views[order[i]];
    uoff[order[i]] = N;
    unnz[order[i]] = NNZ;
    N += g->n;
    NNZ += g->nnz;
    maxn = std::max(maxn, g->n);
    weighted = weighted || g->weighted;
  }
  if (N > INT32_MAX) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "the views hold more than 2^31 - 1 nodes in all");
  if (nviews > 65535) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "at most 65,535 views per batch");
  // ---- the union graph, in workspace slots
  PPRVIZ_TRY(ws_ensure(ctx, WS_URP, sizeof(int64_t) * (size_t)(N + 1)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UCOL, sizeof(int32_t) * (size_t)std::max<int64_t>(NNZ, 1)));
  if (weighted) PPRVIZ_TRY(ws_ensure(ctx, WS_UW, sizeof(float) * (size_t)std::max<int64_t>(NNZ, 1)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UDEG, sizeof(double) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UINVD, sizeof(double) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UINVF, sizeof(float) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UDWFF, sizeof(float2) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_ULIDX, sizeof(int32_t) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UNV, sizeof(int32_t) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UCOMP, sizeof(int32_t) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UKAP, 2 * sizeof(double) * (size_t)N));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UDESC, sizeof(UnionDesc) * (size_t)nviews));
  std::vector<UnionDesc> desc((size_t)nviews);
  for (int32_t v = 0; v < nviews; ++v) {
    const pprviz_graph *g = views[v];
    desc[v] = UnionDesc{g->rp.as<int64_t>(), g->col.as<int32_t>(), g->weighted ? g->w.as<float>() : nullptr,
                        g->deg.as<double>(), g->invdw_d.as<double>(), g->invdw_f.as<float>(), g->dwff.as<float2>(),
                        g->n, uoff[v], unnz[v]};
  }
  UnionDesc *desc_d = ctx->ws[WS_UDESC].as<UnionDesc>();
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(desc_d, desc.data(), sizeof(UnionDesc) * (size_t)nviews, cudaMemcpyHostToDevice,
                                   ctx->stream));
  {
    dim3 grid((unsigned)((maxn + 255) / 256), (unsigned)nviews);
    PPRVIZ_PROF(ctx, PPRVIZ_K_GRAPH);
    k_union_build<<<grid, 256, 0, ctx->stream>>>(desc_d, ctx->ws[WS_URP].as<int64_t>(), ctx->ws[WS_UCOL].as<int32_t>(),
                                                 weighted ? ctx->ws[WS_UW].as<float>() : nullptr,
                                                 ctx->ws[WS_UDEG].as<double>(), ctx->ws[WS_UINVF].as<float>(),
                                                 ctx->ws[WS_UINVD].as<double>(), ctx->ws[WS_UDWFF].as<float2>(),
                                                 ctx->ws[WS_ULIDX].as<int32_t>(), ctx->ws[WS_UNV].as<int32_t>());
  }
  PPRVIZ_LAUNCHED(ctx);
  pprviz_graph U;
  U.ctx = ctx;
  U.device = ctx->device;
  U.n = N;
  U.nnz = NNZ;
  U.weighted = weighted;
  U.rp = slot_view(ctx, WS_URP);
  U.col = slot_view(ctx, WS_UCOL);
  if (weighted) U.w = slot_view(ctx, WS_UW);
  U.deg = slot_view(ctx, WS_UDEG);
  U.invdw_d = slot_view(ctx, WS_UINVD);
  U.invdw_f = slot_view(ctx, WS_UINVF);
  U.dwff = slot_view(ctx, WS_UDWFF);
  U.comp = slot_view(ctx, WS_UCOMP);  // component roots, filled from the views below
  U.h_deg.resize((size_t)N);
  for (int32_t v = 0; v < nviews; ++v)
    std::copy(views[v]->h_deg.begin(), views[v]->h_deg.end(), U.h_deg.begin() + uoff[v]);
  const int32_t *lidx = ctx->ws[WS_ULIDX].as<int32_t>();
  const int32_t *nvr = ctx->ws[WS_UNV].as<int32_t>();
  // components and spectral bound of every view (computed once per graph and
  // kept with it); the union's component roots are the views' roots offset
  bool defl = true;
  for (int32_t v = 0; v < nviews; ++v) {
    PPRVIZ_TRY(graph_spectral(ctx, views[v]));
    defl = defl && views[v]->spec_deflate;
  }
  U.h_comp.resize((size_t)N);
  U.h_mc.assign((size_t)N, 0.0);
  for (int32_t v = 0; v < nviews; ++v) {
    const pprviz_graph *g = views[v];
    for (int64_t i = 0; i < g->n; ++i) {
      U.h_comp[(size_t)(uoff[v] + i)] = (int32_t)(uoff[v] + g->h_comp[(size_t)i]);
      U.h_mc[(size_t)(uoff[v] + i)] = g->h_mc[(size_t)i];
    }
  }
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(U.comp.p, U.h_comp.data(), sizeof(int32_t) * (size_t)N, cudaMemcpyHostToDevice,
                                   ctx->stream));
  double *kap_main = ctx->ws[WS_UKAP].as<double>(), *kap_corr = kap_main + N;
  std::vector<double> kap_h((size_t)N, 0.0);
  if (defl) {
    for (int64_t sidx = 0; sidx < N; ++sidx) kap_h[sidx] = 1.0 / U.h_mc[(size_t)U.h_comp[sidx]];
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(kap_main, kap_h.data(), sizeof(double) * (size_t)N, cudaMemcpyHostToDevice,
                                     ctx->stream));
  }

  // ---- waves: consecutive views (largest first) whose state of full width
  // keeps ~3 live buffers within ~64 MB of L2; a view too large for that
  // alone gets its own wave and a narrower source group
  struct WaveDef {
    int32_t first, last;  // positions in `order`, inclusive first, exclusive last
    int64_t row0, nrows, width, ld;
  };
  std::vector<WaveDef> waves;
  const double budget = 64.0 * 1024 * 1024;
  for (int32_t i = 0; i < nviews;) {
    const int64_t n0 = views[order[i]]->n;
    const int64_t width = (n0 + kChunk - 1) / kChunk * kChunk;
    WaveDef wd{i, i + 1, uoff[order[i]], n0, width, width};
    while (wd.last < nviews && (double)(wd.nrows + views[order[wd.last]]->n) * (double)width * 12.0 <= budget)
      wd.nrows += views[order[wd.last++]]->n;
    int64_t ld = (int64_t)(budget / (12.0 * (double)wd.nrows)) / kChunk * kChunk;
    wd.ld = std::min(width, std::max<int64_t>(kChunk, std::min<int64_t>(ld, 4096)));
    waves.push_back(wd);
    i = wd.last;
  }
  // buffers: five states of the largest wave x group, the wave's DPPR
  // matrices, the residual's row blocks
  size_t smax = 0, dmax = 0;
  int nbmax = 0;
  for (const WaveDef &wd : waves) {
    smax = std::max(smax, sizeof(float) * (size_t)(wd.nrows * wd.ld));
    size_t dd = 0;
    for (int32_t i = wd.first; i < wd.last; ++i) dd += (size_t)views[order[i]]->n * (size_t)views[order[i]]->n;
    dmax = std::max(dmax, dd);
    nbmax = std::max(nbmax, (int)(wd.last - wd.first) + 1216);
  }
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y0, smax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y1, smax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y2, smax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_Y3, smax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_RHS, smax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_DPPR, sizeof(float) * std::max<size_t>(dmax, 1)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UBROWS, sizeof(int2) * (size_t)nbmax));
  PPRVIZ_TRY(ws_ensure(ctx, WS_UBPTR, sizeof(int) * (size_t)(nviews + 1)));
  // split work items of every wave (rows of more than kSegEdges edges in
  // segments), from the union CSR, concatenated wave after wave
  std::vector<int64_t> urp((size_t)N + 1);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(urp.data(), U.rp.p, sizeof(int64_t) * urp.size(), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  std::vector<int4> witems;
  std::vector<int2> wsrow;
  struct WaveSplit { size_t item0, srow0; int64_t nitems, nsplit, nslots; };
  std::vector<WaveSplit> wsplit;
  for (const WaveDef &wd : waves) {
    WaveSplit ws{witems.size(), wsrow.size(), 0, 0, 0};
    std::vector<int2> sr;
    ws.nslots = split_items(urp, wd.row0, wd.row0 + wd.nrows, witems, sr);
    ws.nitems = (int64_t)(witems.size() - ws.item0);
    ws.nsplit = (int64_t)sr.size();
    wsrow.insert(wsrow.end(), sr.begin(), sr.end());
    wsplit.push_back(ws);
  }
  PPRVIZ_TRY(ws_ensure(ctx, WS_UITEMS, sizeof(int4) * std::max<size_t>(1, witems.size())));
  PPRVIZ_TRY(ws_ensure(ctx, WS_USROW, sizeof(int2) * std::max<size_t>(1, wsrow.size())));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ctx->ws[WS_UITEMS].p, witems.data(), sizeof(int4) * witems.size(),
                                   cudaMemcpyHostToDevice, ctx->stream));
  if (!wsrow.empty())
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ctx->ws[WS_USROW].p, wsrow.data(), sizeof(int2) * wsrow.size(),
                                     cudaMemcpyHostToDevice, ctx->stream));
  int64_t ldmax = 0;
  for (const WaveDef &wd : waves) ldmax = std::max(ldmax, wd.ld);
  PPRVIZ_TRY(ws_ensure(ctx, WS_CERT, 2 * sizeof(double) * (size_t)ldmax * (size_t)nviews));
  float *dppr_w = ctx->ws[WS_DPPR].as<float>();
  int2 *brows_d = ctx->ws[WS_UBROWS].as<int2>();
  int *bptr_d = ctx->ws[WS_UBPTR].as<int>();
  double *l1 = ctx->ws[WS_CERT].as<double>();
  pprviz_stats &st = ctx->stats;
  const bool exact_res = eps < 1e-9;
  auto rate = [](double delta) { return delta > 1e-12 ? chebyshev_rate(delta) : 0.0; };
  auto sweeps_for = [](double factor, double r) { return r > 0.0 ? (int)ceil(log(0.5 * factor) / log(r)) : 1; };
  bool not_converged = false;

  for (size_t wi = 0; wi < waves.size(); ++wi) {
    WaveDef wd = waves[wi];
    const int nvw = (int)(wd.last - wd.first);
    {
      // autotuned source-group width of the wave (cached per size class)
      Wave tw;
      tw.lidx = lidx;
      tw.nv = nvr;
      tw.row0 = wd.row0;
      tw.nrows = wd.nrows;
      tw.nviews = nvw;
      tw.items = ctx->ws[WS_UITEMS].as<int4>() + wsplit[wi].item0;
      tw.srow = ctx->ws[WS_USROW].as<int2>() + wsplit[wi].srow0;
      tw.nitems = wsplit[wi].nitems;
      tw.nsplit = wsplit[wi].nsplit;
      tw.nslots = wsplit[wi].nslots;
      int64_t nnzw = urp[(size_t)(wd.row0 + wd.nrows)] - urp[(size_t)wd.row0];
      int ts = PPRVIZ_OK;
      wd.ld = tuned_wave_group(ctx, &U, tw, wd.width, wd.ld, nnzw, &ts);
      PPRVIZ_TRY(ts);
    }
    // residual row blocks: ~1,216 blocks of the wave shared in proportion to
    // the views' sizes (at least one each), never straddling two views
    std::vector<int2> brows;
    std::vector<int> bptr((size_t)nvw + 1, 0);
    const int nchunks = (int)(wd.ld / 128);
    const double share = std::max(1.0, 1216.0 / nchunks) / (double)wd.nrows;
    for (int w = 0; w < nvw; ++w) {
      const pprviz_graph *g = views[order[wd.first + w]];
      const int64_t r0 = uoff[order[wd.first + w]] - wd.row0;
      int64_t nb = std::max<int64_t>(1, (int64_t)(share * (double)g->n));
      nb = std::min<int64_t>(nb, (g->n + kWarps - 1) / kWarps);
      const int64_t per = (g->n + nb - 1) / nb;
      for (int64_t r = 0; r < g->n; r += per) brows.push_back(make_int2((int)(r0 + r), (int)(r0 + std::min(g->n, r + per))));
      bptr[w + 1] = (int)brows.size();
    }
    PPRVIZ_TRY(ws_ensure(ctx, WS_UBROWS, sizeof(int2) * brows.size()));
    brows_d = ctx->ws[WS_UBROWS].as<int2>();
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(brows_d, brows.data(), sizeof(int2) * brows.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(bptr_d, bptr.data(), sizeof(int) * bptr.size(), cudaMemcpyHostToDevice,
                                     ctx->stream));
    Wave wv;
    wv.lidx = lidx;
    wv.nv = nvr;
    wv.row0 = wd.row0;
    wv.nrows = wd.nrows;
    wv.brows = brows_d;
    wv.bptr = bptr_d;
    wv.nblocks = (int)brows.size();
    wv.nviews = nvw;
    wv.items = ctx->ws[WS_UITEMS].as<int4>() + wsplit[wi].item0;
    wv.srow = ctx->ws[WS_USROW].as<int2>() + wsplit[wi].srow0;
    wv.nitems = wsplit[wi].nitems;
    wv.nsplit = wsplit[wi].nsplit;
    wv.nslots = wsplit[wi].nslots;
    const int64_t ld = wd.ld;
    const int64_t cnt = wd.nrows * ld;
    // the wave's iterated modes: |lambda| <= the largest bound of its views
    double bsp = 0.0;
    for (int w = 0; w < nvw; ++w) bsp = std::max(bsp, views[order[wd.first + w]]->spec_b);
    if (!defl) bsp = 1.0;
    // DPPR matrices of the wave's views, packed in wave order
    std::vector<size_t> doff((size_t)nvw + 1, 0);
    for (int w = 0; w < nvw; ++w) {
      const int64_t n = views[order[wd.first + w]]->n;
      doff[w + 1] = doff[w] + (size_t)n * (size_t)n;
    }
    for (int64_t g0 = 0; g0 < wd.width; g0 += ld) {
      wv.g0 = (int32_t)g0;
      st.groups++;
      float *bufs[4] = {ctx->ws[WS_Y0].as<float>(), ctx->ws[WS_Y1].as<float>(), ctx->ws[WS_Y2].as<float>(),
                        ctx->ws[WS_Y3].as<float>()};
      float *rhs = ctx->ws[WS_RHS].as<float>();
      double delta_c = c * bsp;
      const int K1 = std::max(2, sweeps_for(1e-5, rate(delta_c)));
      float *hi = nullptr;
      PPRVIZ_TRY(chebyshev_solve(ctx, &U, ld, nullptr, (int32_t)ld, nullptr, bufs[0], bufs[1], K1, alpha, nullptr,
                                 nullptr, defl ? kap_main : nullptr, delta_c, &hi, &wv));
      st.sweeps_main += K1;
      st.bytes_sweep += 12.0 * (double)cnt * (K1 - 1);
      float *fa = hi == bufs[0] ? bufs[1] : bufs[0], *fb = bufs[2], *fc = bufs[3];
      float *lo = nullptr;
      // certificates: cert of source (view w, column q) = d(s) ||res||_1 / alpha
      std::vector<double> l1h((size_t)2 * ld * nvw), cert;
      double cmax = 0.0;
      auto certs = [&]() -> int {
        PPRVIZ_CUDA(ctx, cudaMemcpyAsync(l1h.data(), l1, sizeof(double) * l1h.size(), cudaMemcpyDeviceToHost,
                                         ctx->stream));
        PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        cmax = 0.0;
        for (int w = 0; w < nvw; ++w) {
          const int32_t v = order[wd.first + w];
          const int64_t gv = std::min<int64_t>(ld, views[v]->n - g0);
          for (int64_t q = 0; q < gv; ++q) {
            const double cq = views[v]->h_deg[(size_t)(g0 + q)] * l1h[(size_t)(w * 2) * ld + q] / alpha;
            cmax = std::max(cmax, cq);
          }
        }
        return PPRVIZ_OK;
      };
      PPRVIZ_TRY((exact_res ? launch_residual<float, true>(ctx, &U, ld, nullptr, hi, nullptr, rhs, l1, alpha, &wv)
                            : launch_residual<float, false>(ctx, &U, ld, nullptr, hi, nullptr, rhs, l1, alpha, &wv)));
      st.residual_passes++;
      PPRVIZ_TRY(certs());
      double cprev = 0.0;
      for (int pass = 0; pass < kMaxRefine && cmax > eps; ++pass) {
        if (pass > 0 && cmax > 0.1 * cprev) delta_c = c;
        cprev = cmax;
        if (defl) {
          // the corrections' stationary coefficients, by source node
          for (int w = 0; w < nvw; ++w) {
            const int32_t v = order[wd.first + w];
            const int64_t gv = std::min<int64_t>(ld, views[v]->n - g0);
            for (int64_t q = 0; q < gv; ++q) {
              const int64_t sn = uoff[v] + g0 + q;
              kap_h[(size_t)sn] = l1h[(size_t)(w * 2 + 1) * ld + q] / (alpha * U.h_mc[(size_t)U.h_comp[(size_t)sn]]);
            }
          }
          PPRVIZ_CUDA(ctx, cudaMemcpyAsync(kap_corr + wd.row0, kap_h.data() + wd.row0, sizeof(double) * (size_t)wd.nrows,
                                           cudaMemcpyHostToDevice, ctx->stream));
        }
        int K2 = sweeps_for(0.5 * eps / cmax, rate(delta_c)) + 2;
        K2 = std::min(std::max(K2, 4), kMaxRefineSweeps);
        float *dl = nullptr;
        PPRVIZ_TRY(chebyshev_solve(ctx, &U, ld, nullptr, (int32_t)ld, rhs, fa, fb, K2, alpha, nullptr, nullptr,
                                   defl ? kap_corr : nullptr, delta_c, &dl, &wv));
        st.sweeps_refine += K2;
        st.bytes_sweep += 16.0 * (double)cnt * (K2 - 1);
        st.refine_passes++;
        if (!lo) {
          lo = dl;
          fa = (dl == fa) ? fb : fa;
          fb = fc;
        } else {
          { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_axpy<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, dl, lo); }
          PPRVIZ_LAUNCHED(ctx);
        }
        { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_renorm<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, hi, lo); }
        PPRVIZ_LAUNCHED(ctx);
        PPRVIZ_TRY((exact_res ? launch_residual<float, true>(ctx, &U, ld, nullptr, hi, lo, rhs, l1, alpha, &wv)
                              : launch_residual<float, false>(ctx, &U, ld, nullptr, hi, lo, rhs, l1, alpha, &wv)));
        st.residual_passes++;
        PPRVIZ_TRY(certs());
      }
      // per view: certificates and the DPPR rows g0 .. g0 + gvalid
      for (int w = 0; w < nvw; ++w) {
        const int32_t v = order[wd.first + w];
        const pprviz_graph *g = views[v];
        const int64_t gv = std::min<int64_t>(ld, g->n - g0);
        if (gv <= 0) continue;
        for (int64_t q = 0; q < gv; ++q) {
          const double cq = g->h_deg[(size_t)(g0 + q)] * l1h[(size_t)(w * 2) * ld + q] / alpha;
          st.max_cert = std::max(st.max_cert, cq);
          if (cq > eps) not_converged = true;
          if (cert_h) cert_h[node_off[v] + g0 + q] = cq;
        }
        const int64_t rs = uoff[v] - wd.row0;  // first state row of the view
        dim3 grid((unsigned)((gv + 31) / 32), (unsigned)((g->n + 31) / 32));
        dim3 block(32, 8);
        { PPRVIZ_PROF(ctx, PPRVIZ_K_EXTRACT); k_extract<float, float><<<grid, block, 0, ctx->stream>>>(
            (int32_t)g->n, (int32_t)g0, (int32_t)gv, ld, iota_d, U.deg.as<double>() + uoff[v],
            U.invdw_d.as<double>() + uoff[v], U.dwff.as<float2>() + uoff[v], hi + rs * ld,
            lo ? lo + rs * ld : nullptr, dppr_w + doff[w]); }
        PPRVIZ_LAUNCHED(ctx);
      }
    }
    for (int w = 0; w < nvw; ++w) {
      const int32_t v = order[wd.first + w];
      const int64_t n = views[v]->n;
      PPRVIZ_TRY(pdist_launch(ctx, dppr_w + doff[w], (int32_t)n, n, pdist_all + sq_off[v], false));
    }
  }
  st.source_group = (int32_t)ldmax;
  if (not_converged)
    return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "a view's certificate stayed above eps after the refinement cap");
  return PPRVIZ_OK;
}

}  // namespace pprviz
