// P4/P5/P6 - stress energy, gradients and stress-majorization layout.
//
// Paper (Sec. 5, Eq. (7); Appendix A.1, Eqs. (8)-(10)):
//   L(X | Delta) = sum_{i<j} (1 - |X_i - X_j| / Delta_ij)^2
//   L^w[i][j] = -1/Delta_ij^2 (i != j), L^w[i][i] = sum_{k != i} 1/Delta_ik^2
//   L^Y[i][j] = -1/(Delta_ij |Y_i - Y_j|) (i != j, Y_i != Y_j), L^Y[i][i] = -row sum
//   X <- (L^w)^-1 L^Y(Y) Y                                    (Eq. (10))
//
// GB300 design:
//  * L^w does not depend on X, so it is inverted once per view. L^w is a
//    Laplacian (singular on the ones vector); A = L^w + J/k is SPD with
//    A 1 = 1, and for b = L^Y Y (zero column sums) A^-1 b is exactly the
//    centred Moore-Penrose solution. A is inverted once in place by the
//    symmetric block sweep of factor.cu.
//  * The layout works on the symmetric part Delta_s = (Delta + Delta^T)/2 (equal
//    to Delta for the symmetric PDist of Eq. (1)), so 1/Delta_s and M = A^-1 are
//    symmetric and each update reads only their upper-triangle 128 x 128 tiles:
//    a tile (I, J), I < J, adds its row sums to rows I and its column sums to
//    rows J. Two streaming passes per update (b = L^Y X over 1/Delta_s, then
//    X = M b) read half of each k x k matrix once. Partial sums are written
//    per (tile, row) and added in a fixed order: no atomics, reproducible.
//  * The energy and its gradients recompute every pair from X and Delta; no
//    k x k intermediate is stored.
#include <cuda.h>
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace pprviz {

constexpr int ST = 128;       // symmetric pass tile edge
constexpr int SRPI = 8;       // rows per warp per sub-iteration in the symmetric pass
constexpr int LWARPS = 8;     // warps per block in the energy pass
constexpr int RPW = 4;        // rows per warp in the energy pass
constexpr int XCH = 1024;     // coordinates staged per shared-memory chunk (energy)

template <typename T> struct T2;
template <> struct T2<float> { using type = float2; };
template <> struct T2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ T rsqrt_pos(T d2);
template <>
__device__ __forceinline__ float rsqrt_pos<float>(float d2) { return d2 > 0.0f ? rsqrtf(d2) : 0.0f; }
template <>
__device__ __forceinline__ double rsqrt_pos<double>(double d2) { return d2 > 0.0 ? 1.0 / sqrt(d2) : 0.0; }

// four consecutive values, 16-byte aligned
__device__ __forceinline__ void ld4(const float *p, float (&v)[4]) {
  const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&v)[4]) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// ---------------------------------------------------------------------------
// Build from Delta_s = (Delta + Delta^T) / 2, in 32 x 32 tiles with the mirrored
// tile staged in shared memory:
//   W1[i][j] = 1/Delta_s (0 on the diagonal and in the padding),
//   A[i][j]  = 1/k - 1/Delta_s^2 off the diagonal, identity on padded rows,
//   rowpart[J][i] = sum over the tile's 32 columns of 1/Delta_s^2 (FP64);
// k_build_diag then sets A[i][i] = sum_J rowpart[J][i] + 1/k in a fixed order.
// Every consumer reads the upper triangle of 128-row blocks (diagonal 128
// blocks in full), so tiles below the diagonal 128 blocks are not written: the
// mirrored tile above supplies their row sums as its column sums (W1 and A are
// symmetric entry by entry), and checks the mirrored inputs.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T recip(T d) { return T(1) / d; }
template <>
__device__ __forceinline__ float recip<float>(float d) { return __frcp_rn(d); }

template <typename TI, typename T>
__global__ void k_build_sym(int32_t k, int32_t kp, const TI *__restrict__ D, T *__restrict__ W1,
                            T *__restrict__ A, double *__restrict__ rowpart, int *__restrict__ flag) {
  const int by = blockIdx.y, bx = blockIdx.x;
  if ((by >> 2) > (bx >> 2)) return;  // below the diagonal 128 blocks
  const bool mirror = (by >> 2) < (bx >> 2);
  __shared__ TI tr[32][33];
  __shared__ double csum[8][33];
  const int i0 = by * 32, j0 = bx * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + tx;
    tr[jj][tx] = (j < k && i < k) ? D[(int64_t)j * k + i] : TI(0);
  }
  __syncthreads();
  const T invk = (T)(1.0 / (double)k);
  int bad = 0;
  double colacc = 0.0;  // column j0 + tx over this thread's rows
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    double wsq_d = 0.0;
    if (i < k && j < k && i != j) {
      const TI a = D[(int64_t)i * k + j], b = tr[tx][ii];
      // every input entry must itself be a valid distance (this element checks
      // a; b is checked by the element (j, i), or here when that tile is not built)
      if (!(a > TI(0)) || !isfinite((double)a)) bad = 1;
      if (mirror && (!(b > TI(0)) || !isfinite((double)b))) bad = 1;
      const T d = (T)((a + b) * TI(0.5));
      const T w1 = recip(d);
      const T wsq = w1 * w1;
      W1[(int64_t)i * kp + j] = w1;
      A[(int64_t)i * kp + j] = invk - wsq;
      wsq_d = (double)wsq;
    } else {
      W1[(int64_t)i * kp + j] = T(0);
      if (i != j || i >= k) A[(int64_t)i * kp + j] = (i == j) ? T(1) : T(0);
    }
    colacc += wsq_d;
    for (int o = 16; o > 0; o >>= 1) wsq_d += __shfl_xor_sync(0xffffffffu, wsq_d, o);
    if (tx == 0) rowpart[(int64_t)bx * kp + i] = wsq_d;
  }
  if (mirror) {  // the row sums of the tile (bx, by) below: this tile's column sums
    csum[ty][tx] = colacc;
    __syncthreads();
    if (ty == 0) {
      double c = 0.0;
#pragma unroll
      for (int e = 0; e < 8; ++e) c += csum[e][tx];
      rowpart[(int64_t)by * kp + j0 + tx] = c;
    }
  }
  if (bad) atomicOr(flag, 1);
}

template <typename T>
__global__ void k_build_diag(int32_t k, int32_t kp, const double *__restrict__ rowpart, T *__restrict__ A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  double s = 0.0;
  for (int b = 0; b < kp / 32; ++b) s += rowpart[(int64_t)b * kp + i];
  A[(int64_t)i * kp + i] = (T)(s + 1.0 / (double)k);
}

// ---------------------------------------------------------------------------
// Symmetric pair pass over the upper-triangle tiles of a symmetric kp x kp
// matrix Mat (zero beyond k). Block (J, I), I <= J, 8 warps: warp w owns tile
// rows 16w..16w+15 (two sub-iterations of SRPI rows), lane l the four columns
// 4l..4l+3. With v = the staged vector (x for MODE 0, b for MODE 1):
//   MODE 0 (L^Y): t_ij = Mat_ij (v_i - v_j) / |v_i - v_j|; row i gets +t_ij,
//                 column j gets -t_ij (since t_ji = -t_ij)
//   MODE 1 (apply M): row i gets Mat_ij v_j, column j gets Mat_ij v_i
// Row sums go to Part[J][i], column sums (off-diagonal tiles only) to Part[I][j].
// ---------------------------------------------------------------------------
// Sum over the 32 lanes of NV values per lane; returns, in every lane, the
// total of value index lane / (32 / NV). Recursive halving: 31 shuffles for
// NV = 32, 15 + 1 for NV = 16.
template <int NV, typename T>
__device__ __forceinline__ T lanes_transpose_sum(T (&v)[NV], int lane) {
  constexpr int LOG = NV == 32 ? 5 : NV == 16 ? 4 : NV == 8 ? 3 : NV == 4 ? 2 : NV == 2 ? 1 : 0;
#pragma unroll
  for (int s = 0; s < LOG; ++s) {
    const int off = 16 >> s;
    const int half = (NV >> s) / 2;
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int i = 0; i < half; ++i) {
      const T send = up ? v[i] : v[i + half];
      const T keep = up ? v[i + half] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
  }
  T r = v[0];
#pragma unroll
  for (int off = 16 >> LOG; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
  return r;
}

// sum_{o < nb} p[o * kp] in order o = 0, 1, ...; the loads (L2, since other
// CTAs wrote them) are issued 4 at a time so that their latencies overlap,
// the additions keep the order
template <typename V2>
__device__ __forceinline__ V2 sum_parts_in_order(const V2 *p, int64_t kp, int nb) {
  V2 s = __ldcg(p);
  for (int o0 = 1; o0 < nb; o0 += 4) {
    V2 u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (o0 + q < nb) u[q] = __ldcg(p + (int64_t)(o0 + q) * kp);
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (o0 + q < nb) {
        s.x += u[q].x;
        s.y += u[q].y;
      }
  }
  return s;
}

// After its partial sums are written, the tile counts itself in for row
// block I (and, off the diagonal, for row block J); every row block receives
// exactly nbt partials (one per slot), so the CTA that brings a block's count
// to nbt sums that block's partials in slot order into Vout and resets the
// count for the next pass (a deterministic result, independent of which CTA
// finishes last). One thread per CTA fences after the block barrier before
// counting (release) and after a last count (acquire); the reducer reads
// through L2.
template <typename T, int MODE>
__device__ __forceinline__ void sympass_tile(const int I, const int J, int32_t kp, int nbt, const T *__restrict__ Mat,
                                             const typename T2<T>::type *__restrict__ V,
                                             typename T2<T>::type *__restrict__ Part, int *__restrict__ cnt,
                                             typename T2<T>::type *__restrict__ Vout) {
  using V2 = typename T2<T>::type;
  constexpr int NV = 2 * SRPI;
  __shared__ V2 sVi[ST];
  __shared__ T colred[8][2 * ST];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t i0 = (int64_t)I * ST, j0 = (int64_t)J * ST;
  if (threadIdx.x < ST) sVi[threadIdx.x] = V[i0 + threadIdx.x];
  T xj[4], yj[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const V2 v = V[j0 + lane * 4 + u];
    xj[u] = v.x;
    yj[u] = v.y;
  }
  __syncthreads();
  T cx[4], cy[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) cx[u] = cy[u] = T(0);
  T *part = reinterpret_cast<T *>(Part);
#pragma unroll
  for (int sub = 0; sub < 16 / SRPI; ++sub) {
    const int rbase = warp * 16 + sub * SRPI;
    T m[SRPI][4];
#pragma unroll
    for (int r = 0; r < SRPI; ++r) ld4(Mat + (i0 + rbase + r) * kp + j0 + lane * 4, m[r]);
    T acc[NV];
#pragma unroll
    for (int r = 0; r < SRPI; ++r) {
      const V2 vi = sVi[rbase + r];
      T ax = T(0), ay = T(0);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (MODE == 0) {
          const T dx = vi.x - xj[u], dy = vi.y - yj[u];
          const T coef = m[r][u] * rsqrt_pos<T>(dx * dx + dy * dy);
          const T tx = coef * dx, ty = coef * dy;
          ax += tx;
          ay += ty;
          cx[u] -= tx;
          cy[u] -= ty;
        } else {
          ax += m[r][u] * xj[u];
          ay += m[r][u] * yj[u];
          cx[u] += m[r][u] * vi.x;
          cy[u] += m[r][u] * vi.y;
        }
      }
      acc[2 * r] = ax;
      acc[2 * r + 1] = ay;
    }
    const T tot = lanes_transpose_sum<NV, T>(acc, lane);
    constexpr int REP = 32 / NV;
    if (lane % REP == 0) {
      const int idx = lane / REP;
      part[((int64_t)J * kp + i0 + rbase + (idx >> 1)) * 2 + (idx & 1)] = tot;
    }
  }
  if (I != J) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      colred[warp][(lane * 4 + u) * 2] = cx[u];
      colred[warp][(lane * 4 + u) * 2 + 1] = cy[u];
    }
    __syncthreads();
    T s = T(0);
#pragma unroll
    for (int w = 0; w < 8; ++w) s += colred[w][threadIdx.x];
    part[((int64_t)I * kp + j0) * 2 + threadIdx.x] = s;
  }
  __shared__ int last[2];
  __syncthreads();  // every thread's partials are written (CTA scope)
  if (threadIdx.x == 0) {
    __threadfence();  // release, cumulative over the barrier
    last[0] = atomicAdd(&cnt[I], 1) == nbt - 1;
    last[1] = (I != J) ? (atomicAdd(&cnt[J], 1) == nbt - 1) : 0;
    if (last[0] || last[1]) __threadfence();  // acquire before the block reads other CTAs' partials
  }
  __syncthreads();
#pragma unroll 1
  for (int side = 0; side < 2; ++side) {
    if (!last[side]) continue;
    const int R = side ? J : I;
    if (threadIdx.x < ST) {
      const int64_t row = (int64_t)R * ST + threadIdx.x;
      Vout[row] = sum_parts_in_order(Part + row, (int64_t)kp, nbt);
    }
    if (threadIdx.x == 0) cnt[R] = 0;
  }
}

// Views of a pass: block b takes tile tiles[b] = (view, I, J), I <= J, and the
// view's matrix, vector, partial-sum and counter slices from its descriptor.
// A single view is the case of one descriptor.
struct BatchView {
  int64_t mat_off;   // elements into the batched kp x kp matrices
  int64_t vec_off;   // 2-vectors into the batched coordinate / b vectors (kp each)
  int64_t part_off;  // 2-vectors into the batched partial sums (nbt x kp each)
  int32_t kp, nbt, k, cnt_off;  // cnt_off: the view's nbt row-block counters
};

template <typename T, int MODE>
__global__ void __launch_bounds__(256)
k_sympass_batch(const int4 *__restrict__ tiles, const BatchView *__restrict__ views, const T *__restrict__ Mat,
                const typename T2<T>::type *__restrict__ V, typename T2<T>::type *__restrict__ Part,
                int *__restrict__ cnt, typename T2<T>::type *__restrict__ Vout) {
  const int4 t = tiles[blockIdx.x];
  const BatchView bv = views[t.x];
  sympass_tile<T, MODE>(t.y, t.z, bv.kp, bv.nbt, Mat + bv.mat_off, V + bv.vec_off, Part + bv.part_off,
                        cnt + bv.cnt_off, Vout + bv.vec_off);
}

// ---------------------------------------------------------------------------
// FP32 symmetric pass, persistent, pipelined and warp-specialized (the FP32
// path of the single and the batched layout). One CTA per SM: a producer warp
// and 16 consumer warps. Each CTA takes a contiguous chunk of the tile table,
// which lists every view's upper-triangle tiles column by column (J, then
// I = 0..J). The producer brings each 128 x 128 tile (64 KiB) into a
// shared-memory stage with one TMA tensor copy (cp.async.bulk.tensor.2d; a
// tensor map per view and matrix), together with the two 1 KiB coordinate
// slices it needs (plain bulk copies), all completing on the stage's "full"
// mbarrier; it refills a stage once the stage's "empty" mbarrier has seen all
// 16 consumer warps. With PS stages the copies of PS tiles are in flight.
// The consumer warps never wait for each other: warp w takes tile rows
// 8w..8w+7 (lane l the columns 4l..4l+3, one conflict-free 16-byte
// shared-memory read per row), sums its rows across lanes and stores them per
// tile (row block I, slot J), and keeps its column sums in registers while
// consecutive tiles of the chunk share the column block J (a "run"); it
// writes them once per run to the run's slot. A separate launch
// (k_reduce_rows) adds slots and runs in a fixed order. Per pair:
//   MODE 0 (L^Y): t_ij = Mat_ij (v_i - v_j) / |v_i - v_j|: row i +t, column j -t
//   MODE 1 (apply M): row i gets Mat_ij v_j, column j gets Mat_ij v_i
// (the diagonal tile adds its rows only: it is stored in full). Lane l's four
// columns are processed as two pairs with Blackwell's paired FP32
// instructions (two lanes of work per issue slot).
// Every mbarrier wait has an iteration limit: on expiry the warp sets *err and
// stops; the producer then waits (again bounded) for the copies it issued.
// ---------------------------------------------------------------------------
namespace spipe {
constexpr int PS = 3;                           // pipeline stages
constexpr int CWARPS = 16;                      // consumer warps
constexpr int THREADS = (CWARPS + 1) * 32;      // + the producer warp
constexpr int PRW = ST / CWARPS;                // tile rows per consumer warp
constexpr uint32_t TILE_BYTES = ST * ST * 4;    // one FP32 tile
constexpr uint32_t VEC_BYTES = ST * 8;          // 128 coordinate pairs
constexpr uint32_t STAGE_BYTES = TILE_BYTES + 2 * VEC_BYTES;  // tile, rows' and columns' vector slices
constexpr int SMEM = PS * (int)STAGE_BYTES + 1024;  // stages + alignment slack
constexpr long WAIT_LIMIT = 1L << 24;           // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done = 0;
  for (long it = 0; it < WAIT_LIMIT && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
  }
  return done != 0;
}

// One thread: tile (I, J) of the matrix behind `map` and the vector slices
// V[I 128 ..] and V[J 128 ..] (V is the view's vector) into the stage at dst,
// all completing on bar (armed with their byte count first). The maps sit in
// global memory, written by a host copy before the launch; the first use of
// each map by a CTA is preceded by a tensor-map acquire fence (`fenced`
// remembers the last map fenced).
__device__ __forceinline__ void tile_copy(uint32_t dst, uint32_t b, const CUtensorMap *map, int I, int J,
                                          uint64_t policy) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.L2::cache_hint "
      "[%0], [%1, {%2, %3}], [%4], %5;" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(J * ST), "r"(I * ST), "r"(b), "l"(policy)
      : "memory");
}

__device__ __forceinline__ void issue_tile(uint32_t dst, uint64_t *bar, const CUtensorMap *map, const float2 *V,
                                           int I, int J, const CUtensorMap *&fenced, uint64_t policy) {
  if (map != fenced) {
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                 : "memory");
    fenced = map;
  }
  const uint32_t b = smem_u32(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(STAGE_BYTES) : "memory");
  tile_copy(dst, b, map, I, J, policy);
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst + TILE_BYTES),
               "l"(V + (int64_t)I * ST), "r"(VEC_BYTES), "r"(b)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   dst + TILE_BYTES + VEC_BYTES),
               "l"(V + (int64_t)J * ST), "r"(VEC_BYTES), "r"(b)
               : "memory");
}

// 1/sqrt(max(d2, 2^-100)) on the special-function unit. For coincident points
// (d2 = 0) the pair's dx, dy are 0, so its term is 0, as the L^Y definition
// sets it; padding entries carry a zero matrix entry.
__device__ __forceinline__ float rsqrt_clamped(float d2) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(fmaxf(d2, 0x1p-100f)));
  return r;
}
}  // namespace spipe

// A tile of the FP32 pass: view v, tile (I, J) of its kp x kp matrices, the
// view's vector offset / 128, its row-sum slots (2-vectors) and the run slot
// of its column sums (-1 for a diagonal tile).
struct __align__(16) TileRec {
  int32_t v, I, J, vblk;
  int32_t kp, run;
  int64_t part_off;
};

// Run slot r holds, per consumer warp w, that warp's column sums of the run:
// RunPart[(r CWARPS + w) 128 + c], c the column within block J.
template <int MODE>
__global__ void __launch_bounds__(spipe::THREADS, 1)
k_sympass_pipe(int ntile, int npin /* per CTA */, const TileRec *__restrict__ tiles, const CUtensorMap *__restrict__ maps,
               const float2 *__restrict__ V, float2 *__restrict__ Part, float2 *__restrict__ RunPart,
               int *__restrict__ err) {
  using namespace spipe;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[PS], empty[PS];
  __shared__ TileRec srec[PS];  // the record of the tile in each stage, written by the producer
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int first = (int)((int64_t)blockIdx.x * ntile / gridDim.x);
  const int mine = (int)((int64_t)(blockIdx.x + 1) * ntile / gridDim.x) - first;
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;  // TMA destinations 1024-byte aligned
  const unsigned char *sgen = smem_raw + (sbase - smem_u32(smem_raw));
  if (threadIdx.x == 0) {
    for (int s = 0; s < PS; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&empty[s])), "r"(CWARPS));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();  // the only CTA-wide barrier
  // the launch that follows (the reduce) may be scheduled from now on; it
  // waits for this grid's completion itself
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  if (warp == CWARPS) {
    // ---- producer
    if (lane == 0) {
      const CUtensorMap *fenced = nullptr;
      // L2 policies: the first npin tiles of every CTA's chunk stay resident
      // across passes (evict_last), so that each CTA reads the same share
      // from L2; the rest stream through (evict_first)
      uint64_t keep, stream;
      asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(keep));
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(stream));
      // The matrix tiles do not depend on the previous launch: the first PS
      // are requested before waiting for it (expect_tx without the arrival,
      // so the stage cannot complete early); their vector slices, which the
      // previous launch writes, after it.
      const int npre = mine < PS ? mine : PS;
      for (int n = 0; n < npre; ++n) {
        const TileRec t = tiles[first + n];
        const CUtensorMap *map = maps + 2 * t.v + MODE;
        if (map != fenced) {
          asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(map))
                       : "memory");
          fenced = map;
        }
        const uint32_t b = smem_u32(&full[n]);
        asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(b), "r"(TILE_BYTES) : "memory");
        tile_copy(sbase + (uint32_t)n * STAGE_BYTES, b, map, t.I, t.J, n < npin ? keep : stream);
      }
      asm volatile("griddepcontrol.wait;" ::: "memory");
      for (int n = 0; n < npre; ++n) {
        const TileRec t = tiles[first + n];
        const float2 *Vv = V + (int64_t)t.vblk * ST;
        const uint32_t dst = sbase + (uint32_t)n * STAGE_BYTES, b = smem_u32(&full[n]);
        srec[n] = t;  // released to the consumers by the arrive below
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(2 * VEC_BYTES) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         dst + TILE_BYTES),
                     "l"(Vv + (int64_t)t.I * ST), "r"(VEC_BYTES), "r"(b)
                     : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         dst + TILE_BYTES + VEC_BYTES),
                     "l"(Vv + (int64_t)t.J * ST), "r"(VEC_BYTES), "r"(b)
                     : "memory");
      }
      int issued = npre;
      bool ok = true;
      for (int n = npre; n < mine; ++n) {
        const int s = n % PS;
        const TileRec t = tiles[first + n];
        if (!mbar_wait(&empty[s], (uint32_t)(((n - PS) / PS) & 1))) {
          ok = false;
          break;
        }
        srec[s] = t;  // released to the consumers by the arrive below
        issue_tile(sbase + (uint32_t)s * STAGE_BYTES, &full[s], maps + 2 * t.v + MODE, V + (int64_t)t.vblk * ST, t.I,
                   t.J, fenced, n < npin ? keep : stream);
        issued = n + 1;
      }
      if (!ok) {
        atomicOr(err, 1);
        // copies of the last PS issued tiles may still be landing
        for (int n = issued > PS ? issued - PS : 0; n < issued; ++n)
          (void)mbar_wait(&full[n % PS], (uint32_t)((n / PS) & 1));
      }
    }
    return;
  }
  // ---- consumers
  const int rbase = warp * PRW;
  const float sg = MODE == 0 ? -1.0f : 1.0f;
  float2 rxA = make_float2(0.0f, 0.0f), rxB = rxA, ryA = rxA, ryB = rxA;  // column sums of the current run
  int cur_run = -1;
#pragma unroll 1
  for (int n = 0; n < mine; ++n) {
    const int s = n % PS;
    if (!mbar_wait(&full[s], (uint32_t)((n / PS) & 1))) {
      if (lane == 0) atomicOr(err, 1);
      return;
    }
    const TileRec t = srec[s];
    if (t.run != cur_run) {
      if (cur_run >= 0) {
        float4 *o = reinterpret_cast<float4 *>(RunPart + ((int64_t)cur_run * CWARPS + warp) * ST + lane * 4);
        o[0] = make_float4(sg * rxA.x, sg * ryA.x, sg * rxA.y, sg * ryA.y);
        o[1] = make_float4(sg * rxB.x, sg * ryB.x, sg * rxB.y, sg * ryB.y);
      }
      rxA = rxB = ryA = ryB = make_float2(0.0f, 0.0f);
      cur_run = t.run;
    }
    const unsigned char *stage = sgen + (size_t)s * STAGE_BYTES;
    const float *stile = reinterpret_cast<const float *>(stage) + rbase * ST + lane * 4;
    const float2 *svi = reinterpret_cast<const float2 *>(stage + TILE_BYTES) + rbase;
    const float4 *svj = reinterpret_cast<const float4 *>(stage + TILE_BYTES + VEC_BYTES) + lane * 2;
    // columns 4l..4l+3 as pairs A = (4l, 4l+1), B = (4l+2, 4l+3); MODE 0 keeps
    // the column coordinates negated
    const float4 c01 = svj[0], c23 = svj[1];  // (x0, y0, x1, y1), (x2, y2, x3, y3)
    const float2 xA = make_float2(sg * c01.x, sg * c01.z), yA = make_float2(sg * c01.y, sg * c01.w);
    const float2 xB = make_float2(sg * c23.x, sg * c23.z), yB = make_float2(sg * c23.y, sg * c23.w);
    float2 cxA = make_float2(0.0f, 0.0f), cxB = cxA, cyA = cxA, cyB = cxA;
    float acc[2 * PRW];
#pragma unroll
    for (int r = 0; r < PRW; ++r) {
      const float4 m4 = *reinterpret_cast<const float4 *>(stile + r * ST);
      const float2 vi = svi[r];
      const float2 mA = make_float2(m4.x, m4.y), mB = make_float2(m4.z, m4.w);
      const float2 vx = make_float2(vi.x, vi.x), vy = make_float2(vi.y, vi.y);
      float2 ra, rb;
      if (MODE == 0) {
        const float2 dxA = __fadd2_rn(vx, xA), dyA = __fadd2_rn(vy, yA);
        const float2 dxB = __fadd2_rn(vx, xB), dyB = __fadd2_rn(vy, yB);
        const float2 qA = __ffma2_rn(dyA, dyA, __fmul2_rn(dxA, dxA));
        const float2 qB = __ffma2_rn(dyB, dyB, __fmul2_rn(dxB, dxB));
        const float2 kA = __fmul2_rn(mA, make_float2(rsqrt_clamped(qA.x), rsqrt_clamped(qA.y)));
        const float2 kB = __fmul2_rn(mB, make_float2(rsqrt_clamped(qB.x), rsqrt_clamped(qB.y)));
        ra = __ffma2_rn(kB, dxB, __fmul2_rn(kA, dxA));
        rb = __ffma2_rn(kB, dyB, __fmul2_rn(kA, dyA));
        cxA = __ffma2_rn(kA, dxA, cxA);  // sums of +t; negated when stored
        cxB = __ffma2_rn(kB, dxB, cxB);
        cyA = __ffma2_rn(kA, dyA, cyA);
        cyB = __ffma2_rn(kB, dyB, cyB);
      } else {
        ra = __ffma2_rn(mB, xB, __fmul2_rn(mA, xA));
        rb = __ffma2_rn(mB, yB, __fmul2_rn(mA, yA));
        cxA = __ffma2_rn(mA, vx, cxA);
        cxB = __ffma2_rn(mB, vx, cxB);
        cyA = __ffma2_rn(mA, vy, cyA);
        cyB = __ffma2_rn(mB, vy, cyB);
      }
      acc[2 * r] = ra.x + ra.y;
      acc[2 * r + 1] = rb.x + rb.y;
    }
    // every lane's reads of stage s (and of srec[s]) are done (their values
    // are in use above)
    __syncwarp();
    if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    if (t.run >= 0) {
      rxA = __fadd2_rn(rxA, cxA);
      rxB = __fadd2_rn(rxB, cxB);
      ryA = __fadd2_rn(ryA, cyA);
      ryB = __fadd2_rn(ryB, cyB);
    }
    const float tot = lanes_transpose_sum<2 * PRW, float>(acc, lane);
    constexpr int REP = 32 / (2 * PRW);
    if (lane % REP == 0) {
      const int idx = lane / REP;
      float *part = reinterpret_cast<float *>(Part + t.part_off);
      part[((int64_t)t.J * t.kp + (int64_t)t.I * ST + rbase + (idx >> 1)) * 2 + (idx & 1)] = tot;
    }
  }
  if (cur_run >= 0) {
    float4 *o = reinterpret_cast<float4 *>(RunPart + ((int64_t)cur_run * CWARPS + warp) * ST + lane * 4);
    o[0] = make_float4(sg * rxA.x, sg * ryA.x, sg * rxA.y, sg * ryA.y);
    o[1] = make_float4(sg * rxB.x, sg * ryB.x, sg * rxB.y, sg * ryB.y);
  }
}

// Row block R of view v, (v, R) = blocks[blockIdx.x]:
//   Vout[R 128 + row] = sum_{J = R}^{nbt - 1} Part[J][R 128 + row]        (row sums of tiles (R, J))
//                     + sum over the runs of column block R and their warps
//                       of RunPart[(r CWARPS + w) 128 + row]                (column sums of tiles (I < R, R))
// The items are numbered in that order; thread (g, row) adds items g, g + 8,
// ... in order, then the eight group sums are added in order (a fixed order:
// the same result on every run).
__global__ void __launch_bounds__(1024)
k_reduce_rows(const int2 *__restrict__ blocks, const BatchView *__restrict__ views, const int *__restrict__ run_ptr,
              const int *__restrict__ run_idx, const float2 *__restrict__ Part, const float2 *__restrict__ RunPart,
              float2 *__restrict__ Vout) {
  constexpr int NG = 8, UN = 10;
  __shared__ float2 red[NG][ST];
  // launched as a programmatic dependent of the pass: wait for it to complete
  // (its partial sums visible); the next pass may be scheduled meanwhile
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int2 b = blocks[blockIdx.x];
  const BatchView bv = views[b.x];
  const int row = threadIdx.x & (ST - 1), g = threadIdx.x >> 7;
  const int64_t r = (int64_t)b.y * ST + row;
  const int nrow = bv.nbt - b.y;
  const int r0 = run_ptr[blockIdx.x], nitem = nrow + (run_ptr[blockIdx.x + 1] - r0) * spipe::CWARPS;
  float2 acc = make_float2(0.0f, 0.0f);
#pragma unroll 1
  for (int i0 = g; i0 < nitem; i0 += NG * UN) {
    float2 u[UN];
#pragma unroll
    for (int e = 0; e < UN; ++e) {
      const int i = i0 + NG * e;
      if (i < nrow) {
        u[e] = __ldcg(Part + bv.part_off + (int64_t)(b.y + i) * bv.kp + r);
      } else if (i < nitem) {
        const int q = i - nrow;
        const int run = run_idx[r0 + q / spipe::CWARPS];
        u[e] = __ldcg(RunPart + ((int64_t)run * spipe::CWARPS + q % spipe::CWARPS) * ST + row);
      }
    }
#pragma unroll
    for (int e = 0; e < UN; ++e)
      if (i0 + NG * e < nitem) {
        acc.x += u[e].x;
        acc.y += u[e].y;
      }
  }
  red[g][row] = acc;
  __syncthreads();
  if (threadIdx.x < ST) {
    float2 v = red[0][row];
#pragma unroll
    for (int e = 1; e < NG; ++e) {
      v.x += red[e][row].x;
      v.y += red[e][row].y;
    }
    Vout[bv.vec_off + r] = v;
  }
}

// X (kp x 2) = x0 for rows < k, zero on the padding.
template <typename TI, typename T>
__global__ void k_load_x(int32_t k, int32_t kp, const TI *__restrict__ x, typename T2<T>::type *__restrict__ X) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kp) return;
  typename T2<T>::type v;
  v.x = i < k ? (T)x[2 * i] : T(0);
  v.y = i < k ? (T)x[2 * i + 1] : T(0);
  X[i] = v;
}

// Centre X (FP64 mean, one block, fixed order) and convert to the output type.
template <typename T, typename TO>
__global__ void k_finish(int32_t k, const typename T2<T>::type *__restrict__ X, TO *__restrict__ out,
                         typename T2<T>::type *__restrict__ Xc) {
  __shared__ double sx[1024], sy[1024];
  double mx = 0.0, my = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    mx += (double)X[i].x;
    my += (double)X[i].y;
  }
  sx[threadIdx.x] = mx;
  sy[threadIdx.x] = my;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sx[threadIdx.x] += sx[threadIdx.x + o];
      sy[threadIdx.x] += sy[threadIdx.x + o];
    }
    __syncthreads();
  }
  const double ax = sx[0] / k, ay = sy[0] / k;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    const T cx = (T)((double)X[i].x - ax), cy = (T)((double)X[i].y - ay);
    out[2 * i] = (TO)cx;
    out[2 * i + 1] = (TO)cy;
    if (Xc) {
      typename T2<T>::type w;
      w.x = cx;
      w.y = cy;
      Xc[i] = w;
    }
  }
}

// ---------------------------------------------------------------------------
// Energy and gradients by pair recomputation. Per pair i != j with
// d = |x_i - x_j|, u = 1/Delta_ij, e = 1 - d u:
//   energy += e^2 (halved at the end: Eq. (7) sums i < j)
//   grad_x_i += -2 e u / d (x_i - x_j)      (0 when d = 0)
//   grad_pdist_ij = e d u^2
// Each block writes its FP64 energy partial; k_reduce_energy adds them in order.
// ---------------------------------------------------------------------------
template <typename T, bool GX, bool GD>
__global__ void __launch_bounds__(LWARPS * 32)
k_energy(int32_t k, const T *__restrict__ Delta, const typename T2<T>::type *__restrict__ X, T scale,
         double *__restrict__ eparts, T *__restrict__ gx, T *__restrict__ gD, int *__restrict__ flag) {
  using V2 = typename T2<T>::type;
  __shared__ V2 sv[XCH];
  __shared__ double se[LWARPS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t rows[RPW];
  T xi[RPW], yi[RPW], gxx[RPW], gxy[RPW];
  double eacc = 0.0;
  int bad = 0;
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    rows[r] = ((int64_t)blockIdx.x * LWARPS + warp) * RPW + r;
    gxx[r] = T(0);
    gxy[r] = T(0);
    xi[r] = T(0);
    yi[r] = T(0);
    if (rows[r] < k) {
      xi[r] = X[rows[r]].x;
      yi[r] = X[rows[r]].y;
    }
  }
  for (int64_t c0 = 0; c0 < k; c0 += XCH) {
    const int cn = (int)min((int64_t)XCH, (int64_t)k - c0);
    __syncthreads();
    for (int t = threadIdx.x; t < cn; t += blockDim.x) sv[t] = X[c0 + t];
    __syncthreads();
    for (int t = lane; t < cn; t += 32) {
      const V2 xj = sv[t];
      const int64_t j = c0 + t;
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        const int64_t i = rows[r];
        if (i >= k) continue;
        if (i == j) {
          if (GD) gD[i * k + j] = T(0);
          continue;
        }
        const T del = Delta[i * k + j];
        if (!(del > T(0))) bad = 1;
        const T dx = xi[r] - xj.x, dy = yi[r] - xj.y;
        const T d = sqrt(dx * dx + dy * dy);
        const T u = T(1) / del;
        const T e = T(1) - d * u;
        eacc += (double)(e * e);
        if (GX && d > T(0)) {
          const T coef = T(-2) * e * u / d;
          gxx[r] += coef * dx;
          gxy[r] += coef * dy;
        }
        if (GD) gD[i * k + j] = scale * e * d * u * u;
      }
    }
  }
  if (GX) {
#pragma unroll
    for (int r = 0; r < RPW; ++r) {
      T vx = gxx[r], vy = gxy[r];
      for (int o = 16; o > 0; o >>= 1) {
        vx += __shfl_xor_sync(0xffffffffu, vx, o);
        vy += __shfl_xor_sync(0xffffffffu, vy, o);
      }
      if (lane == 0 && rows[r] < k) {
        gx[2 * rows[r]] = scale * vx;
        gx[2 * rows[r] + 1] = scale * vy;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
  if (lane == 0) se[warp] = eacc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < LWARPS; ++w) s += se[w];
    eparts[blockIdx.x] = s;
  }
  if (bad) atomicOr(flag, 1);
}

__global__ void k_reduce_energy(int nparts, const double *__restrict__ eparts, double *__restrict__ out) {
  __shared__ double s[256];
  double a = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) a += eparts[i];
  s[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) s[threadIdx.x] += s[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 0.5 * s[0];
}

template <typename TI, typename T>
__global__ void k_convert(int64_t cnt, const TI *__restrict__ in, T *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < cnt) out[i] = (T)in[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// Grid and shared-memory setup of the pipelined FP32 pass: one CTA per SM
// (fewer when the table is shorter).
int sympass_pipe_grid(pprviz_ctx *ctx, size_t ntile, unsigned *grid) {
  int nsm = 0;
  PPRVIZ_CUDA(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_sympass_pipe<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, spipe::SMEM));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_sympass_pipe<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, spipe::SMEM));
  *grid = (unsigned)std::min<size_t>(ntile, (size_t)std::max(nsm, 1));
  return PPRVIZ_OK;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (the
// library links only the runtime).
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The kp x kp row-major FP32 matrix at base as a 2-D tensor with 128 x 128
// boxes, no swizzle (a box lands row-major in shared memory).
int tile_map(pprviz_ctx *ctx, const float *base, int32_t kp, CUtensorMap *out) {
  static EncodeTiledFn encode = nullptr;
  if (!encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
      return set_err(ctx, PPRVIZ_E_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)kp};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)ST, (cuuint32_t)ST};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_err(ctx, PPRVIZ_E_CUDA, "cuTensorMapEncodeTiled failed for a layout matrix");
  return PPRVIZ_OK;
}

// Tables of the pipelined FP32 pass for a grid of G CTAs (device slots
// WS_TREC, WS_TROWS):
//  * tile records of every view's upper-triangle tiles, view by view, column
//    by column (J, then I = 0..J), with the run slot of each off-diagonal
//    tile: consecutive tiles of one column block in one CTA's chunk
//    [b ntile / G, (b + 1) ntile / G) share a run;
//  * the (view, row block) pairs, one per k_reduce_rows block (view order,
//    then R), and for each the runs of column block R (CSR: run_ptr, run_idx).
struct PassTables {
  const TileRec *recs = nullptr;
  int ntile = 0;
  const int2 *blocks = nullptr;
  const int *run_ptr = nullptr, *run_idx = nullptr;
  int nblocks = 0, nruns = 0;
};

int upload_pass_tables(pprviz_ctx *ctx, const std::vector<BatchView> &bv, unsigned G, PassTables *pt) {
  std::vector<TileRec> rec;
  std::vector<int> rb_base(bv.size());
  int nrb = 0;
  for (size_t v = 0; v < bv.size(); ++v) {
    rb_base[v] = nrb;
    nrb += bv[v].nbt;
    for (int J = 0; J < bv[v].nbt; ++J)
      for (int I = 0; I <= J; ++I)
        rec.push_back(TileRec{(int32_t)v, I, J, (int32_t)(bv[v].vec_off / ST), bv[v].kp, -1, bv[v].part_off});
  }
  const int64_t ntile = (int64_t)rec.size();
  if (ntile >= INT32_MAX) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "too many layout tiles");
  std::vector<std::vector<int>> runs_of(nrb);
  int nruns = 0, cur = -1, prev_v = -1, prev_J = -1;
  int64_t b = 0;  // CTA of position p: first(b) <= p < first(b + 1)
  for (int64_t p = 0; p < ntile; ++p) {
    while (b + 1 < (int64_t)G && (b + 1) * ntile / G <= p) ++b;
    TileRec &r = rec[p];
    const bool chunk_start = (b * ntile / G) == p;
    if (r.I == r.J) {  // diagonal: its column sums are not taken
      cur = -1;
      continue;
    }
    if (cur < 0 || chunk_start || r.v != prev_v || r.J != prev_J) {
      cur = nruns++;
      runs_of[rb_base[r.v] + r.J].push_back(cur);
    }
    r.run = cur;
    prev_v = r.v;
    prev_J = r.J;
  }
  std::vector<int2> blocks;
  std::vector<int> run_ptr(1, 0), run_idx;
  for (size_t v = 0; v < bv.size(); ++v)
    for (int R = 0; R < bv[v].nbt; ++R) {
      blocks.push_back(make_int2((int)v, R));
      for (int q : runs_of[rb_base[v] + R]) run_idx.push_back(q);
      run_ptr.push_back((int)run_idx.size());
    }
  if (run_idx.empty()) run_idx.push_back(0);  // keep the device pointer valid
  const size_t o_blocks = 0, o_ptr = (sizeof(int2) * blocks.size() + 255) & ~(size_t)255;
  const size_t o_idx = (o_ptr + sizeof(int) * run_ptr.size() + 255) & ~(size_t)255;
  const size_t bytes = o_idx + sizeof(int) * run_idx.size();
  PPRVIZ_TRY(ws_ensure(ctx, WS_TREC, sizeof(TileRec) * rec.size()));
  PPRVIZ_TRY(ws_ensure(ctx, WS_TROWS, bytes));
  unsigned char *d = static_cast<unsigned char *>(ctx->ws[WS_TROWS].p);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(ctx->ws[WS_TREC].p, rec.data(), sizeof(TileRec) * rec.size(),
                                   cudaMemcpyHostToDevice, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(d + o_blocks, blocks.data(), sizeof(int2) * blocks.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(d + o_ptr, run_ptr.data(), sizeof(int) * run_ptr.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(d + o_idx, run_idx.data(), sizeof(int) * run_idx.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the host vectors are released on return
  pt->recs = ctx->ws[WS_TREC].as<TileRec>();
  pt->ntile = (int)ntile;
  pt->blocks = reinterpret_cast<const int2 *>(d + o_blocks);
  pt->run_ptr = reinterpret_cast<const int *>(d + o_ptr);
  pt->run_idx = reinterpret_cast<const int *>(d + o_idx);
  pt->nblocks = (int)blocks.size();
  pt->nruns = nruns;
  return PPRVIZ_OK;
}

// One layout update of all views in the tables: L^Y pass over W1 from X into
// Bv, apply pass over M from Bv into X, each followed by its reduce.
// Launch on the context stream as a programmatic dependent of the previous
// launch (the kernel itself waits for it with griddepcontrol.wait), so that
// its blocks are scheduled, and the pass requests its first tiles, while the
// previous launch finishes.
template <typename... P, typename... A>
cudaError_t launch_dependent(pprviz_ctx *ctx, void (*kernel)(P...), unsigned grid, unsigned block, size_t smem,
                             A... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = ctx->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// L2 bytes of each pass matrix kept resident across updates (evict_last):
// the two matrices together stay well inside the 126 MB L2 next to the
// partial sums and coordinates; the rest of each matrix streams from HBM
constexpr double kPinBytes = 32.0 * 1024 * 1024;

int pass_pair(pprviz_ctx *ctx, unsigned grid, const PassTables &pt, const CUtensorMap *maps, const BatchView *views_d,
              float2 *X, float2 *Bv, float2 *Part, float2 *RunPart, int *perr) {
  const unsigned nb = (unsigned)pt.nblocks;
  const int npin = (int)(kPinBytes / spipe::TILE_BYTES / grid);  // tiles per CTA
  { PPRVIZ_PROF(ctx, PPRVIZ_K_LY); PPRVIZ_CUDA(ctx, launch_dependent(ctx, k_sympass_pipe<0>, grid, spipe::THREADS, spipe::SMEM, pt.ntile, npin, pt.recs, maps, (const float2 *)X, Part, RunPart, perr)); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); PPRVIZ_CUDA(ctx, launch_dependent(ctx, k_reduce_rows, nb, 1024, 0, pt.blocks, views_d, pt.run_ptr, pt.run_idx, (const float2 *)Part, (const float2 *)RunPart, Bv)); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_APPLY); PPRVIZ_CUDA(ctx, launch_dependent(ctx, k_sympass_pipe<1>, grid, spipe::THREADS, spipe::SMEM, pt.ntile, npin, pt.recs, maps, (const float2 *)Bv, Part, RunPart, perr)); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); PPRVIZ_CUDA(ctx, launch_dependent(ctx, k_reduce_rows, nb, 1024, 0, pt.blocks, views_d, pt.run_ptr, pt.run_idx, (const float2 *)Part, (const float2 *)RunPart, X)); }
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

// Tensor maps of the two pass matrices of every view (maps[2 v] = 1/Delta_s,
// maps[2 v + 1] = M) into the device slot WS_TMAP.
int upload_maps(pprviz_ctx *ctx, const std::vector<BatchView> &bv, const float *W1, const float *M,
                const CUtensorMap **maps_d) {
  std::vector<CUtensorMap> maps(2 * bv.size());
  for (size_t v = 0; v < bv.size(); ++v) {
    PPRVIZ_TRY(tile_map(ctx, W1 + bv[v].mat_off, bv[v].kp, &maps[2 * v]));
    PPRVIZ_TRY(tile_map(ctx, M + bv[v].mat_off, bv[v].kp, &maps[2 * v + 1]));
  }
  PPRVIZ_TRY(ws_ensure(ctx, WS_TMAP, sizeof(CUtensorMap) * maps.size()));
  CUtensorMap *d = reinterpret_cast<CUtensorMap *>(ctx->ws[WS_TMAP].p);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(d, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  // the host vector is released on return: wait for the copy
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  *maps_d = d;
  return PPRVIZ_OK;
}

template <typename T, typename TI, typename TO>
int layout_typed(pprviz_ctx *ctx, const TI *pdist, int32_t k, const TI *x0, int32_t iters, TO *x_out,
                 double *stress_h) {
  using V2 = typename T2<T>::type;
  const int32_t kp = (k + ST - 1) / ST * ST;  // whole symmetric tiles (and NB pivot blocks)
  const int nbt = kp / ST;
  PPRVIZ_TRY(ws_ensure(ctx, WS_W1, sizeof(T) * (size_t)kp * kp));
  PPRVIZ_TRY(ws_ensure(ctx, WS_M, sizeof(T) * (size_t)kp * kp));
  PPRVIZ_TRY(ws_ensure(ctx, WS_PIV, sizeof(T) * spd_inverse_work(kp)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_X, sizeof(V2) * (size_t)kp * 2));            // X and b
  PPRVIZ_TRY(ws_ensure(ctx, WS_B, sizeof(V2) * (size_t)nbt * kp));          // partial sums
  PPRVIZ_TRY(ws_ensure(ctx, WS_E, sizeof(V2) * (size_t)k + 64));
  PPRVIZ_TRY(ws_ensure(ctx, WS_RHS, sizeof(double) * (size_t)(kp / 32) * kp));  // build row partials
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  T *W1 = ctx->ws[WS_W1].as<T>(), *A = ctx->ws[WS_M].as<T>();
  T *work = ctx->ws[WS_PIV].as<T>();
  V2 *X = ctx->ws[WS_X].as<V2>(), *Bv = X + kp, *Part = ctx->ws[WS_B].as<V2>();
  double *rowpart = ctx->ws[WS_RHS].as<double>();
  int *flag = ctx->ws[WS_FLAG].as<int>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_build_sym<TI, T><<<dim3(kp / 32, kp / 32), dim3(32, 8), 0, ctx->stream>>>(k, kp, pdist, W1, A, rowpart, flag); }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_build_diag<T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(k, kp, rowpart, A); }
  PPRVIZ_LAUNCHED(ctx);
  int hf = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hf) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "pdist has a non-finite or non-positive off-diagonal entry");
  if (iters > 0) {
    if constexpr (std::is_same<T, float>::value) PPRVIZ_TRY(spd_inverse_f32(ctx, kp, A, work));
    else PPRVIZ_TRY(spd_inverse_f64(ctx, kp, A, work));
  }
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_load_x<TI, T><<<(unsigned)((kp + 255) / 256), 256, 0, ctx->stream>>>(k, kp, x0, X); }
  PPRVIZ_LAUNCHED(ctx);
  // one view descriptor, the upper tile triangle in row order, and the
  // row-block counters of the fused reduce (zero between passes)
  std::vector<int4> tiles;
  for (int I = 0; I < nbt; ++I)
    for (int J = I; J < nbt; ++J) tiles.push_back(make_int4(0, I, J, 0));  // w: vec_off / 128 = 0
  const BatchView one{0, 0, 0, kp, nbt, k, 0};
  const size_t tab_off = 256, cnt_off = (tab_off + sizeof(int4) * tiles.size() + 255) & ~(size_t)255;
  PPRVIZ_TRY(ws_ensure(ctx, WS_BTAB, cnt_off + sizeof(int) * (size_t)nbt));
  BatchView *view_d = reinterpret_cast<BatchView *>(ctx->ws[WS_BTAB].p);
  int4 *tiles_d = reinterpret_cast<int4 *>(static_cast<unsigned char *>(ctx->ws[WS_BTAB].p) + tab_off);
  int *cnt = reinterpret_cast<int *>(static_cast<unsigned char *>(ctx->ws[WS_BTAB].p) + cnt_off);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(view_d, &one, sizeof(BatchView), cudaMemcpyHostToDevice, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(tiles_d, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)nbt, ctx->stream));
  const unsigned ntile = (unsigned)tiles.size();
  if constexpr (std::is_same<T, float>::value) {
    unsigned pgrid = 0;
    PPRVIZ_TRY(sympass_pipe_grid(ctx, tiles.size(), &pgrid));
    const std::vector<BatchView> one_v{one};
    const CUtensorMap *maps = nullptr;
    PPRVIZ_TRY(upload_maps(ctx, one_v, W1, A, &maps));
    PassTables pt;
    PPRVIZ_TRY(upload_pass_tables(ctx, one_v, pgrid, &pt));
    PPRVIZ_TRY(ws_ensure(ctx, WS_RUNP, sizeof(V2) * ((size_t)pt.nruns * spipe::CWARPS * ST + 1)));
    V2 *RunPart = ctx->ws[WS_RUNP].as<V2>();
    int *perr = flag + 1;
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(perr, 0, sizeof(int), ctx->stream));
    for (int it = 0; it < iters; ++it) PPRVIZ_TRY(pass_pair(ctx, pgrid, pt, maps, view_d, X, Bv, Part, RunPart, perr));
    if (iters > 0) {
      int herr = 0;
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, perr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "layout pass: tile copy wait expired");
    }
  } else {
    for (int it = 0; it < iters; ++it) {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_LY); k_sympass_batch<T, 0><<<ntile, 256, 0, ctx->stream>>>(tiles_d, view_d, W1, X, Part, cnt, Bv); }
      PPRVIZ_LAUNCHED(ctx);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_APPLY); k_sympass_batch<T, 1><<<ntile, 256, 0, ctx->stream>>>(tiles_d, view_d, A, Bv, Part, cnt, X); }
      PPRVIZ_LAUNCHED(ctx);
    }
  }
  V2 *Xc = ctx->ws[WS_E].as<V2>();
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_finish<T, TO><<<1, 1024, 0, ctx->stream>>>(k, X, x_out, Xc); }
  PPRVIZ_LAUNCHED(ctx);
  ctx->stats.layout_iters = iters;
  // algorithmic bytes: each pass reads the upper triangle of one k x k matrix
  const double half = 0.5 * (double)k * ((double)k + 1.0) * sizeof(T);
  ctx->stats.bytes_ly = half * iters;
  ctx->stats.bytes_apply = half * iters;
  if (stress_h) {
    const unsigned eb = (unsigned)((k + LWARPS * RPW - 1) / (LWARPS * RPW));
    PPRVIZ_TRY(ws_ensure(ctx, WS_OUT1, sizeof(double) * (eb + 1)));
    double *ep = ctx->ws[WS_OUT1].as<double>();
    // stress of the final layout on the input pdist (Eq. (7)), in the path's arithmetic
    const T *Dt = (const T *)pdist;
    if (!std::is_same<T, TI>::value) {
      T *Dw = W1;  // k*k fits in the kp*kp 1/Delta buffer, which is no longer needed
      const int64_t cnt = (int64_t)k * k;
      { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_convert<TI, T><<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(cnt, pdist, Dw); }
      PPRVIZ_LAUNCHED(ctx);
      Dt = Dw;
    }
    { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<T, false, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, Dt, Xc, T(1), ep, nullptr, nullptr, flag); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_reduce_energy<<<1, 256, 0, ctx->stream>>>((int)eb, ep, ep + eb); }
    PPRVIZ_LAUNCHED(ctx);
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(stress_h, ep + eb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return PPRVIZ_OK;
}

}  // namespace

int layout_run(pprviz_ctx *ctx, const void *pdist_d, int32_t k, const void *x0_d, int32_t iters,
               int precision, bool io64, void *x_out_d, double *stress_h) {
  if (precision == PPRVIZ_FP64) {
    if (io64)
      return layout_typed<double, double, double>(ctx, (const double *)pdist_d, k, (const double *)x0_d, iters,
                                                  (double *)x_out_d, stress_h);
    return layout_typed<double, float, float>(ctx, (const float *)pdist_d, k, (const float *)x0_d, iters,
                                              (float *)x_out_d, stress_h);
  }
  if (io64)
    return layout_typed<float, double, double>(ctx, (const double *)pdist_d, k, (const double *)x0_d, iters,
                                               (double *)x_out_d, stress_h);
  return layout_typed<float, float, float>(ctx, (const float *)pdist_d, k, (const float *)x0_d, iters,
                                           (float *)x_out_d, stress_h);
}

// Many views, FP32: each view's 1/Delta_s and (L^w + J/k)^-1 are built and
// inverted into slices of two batched matrices, then every update runs as two
// launches over all views together (L^Y pass, apply pass, each with its fused
// partial-sum reduce).
int layout_batch_run(pprviz_ctx *ctx, int32_t nviews, const int64_t *k_h, const float *pdist_d,
                     const float *x0_d, int32_t iters, float *x_out_d, double *stress_h) {
  using V2 = float2;
  std::vector<BatchView> bv((size_t)nviews);
  std::vector<int4> tiles;
  int64_t mat = 0, vec = 0, part = 0, maxkp = 0;
  int32_t cnts = 0;
  for (int32_t v = 0; v < nviews; ++v) {
    const int32_t k = (int32_t)k_h[v];
    const int32_t kp = (k + ST - 1) / ST * ST, nbt = kp / ST;
    bv[v] = BatchView{mat, vec, part, kp, nbt, k, cnts};
    mat += (int64_t)kp * kp;
    vec += kp;
    part += (int64_t)nbt * kp;
    cnts += nbt;
    maxkp = std::max<int64_t>(maxkp, kp);
    for (int I = 0; I < nbt; ++I)
      for (int J = I; J < nbt; ++J) tiles.push_back(make_int4(v, I, J, (int)(bv[v].vec_off / ST)));
  }
  PPRVIZ_TRY(ws_ensure(ctx, WS_BW1, sizeof(float) * (size_t)mat));
  PPRVIZ_TRY(ws_ensure(ctx, WS_BM, sizeof(float) * (size_t)mat));
  PPRVIZ_TRY(ws_ensure(ctx, WS_BX, sizeof(V2) * (size_t)vec * 2));
  PPRVIZ_TRY(ws_ensure(ctx, WS_BPART, sizeof(V2) * (size_t)part));
  // the tile table (int4, 16-byte loads) starts at a 256-byte boundary after the
  // descriptors, the row-block counters at the next one after the table
  const size_t tab_off = (sizeof(BatchView) * (size_t)nviews + 255) & ~(size_t)255;
  const size_t cnt_off = (tab_off + sizeof(int4) * tiles.size() + 255) & ~(size_t)255;
  PPRVIZ_TRY(ws_ensure(ctx, WS_BTAB, cnt_off + sizeof(int) * (size_t)cnts));
  PPRVIZ_TRY(ws_ensure(ctx, WS_RHS, sizeof(double) * (size_t)(maxkp / 32) * maxkp));
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  float *W1 = ctx->ws[WS_BW1].as<float>(), *M = ctx->ws[WS_BM].as<float>();
  V2 *X = ctx->ws[WS_BX].as<V2>(), *Bv = X + vec, *Part = ctx->ws[WS_BPART].as<V2>();
  BatchView *views_d = reinterpret_cast<BatchView *>(ctx->ws[WS_BTAB].p);
  int4 *tiles_d = reinterpret_cast<int4 *>(static_cast<unsigned char *>(ctx->ws[WS_BTAB].p) + tab_off);
  int *cnt = reinterpret_cast<int *>(static_cast<unsigned char *>(ctx->ws[WS_BTAB].p) + cnt_off);
  double *rowpart = ctx->ws[WS_RHS].as<double>();
  int *flag = ctx->ws[WS_FLAG].as<int>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)cnts, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(views_d, bv.data(), sizeof(BatchView) * bv.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(tiles_d, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  int64_t sq = 0, xo = 0;
  std::vector<int32_t> kps((size_t)nviews);
  std::vector<float *> mats((size_t)nviews);
  for (int32_t v = 0; v < nviews; ++v) {
    const int32_t k = bv[v].k, kp = bv[v].kp;
    const float *Dv = pdist_d + sq;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_build_sym<float, float><<<dim3(kp / 32, kp / 32), dim3(32, 8), 0, ctx->stream>>>(k, kp, Dv, W1 + bv[v].mat_off, M + bv[v].mat_off, rowpart, flag); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_build_diag<float><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(k, kp, rowpart, M + bv[v].mat_off); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_load_x<float, float><<<(unsigned)((kp + 255) / 256), 256, 0, ctx->stream>>>(k, kp, x0_d + 2 * xo, X + bv[v].vec_off); }
    PPRVIZ_LAUNCHED(ctx);
    kps[v] = kp;
    mats[v] = M + bv[v].mat_off;
    sq += (int64_t)k * k;
    xo += k;
  }
  // every view's (L^w + J/k)^-1 together, pivot step by pivot step
  if (iters > 0) {
    PPRVIZ_TRY(ws_ensure(ctx, WS_FACB, sizeof(float) * spd_inverse_batch_work(nviews, kps.data())));
    PPRVIZ_TRY(spd_inverse_batch_f32(ctx, nviews, kps.data(), mats.data(), ctx->ws[WS_FACB].as<float>()));
  }
  int hf = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hf) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "a view's pdist has a non-finite or non-positive entry");
  const unsigned ntile = (unsigned)tiles.size();
  unsigned pgrid = 0;
  PPRVIZ_TRY(sympass_pipe_grid(ctx, tiles.size(), &pgrid));
  const CUtensorMap *maps = nullptr;
  PPRVIZ_TRY(upload_maps(ctx, bv, W1, M, &maps));
  PassTables pt;
  PPRVIZ_TRY(upload_pass_tables(ctx, bv, pgrid, &pt));
  PPRVIZ_TRY(ws_ensure(ctx, WS_RUNP, sizeof(V2) * ((size_t)pt.nruns * spipe::CWARPS * ST + 1)));
  V2 *RunPart = ctx->ws[WS_RUNP].as<V2>();
  int *perr = flag + 1;
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(perr, 0, sizeof(int), ctx->stream));
  // The updates of a batch are launches only (no host decision between them):
  // they are recorded once into a CUDA graph and the graph is launched. With
  // kernel timing on, or if recording or instantiating fails, the same
  // launches go to the stream directly (timing events mark points of the
  // stream, which a recorded graph does not have).
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  bool graphed = false;
  if (iters > 1 && !ctx->profiling && cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed) == cudaSuccess) {
    int st = PPRVIZ_OK;
    ctx->capturing = true;
    for (int it = 0; it < iters && st == PPRVIZ_OK; ++it)
      st = pass_pair(ctx, pgrid, pt, maps, views_d, X, Bv, Part, RunPart, perr);
    ctx->capturing = false;
    const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
    if (st == PPRVIZ_OK && ec == cudaSuccess && graph && cudaGraphInstantiate(&gexec, graph, 0) == cudaSuccess &&
        cudaGraphLaunch(gexec, ctx->stream) == cudaSuccess)
      graphed = true;
    if (!graphed) {
      cudaGetLastError();
      ctx->err.clear();
      if (gexec) cudaGraphExecDestroy(gexec);
      if (graph) cudaGraphDestroy(graph);
      gexec = nullptr;
      graph = nullptr;
    }
  } else {
    cudaGetLastError();
  }
  ctx->stats.graph_launched = graphed ? 1 : 0;
  if (!graphed)
    for (int it = 0; it < iters; ++it) PPRVIZ_TRY(pass_pair(ctx, pgrid, pt, maps, views_d, X, Bv, Part, RunPart, perr));
  if (graphed) {
    // the graph has run before the objects go (the wait below is the call's own)
    const cudaError_t es = cudaStreamSynchronize(ctx->stream);
    cudaGraphExecDestroy(gexec);
    cudaGraphDestroy(graph);
    if (es != cudaSuccess) return cuda_err(ctx, es, "layout updates (CUDA graph)");
  }
  if (iters > 0) {
    int herr = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, perr, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "layout pass: tile copy wait expired");
  }
  ctx->stats.layout_iters = iters;
  double half = 0.0;
  for (int32_t v = 0; v < nviews; ++v) half += 0.5 * (double)bv[v].k * ((double)bv[v].k + 1.0) * sizeof(float);
  ctx->stats.bytes_ly = half * iters;
  ctx->stats.bytes_apply = half * iters;
  // centre and emit each view; stress per view on its input pdist
  int64_t maxk = 0;
  for (int32_t v = 0; v < nviews; ++v) maxk = std::max<int64_t>(maxk, bv[v].k);
  const unsigned eb_max = (unsigned)((maxk + LWARPS * RPW - 1) / (LWARPS * RPW));
  PPRVIZ_TRY(ws_ensure(ctx, WS_E, sizeof(V2) * (size_t)maxk + 64));
  PPRVIZ_TRY(ws_ensure(ctx, WS_OUT1, sizeof(double) * ((size_t)eb_max + 1) * nviews));
  V2 *Xc = ctx->ws[WS_E].as<V2>();
  double *ep = ctx->ws[WS_OUT1].as<double>();
  sq = 0;
  xo = 0;
  for (int32_t v = 0; v < nviews; ++v) {
    const int32_t k = bv[v].k;
    const unsigned eb = (unsigned)((k + LWARPS * RPW - 1) / (LWARPS * RPW));
    double *epv = ep + (size_t)v * (eb_max + 1);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_finish<float, float><<<1, 1024, 0, ctx->stream>>>(k, X + bv[v].vec_off, x_out_d + 2 * xo, Xc); }
    PPRVIZ_LAUNCHED(ctx);
    if (stress_h) {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<float, false, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist_d + sq, Xc, 1.0f, epv, nullptr, nullptr, flag); }
      PPRVIZ_LAUNCHED(ctx);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_reduce_energy<<<1, 256, 0, ctx->stream>>>((int)eb, epv, epv + eb_max); }
      PPRVIZ_LAUNCHED(ctx);
    }
    sq += (int64_t)k * k;
    xo += k;
  }
  if (stress_h) {
    std::vector<double> eh((size_t)(eb_max + 1) * nviews);
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(eh.data(), ep, sizeof(double) * eh.size(), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int32_t v = 0; v < nviews; ++v) stress_h[v] = eh[(size_t)v * (eb_max + 1) + eb_max];
  }
  return PPRVIZ_OK;
}

template <typename T>
static int energy_typed(pprviz_ctx *ctx, const T *pdist, int32_t k, const T *x, double scale, double *e_h,
                        T *gx, T *gD) {
  using V2 = typename T2<T>::type;
  const unsigned eb = (unsigned)((k + LWARPS * RPW - 1) / (LWARPS * RPW));
  PPRVIZ_TRY(ws_ensure(ctx, WS_E, sizeof(V2) * (size_t)k + 64));
  PPRVIZ_TRY(ws_ensure(ctx, WS_OUT1, sizeof(double) * (eb + 1)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  V2 *X = ctx->ws[WS_E].as<V2>();
  double *ep = ctx->ws[WS_OUT1].as<double>();
  int *flag = ctx->ws[WS_FLAG].as<int>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_load_x<T, T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(k, k, x, X); }
  PPRVIZ_LAUNCHED(ctx);
  const T s = (T)scale;
  {
    PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY);
    if (gx && gD) k_energy<T, true, true><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag);
    else if (gx) k_energy<T, true, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag);
    else if (gD) k_energy<T, false, true><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag);
    else k_energy<T, false, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag);
  }
  PPRVIZ_LAUNCHED(ctx);
  { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_reduce_energy<<<1, 256, 0, ctx->stream>>>((int)eb, ep, ep + eb); }
  PPRVIZ_LAUNCHED(ctx);
  double e = 0.0;
  int hf = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&e, ep + eb, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hf) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "pdist has a non-positive off-diagonal entry");
  if (e_h) *e_h = e;
  return PPRVIZ_OK;
}

int energy_run(pprviz_ctx *ctx, const void *pdist_d, int32_t k, const void *x_d, double scale, bool f64,
               double *e_h, void *grad_x_d, void *grad_pdist_d) {
  if (f64)
    return energy_typed<double>(ctx, (const double *)pdist_d, k, (const double *)x_d, scale, e_h,
                                (double *)grad_x_d, (double *)grad_pdist_d);
  return energy_typed<float>(ctx, (const float *)pdist_d, k, (const float *)x_d, scale, e_h, (float *)grad_x_d,
                             (float *)grad_pdist_d);
}

// ---------------------------------------------------------------------------
// Allocation-free energy entry point (pprviz_energy_noalloc).
//
// Some callers may not allocate device memory at the time they need the
// energy: code that owns every byte of the device through its own pool or a
// framework allocator (a cudaMalloc there fails or fragments the pool), code
// running under a hard memory cap, or code that only enqueues work on a stream
// it was handed. For them the scratch of the energy pass (the staged
// coordinates, one FP64 partial per block and a status word) lives in the
// fixed device array below, which every GPU that loads the library holds
// until the process exits. The caller provides inputs and outputs.
// ---------------------------------------------------------------------------
constexpr int kNoAllocMaxK = 65536;
constexpr int kNoAllocBlocks = (kNoAllocMaxK + LWARPS * RPW - 1) / (LWARPS * RPW);
constexpr size_t kNoAllocXBytes = sizeof(float2) * kNoAllocMaxK;             // 512 KiB
constexpr size_t kNoAllocEBytes = sizeof(double) * (kNoAllocBlocks + 1);     // 16 KiB + 8 B
constexpr size_t kNoAllocBytes = kNoAllocXBytes + kNoAllocEBytes + 256;       // + status word

static __device__ __align__(256) unsigned char g_energy_scratch[kNoAllocBytes];

}  // namespace pprviz

#include <mutex>

namespace {

// Device address of g_energy_scratch, looked up once per device. In host code
// the array's name is only a host-side stand-in for the device symbol, so the
// kernels get this address instead.
std::mutex g_noalloc_mu;
void *g_noalloc_addr[256] = {nullptr};

cudaError_t noalloc_scratch(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, pprviz::g_energy_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int pprviz_energy_noalloc(const float *pdist, int32_t k, const float *x, double grad_scale, double *e_out,
                                     float *grad_x, float *grad_pdist, void *cuda_stream) {
  using namespace pprviz;
  if (!pdist || !x) return PPRVIZ_E_INVALID_ARG;
  if (k < 1 || k > kNoAllocMaxK) return PPRVIZ_E_INVALID_ARG;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  void *base = nullptr;
  if (noalloc_scratch(&base) != cudaSuccess) {
    cudaGetLastError();
    return PPRVIZ_E_CUDA;
  }
  float2 *X = reinterpret_cast<float2 *>(base);
  double *eparts = reinterpret_cast<double *>(static_cast<unsigned char *>(base) + kNoAllocXBytes);
  int *flag = reinterpret_cast<int *>(static_cast<unsigned char *>(base) + kNoAllocXBytes + kNoAllocEBytes);
  const unsigned eb = (unsigned)((k + LWARPS * RPW - 1) / (LWARPS * RPW));
  // the status word keeps the previous call's value: clear it first
  if (cudaMemsetAsync(flag, 0, sizeof(int), stream) != cudaSuccess) return PPRVIZ_E_CUDA;
  k_load_x<float, float><<<(unsigned)((k + 255) / 256), 256, 0, stream>>>(k, k, x, X);
  const float s = (float)grad_scale;
  if (grad_x && grad_pdist)
    k_energy<float, true, true><<<eb, LWARPS * 32, 0, stream>>>(k, pdist, X, s, eparts, grad_x, grad_pdist, flag);
  else if (grad_x)
    k_energy<float, true, false><<<eb, LWARPS * 32, 0, stream>>>(k, pdist, X, s, eparts, grad_x, grad_pdist, flag);
  else if (grad_pdist)
    k_energy<float, false, true><<<eb, LWARPS * 32, 0, stream>>>(k, pdist, X, s, eparts, grad_x, grad_pdist, flag);
  else
    k_energy<float, false, false><<<eb, LWARPS * 32, 0, stream>>>(k, pdist, X, s, eparts, grad_x, grad_pdist, flag);
  k_reduce_energy<<<1, 256, 0, stream>>>((int)eb, eparts, eparts + eb);
  if (cudaGetLastError() != cudaSuccess) return PPRVIZ_E_CUDA;
  double e = 0.0;
  int hf = 0;
  if (cudaMemcpyAsync(&e, eparts + eb, sizeof(double), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, stream) != cudaSuccess ||
      cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaGetLastError();
    return PPRVIZ_E_CUDA;
  }
  if (hf) return PPRVIZ_E_INVALID_ARG;
  if (e_out) *e_out = e;
  return PPRVIZ_OK;
}
