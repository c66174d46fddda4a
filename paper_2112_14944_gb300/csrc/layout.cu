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
//    centred Moore-Penrose solution. A is inverted in place by a blocked
//    Gauss-Jordan sweep (64-wide pivot blocks, no pivoting needed for SPD):
//    a one-block pivot inverse, panel products, and a register-tiled rank-64
//    trailing update, which carries the O(k^3) work.
//  * Each iteration is two streaming passes over k x k matrices: the L^Y pass
//    b_i = sum_j (x_i - x_j) / (Delta_ij d_ij) over the stored 1/Delta, and
//    X = M b over M = A^-1. Both read their matrix once, coalesced along
//    rows, with the 2-D coordinates staged in shared memory; the column range
//    is split over several blocks whose partial sums are added (in a fixed
//    order) by the consumer, so no atomics and bitwise-reproducible results.
//  * The energy and its gradients recompute every pair from X and Delta; no
//    k x k intermediate is stored.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace pprviz {

constexpr int NB = 64;        // Gauss-Jordan pivot block
constexpr int LWARPS = 8;     // warps per block in the pair passes
constexpr int RPW = 4;        // rows per warp in the pair passes
constexpr int XCH = 1024;     // coordinates staged per shared-memory chunk

template <typename T> struct T2;
template <> struct T2<float> { using type = float2; };
template <> struct T2<double> { using type = double2; };

template <typename T>
__device__ __forceinline__ T rsqrt_pos(T d2);
template <>
__device__ __forceinline__ float rsqrt_pos<float>(float d2) { return d2 > 0.0f ? rsqrtf(d2) : 0.0f; }
template <>
__device__ __forceinline__ double rsqrt_pos<double>(double d2) { return d2 > 0.0 ? 1.0 / sqrt(d2) : 0.0; }

// ---------------------------------------------------------------------------
// W1 = 1/Delta (zero diagonal) and A = L^w + J/k (identity on padded rows).
// One warp per row; the diagonal of L^w is the FP64 sum of the row's 1/Delta^2.
// ---------------------------------------------------------------------------
template <typename TI, typename T>
__global__ void k_build(int32_t k, int32_t kp, const TI *__restrict__ D, T *__restrict__ W1,
                        T *__restrict__ A, int *__restrict__ flag) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (i >= kp) return;
  T *Ai = A + i * kp;
  if (i >= k) {
    for (int64_t j = lane; j < kp; j += 32) Ai[j] = (j == i) ? T(1) : T(0);
    return;
  }
  T *Wi = W1 + i * kp;
  const TI *Di = D + i * (int64_t)k;
  const T invk = (T)(1.0 / (double)k);
  double rowsum = 0.0;
  int bad = 0;
  for (int64_t j = lane; j < kp; j += 32) {
    if (j < k && j != i) {
      const T d = (T)Di[j];
      if (!(d > T(0)) || !isfinite((double)d)) bad = 1;
      const T w1 = T(1) / d;
      const T wsq = w1 * w1;
      Wi[j] = w1;
      Ai[j] = invk - wsq;
      rowsum += (double)wsq;
    } else {
      Wi[j] = T(0);
      if (j != i) Ai[j] = T(0);
    }
  }
  for (int o = 16; o > 0; o >>= 1) rowsum += __shfl_xor_sync(0xffffffffu, rowsum, o);
  if (lane == 0) Ai[i] = (T)(rowsum + 1.0 / (double)k);
  if (bad) atomicOr(flag, 1);
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inversion of the SPD matrix A (kp x kp, kp % NB == 0).
// Sweeping pivot block K with P = A_KK^-1 maps
//   A_KK -> P,  A_KJ -> P A_KJ,  A_IK -> -A_IK P,  A_IJ -> A_IJ - A_IK P A_KJ;
// after sweeping every block the matrix holds A^-1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_gj_diag(int32_t kp, int32_t K0, T *__restrict__ A, T *__restrict__ P) {
  __shared__ T a[NB][NB + 1];
  __shared__ T rowp[NB], colp[NB];
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    a[r][c] = A[(int64_t)(K0 + r) * kp + K0 + c];
  }
  for (int p = 0; p < NB; ++p) {
    __syncthreads();
    if (threadIdx.x < NB) {
      rowp[threadIdx.x] = a[p][threadIdx.x];
      colp[threadIdx.x] = a[threadIdx.x][p];
    }
    __syncthreads();
    const T piv = T(1) / rowp[p];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, c = e % NB;
      T v;
      if (r == p && c == p) v = piv;
      else if (r == p) v = rowp[c] * piv;
      else if (c == p) v = -colp[r] * piv;
      else v = a[r][c] - colp[r] * (rowp[c] * piv);
      a[r][c] = v;
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    A[(int64_t)(K0 + r) * kp + K0 + c] = a[r][c];
    P[e] = a[r][c];
  }
}

// Vt[t][i] = A[i][K0 + t]: the old column panel, transposed (32x32 tiles).
template <typename T>
__global__ void k_gj_vt(int32_t kp, int32_t K0, const T *__restrict__ A, T *__restrict__ Vt) {
  __shared__ T tile[32][33];
  const int i0 = blockIdx.x * 32, t0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += 8) tile[r][threadIdx.x] = A[(int64_t)(i0 + r) * kp + K0 + t0 + threadIdx.x];
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) Vt[(int64_t)(t0 + r) * kp + i0 + threadIdx.x] = tile[threadIdx.x][r];
}

// Row panel: A[K0 + r][J0 + c] <- sum_t P[r][t] A[K0 + t][J0 + c] for every J block != K.
template <typename T>
__global__ void k_gj_rowpanel(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ P) {
  const int J0 = blockIdx.x * NB;
  if (J0 == K0) return;
  extern __shared__ unsigned char smem_raw[];
  T *sP = reinterpret_cast<T *>(smem_raw);  // [NB][NB]
  T *sB = sP + NB * NB;                     // [NB][NB]
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    sP[e] = P[e];
    sB[e] = A[(int64_t)(K0 + r) * kp + J0 + c];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    T s = T(0);
#pragma unroll 8
    for (int t = 0; t < NB; ++t) s += sP[r * NB + t] * sB[t * NB + c];
    A[(int64_t)(K0 + r) * kp + J0 + c] = s;
  }
}

// Column panel: A[I0 + r][K0 + c] <- -sum_t Vt[t][I0 + r] P[t][c] for every I block != K.
template <typename T>
__global__ void k_gj_colpanel(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ Vt,
                              const T *__restrict__ P) {
  const int I0 = blockIdx.x * NB;
  if (I0 == K0) return;
  extern __shared__ unsigned char smem_raw[];
  T *sP = reinterpret_cast<T *>(smem_raw);  // [NB][NB]
  T *sV = sP + NB * NB;                     // [NB][NB]: sV[t][r] = Vt[t][I0 + r]
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int t = e / NB, r = e % NB;
    sP[e] = P[e];
    sV[e] = Vt[(int64_t)t * kp + I0 + r];
  }
  __syncthreads();
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    T s = T(0);
#pragma unroll 8
    for (int t = 0; t < NB; ++t) s += sV[t * NB + r] * sP[t * NB + c];
    A[(int64_t)(I0 + r) * kp + K0 + c] = -s;
  }
}

// Trailing update A[i][j] -= sum_t Vt[t][i] A[K0 + t][j] for i, j outside the
// pivot block. TM x TM tile per block of 256 threads, R x R outputs per thread
// split into two SUB x SUB quadrants so that shared-memory reads are vectors.
template <typename T, int TM>
__global__ void __launch_bounds__(256)
k_gj_trailing(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ Vt) {
  constexpr int R = TM / 16, SUB = R / 2, HALF = TM / 2;
  extern __shared__ unsigned char smem_raw[];
  T *sA = reinterpret_cast<T *>(smem_raw);  // [NB][TM]  sA[t][i] = Vt[t][I0 + i]
  T *sB = sA + NB * TM;                     // [NB][TM]  sB[t][j] = A[K0 + t][J0 + j]
  const int I0 = blockIdx.y * TM, J0 = blockIdx.x * TM;
  // a tile lying entirely inside the pivot block row/column has nothing to do
  if ((I0 >= K0 && I0 + TM <= K0 + NB) || (J0 >= K0 && J0 + TM <= K0 + NB)) return;
  for (int e = threadIdx.x; e < NB * TM; e += 256) {
    const int t = e / TM, x = e % TM;
    sA[e] = (I0 + x < kp) ? Vt[(int64_t)t * kp + I0 + x] : T(0);
    sB[e] = (J0 + x < kp) ? A[(int64_t)(K0 + t) * kp + J0 + x] : T(0);
  }
  __syncthreads();
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T acc[R][R];
#pragma unroll
  for (int r = 0; r < R; ++r)
#pragma unroll
    for (int c = 0; c < R; ++c) acc[r][c] = T(0);
#pragma unroll 4
  for (int t = 0; t < NB; ++t) {
    T a[R], b[R];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int s = 0; s < SUB; ++s) {
        a[h * SUB + s] = sA[t * TM + h * HALF + ty * SUB + s];
        b[h * SUB + s] = sB[t * TM + h * HALF + tx * SUB + s];
      }
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
      for (int c = 0; c < R; ++c) acc[r][c] += a[r] * b[c];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = I0 + (r / SUB) * HALF + ty * SUB + (r % SUB);
    if (i >= kp || (i >= K0 && i < K0 + NB)) continue;
#pragma unroll
    for (int c = 0; c < R; ++c) {
      const int j = J0 + (c / SUB) * HALF + tx * SUB + (c % SUB);
      if (j >= kp || (j >= K0 && j < K0 + NB)) continue;
      A[(int64_t)i * kp + j] -= acc[r][c];
    }
  }
}

// ---------------------------------------------------------------------------
// Pair passes. Coordinates live as S column-split partial sums Xp[s][k]; the
// consumer adds the S parts in order. Block = 8 warps x 4 rows; blockIdx.y
// selects the column split.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ typename T2<T>::type sum_parts(const typename T2<T>::type *__restrict__ Xp, int S,
                                                          int64_t k, int64_t j) {
  typename T2<T>::type v = Xp[j];
  for (int s = 1; s < S; ++s) {
    const typename T2<T>::type u = Xp[(int64_t)s * k + j];
    v.x += u.x;
    v.y += u.y;
  }
  return v;
}

// MODE 0: L^Y pass, out_i = sum_j W1_ij (x_i - x_j) / |x_i - x_j|  (W1 = 1/Delta)
// MODE 1: apply,    out_i = sum_j M_ij v_j
// Mat is k x kp with kp a multiple of 128 and zero columns j >= k, so every
// block streams whole 128-column bands with 16-byte loads and no tail; the
// staged coordinates are zero beyond k. Each lane owns VW consecutive columns.
template <typename T, int MODE>
__global__ void __launch_bounds__(LWARPS * 32)
k_pairpass(int32_t k, int32_t kp, const T *__restrict__ Mat, const typename T2<T>::type *__restrict__ Vp,
           int S_in, typename T2<T>::type *__restrict__ Outp) {
  using V2 = typename T2<T>::type;
  constexpr int VW = 16 / sizeof(T);
  __shared__ __align__(16) T sx[XCH];
  __shared__ __align__(16) T sy[XCH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int S = gridDim.y, s = blockIdx.y;
  const int64_t bands = kp / 128;
  const int64_t jlo = bands * s / S * 128, jhi = bands * (s + 1) / S * 128;
  int64_t rows[RPW];
  T xi[RPW], yi[RPW], ax[RPW], ay[RPW];
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    rows[r] = ((int64_t)blockIdx.x * LWARPS + warp) * RPW + r;
    ax[r] = T(0);
    ay[r] = T(0);
    xi[r] = T(0);
    yi[r] = T(0);
    if (MODE == 0 && rows[r] < k) {
      const V2 v = sum_parts<T>(Vp, S_in, k, rows[r]);
      xi[r] = v.x;
      yi[r] = v.y;
    }
  }
  for (int64_t c0 = jlo; c0 < jhi; c0 += XCH) {
    const int cn = (int)min((int64_t)XCH, jhi - c0);  // a multiple of 128
    __syncthreads();
    for (int t = threadIdx.x; t < cn; t += blockDim.x) {
      V2 v;
      if (c0 + t < k) v = sum_parts<T>(Vp, S_in, k, c0 + t);
      else { v.x = T(0); v.y = T(0); }
      sx[t] = v.x;
      sy[t] = v.y;
    }
    __syncthreads();
#pragma unroll 2
    for (int t = lane * VW; t < cn; t += 32 * VW) {
      T m[RPW][VW];
#pragma unroll
      for (int r = 0; r < RPW; ++r) {
        if (rows[r] < k) {
          const uint4 raw = __ldg(reinterpret_cast<const uint4 *>(Mat + rows[r] * kp + c0 + t));
          memcpy(m[r], &raw, 16);
        } else {
#pragma unroll
          for (int u = 0; u < VW; ++u) m[r][u] = T(0);
        }
      }
      T xv[VW], yv[VW];
      {
        const uint4 rx = *reinterpret_cast<const uint4 *>(sx + t);
        const uint4 ry = *reinterpret_cast<const uint4 *>(sy + t);
        memcpy(xv, &rx, 16);
        memcpy(yv, &ry, 16);
      }
#pragma unroll
      for (int u = 0; u < VW; ++u) {
#pragma unroll
        for (int r = 0; r < RPW; ++r) {
          if (MODE == 0) {
            const T dx = xi[r] - xv[u], dy = yi[r] - yv[u];
            const T coef = m[r][u] * rsqrt_pos<T>(dx * dx + dy * dy);
            ax[r] += coef * dx;
            ay[r] += coef * dy;
          } else {
            ax[r] += m[r][u] * xv[u];
            ay[r] += m[r][u] * yv[u];
          }
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < RPW; ++r) {
    T vx = ax[r], vy = ay[r];
    for (int o = 16; o > 0; o >>= 1) {
      vx += __shfl_xor_sync(0xffffffffu, vx, o);
      vy += __shfl_xor_sync(0xffffffffu, vy, o);
    }
    if (lane == 0 && rows[r] < k) {
      V2 o;
      o.x = vx;
      o.y = vy;
      Outp[(int64_t)s * k + rows[r]] = o;
    }
  }
}

// X = sum of parts, mean subtracted, converted to the output type. One block
// (deterministic FP64 mean).
template <typename T, typename TO>
__global__ void k_finish(int32_t k, const typename T2<T>::type *__restrict__ Xp, int S, TO *__restrict__ out,
                         typename T2<T>::type *__restrict__ Xc) {
  __shared__ double sx[1024], sy[1024];
  double mx = 0.0, my = 0.0;
  for (int64_t i = threadIdx.x; i < k; i += blockDim.x) {
    const typename T2<T>::type v = sum_parts<T>(Xp, S, k, i);
    mx += (double)v.x;
    my += (double)v.y;
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
    const typename T2<T>::type v = sum_parts<T>(Xp, S, k, i);
    const T cx = (T)((double)v.x - ax), cy = (T)((double)v.y - ay);
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

template <typename TI, typename T>
__global__ void k_load_x(int32_t k, const TI *__restrict__ x, typename T2<T>::type *__restrict__ Xp,
                         int S) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= k) return;
  typename T2<T>::type v;
  v.x = (T)x[2 * i];
  v.y = (T)x[2 * i + 1];
  Xp[i] = v;
  typename T2<T>::type z;
  z.x = T(0);
  z.y = T(0);
  for (int s = 1; s < S; ++s) Xp[(int64_t)s * k + i] = z;
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

template <typename T>
int gj_invert(pprviz_ctx *ctx, int32_t kp, T *A, T *Vt, T *P) {
  constexpr int TM = sizeof(T) == 4 ? 128 : 64;
  const size_t trail_smem = 2 * sizeof(T) * NB * TM;
  const size_t panel_smem = 2 * sizeof(T) * NB * NB;
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_gj_trailing<T, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)trail_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_gj_rowpanel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)panel_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_gj_colpanel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)panel_smem));
  const int nblk = kp / NB;
  const unsigned tgrid = (unsigned)((kp + TM - 1) / TM);
  for (int kb = 0; kb < nblk; ++kb) {
    const int K0 = kb * NB;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_gj_diag<T><<<1, 256, 0, ctx->stream>>>(kp, K0, A, P); }
    PPRVIZ_LAUNCHED(ctx);
    if (nblk == 1) break;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_gj_vt<T><<<dim3(kp / 32, NB / 32), dim3(32, 8), 0, ctx->stream>>>(kp, K0, A, Vt); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_gj_rowpanel<T><<<nblk, 256, panel_smem, ctx->stream>>>(kp, K0, A, P); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_gj_trailing<T, TM><<<dim3(tgrid, tgrid), 256, trail_smem, ctx->stream>>>(kp, K0, A, Vt); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_gj_colpanel<T><<<nblk, 256, panel_smem, ctx->stream>>>(kp, K0, A, Vt, P); }
    PPRVIZ_LAUNCHED(ctx);
  }
  return PPRVIZ_OK;
}

int split_count(int32_t k, int32_t kp) {
  // about eight resident 256-thread blocks per SM on 152 SMs; at most one
  // 128-column band per split
  const int rowblocks = (k + LWARPS * RPW - 1) / (LWARPS * RPW);
  int S = (int)std::max(1, std::min(16, (8 * 152 + rowblocks - 1) / std::max(rowblocks, 1)));
  return std::min(S, kp / 128);
}

template <typename T, typename TI, typename TO>
int layout_typed(pprviz_ctx *ctx, const TI *pdist, int32_t k, const TI *x0, int32_t iters, TO *x_out,
                 double *stress_h) {
  using V2 = typename T2<T>::type;
  const int32_t kp = (k + 127) / 128 * 128;  // whole 128-column bands (and NB blocks)
  const int S = split_count(k, kp);
  PPRVIZ_TRY(ws_ensure(ctx, WS_W1, sizeof(T) * (size_t)kp * kp));
  PPRVIZ_TRY(ws_ensure(ctx, WS_M, sizeof(T) * (size_t)kp * kp));
  PPRVIZ_TRY(ws_ensure(ctx, WS_PIV, sizeof(T) * (size_t)(NB * kp + NB * NB)));
  PPRVIZ_TRY(ws_ensure(ctx, WS_X, sizeof(V2) * (size_t)S * k));
  PPRVIZ_TRY(ws_ensure(ctx, WS_B, sizeof(V2) * (size_t)S * k));
  PPRVIZ_TRY(ws_ensure(ctx, WS_E, sizeof(V2) * (size_t)k + 64));
  PPRVIZ_TRY(ws_ensure(ctx, WS_FLAG, 64));
  T *W1 = ctx->ws[WS_W1].as<T>(), *A = ctx->ws[WS_M].as<T>();
  T *Vt = ctx->ws[WS_PIV].as<T>(), *P = Vt + (size_t)NB * kp;
  V2 *Xp = ctx->ws[WS_X].as<V2>(), *Bp = ctx->ws[WS_B].as<V2>();
  int *flag = ctx->ws[WS_FLAG].as<int>();
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_build<TI, T><<<(unsigned)((kp + 7) / 8), 256, 0, ctx->stream>>>(k, kp, pdist, W1, A, flag); }
  PPRVIZ_LAUNCHED(ctx);
  int hf = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&hf, flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (hf) return set_err(ctx, PPRVIZ_E_INVALID_ARG, "pdist has a non-finite or non-positive off-diagonal entry");
  if (iters > 0) PPRVIZ_TRY(gj_invert<T>(ctx, kp, A, Vt, P));
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_load_x<TI, T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(k, x0, Xp, S); }
  PPRVIZ_LAUNCHED(ctx);
  const dim3 grid((unsigned)((k + LWARPS * RPW - 1) / (LWARPS * RPW)), (unsigned)S);
  for (int it = 0; it < iters; ++it) {
    { PPRVIZ_PROF(ctx, PPRVIZ_K_LY); k_pairpass<T, 0><<<grid, LWARPS * 32, 0, ctx->stream>>>(k, kp, W1, Xp, S, Bp); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_APPLY); k_pairpass<T, 1><<<grid, LWARPS * 32, 0, ctx->stream>>>(k, kp, A, Bp, S, Xp); }
    PPRVIZ_LAUNCHED(ctx);
  }
  V2 *Xc = ctx->ws[WS_E].as<V2>();
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_finish<T, TO><<<1, 1024, 0, ctx->stream>>>(k, Xp, S, x_out, Xc); }
  PPRVIZ_LAUNCHED(ctx);
  ctx->stats.layout_iters = iters;
  ctx->stats.bytes_ly = (double)sizeof(T) * k * (double)k * iters;
  ctx->stats.bytes_apply = (double)sizeof(T) * k * (double)k * iters;
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
  { PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER); k_load_x<T, T><<<(unsigned)((k + 255) / 256), 256, 0, ctx->stream>>>(k, x, X, 1); }
  PPRVIZ_LAUNCHED(ctx);
  const T s = (T)scale;
  if (gx && gD) { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<T, true, true><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag); }
  else if (gx) { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<T, true, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag); }
  else if (gD) { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<T, false, true><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag); }
  else { PPRVIZ_PROF(ctx, PPRVIZ_K_ENERGY); k_energy<T, false, false><<<eb, LWARPS * 32, 0, ctx->stream>>>(k, pdist, X, s, ep, gx, gD, flag); }
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

}  // namespace pprviz
