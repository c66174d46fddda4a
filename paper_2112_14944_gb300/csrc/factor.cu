// P5 - inverse of the SPD matrix A = L^w + J/k for the Guttman solve of Eq. (10).
//
// Symmetric block sweep (Gauss-Jordan on an SPD matrix, no pivoting needed).
// With P = A_KK^-1 for pivot block K:
//   A_KK -> -P,   A_IK -> A_IK P (and A_KI -> P A_KI),   A_IJ -> A_IJ - A_IK P A_KJ;
// the matrix stays symmetric after every sweep and equals -A^-1 once every
// block has been swept. Only the upper block triangle (NB x NB blocks I <= J,
// diagonal blocks in full) is stored and updated, which halves the O(k^3)
// trailing work. A final pass negates it (and, with 64-blocks, mirrors the
// lower 64-blocks inside the 128 x 128 diagonal tiles read by the layout).
//
// FP32: NB = 128, the trailing update on the tensor cores (3xTF32); every
// sweep reads and writes the stored triangle once, so the wide block halves
// that traffic against NB = 64. FP64: NB = 64 on the SIMT cores.
#include <math.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace pprviz {

// two sets (the lookahead's parities) of panels Ct, Ut (2 NB x kp each: the
// split high and low parts) and pivot inverse P (NB x NB), and a status word
size_t spd_inverse_work(int32_t kp) { return (size_t)2 * (2 * 256 * (size_t)kp + 128 * 128) + 64; }

// P = A_KK^-1 by an in-place scalar sweep of the NB x NB block in shared memory
// (ping-pong buffers, one barrier per pivot); writes P to `P` and -P into A_KK.
template <typename T, int NB>
__global__ void __launch_bounds__(512) k_fac_diag(int32_t kp, int32_t K0, T *__restrict__ A, T *__restrict__ P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);  // [2][NB][NB + 1]
  constexpr int LD = NB + 1, SZ = NB * LD;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    buf[r * LD + c] = A[(int64_t)(K0 + r) * kp + K0 + c];
  }
  __syncthreads();
  int cur = 0;
  for (int p = 0; p < NB; ++p) {
    const T *a = buf + cur * SZ;
    T *b = buf + (cur ^ 1) * SZ;
    const T piv = T(1) / a[p * LD + p];
    for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
      const int r = e / NB, c = e % NB;
      const T arc = a[r * LD + c], arp = a[r * LD + p], apc = a[p * LD + c];
      T v;
      if (r == p && c == p) v = piv;
      else if (r == p) v = apc * piv;
      else if (c == p) v = -arp * piv;
      else v = arc - arp * (apc * piv);
      b[r * LD + c] = v;
    }
    __syncthreads();
    cur ^= 1;
  }
  const T *a = buf + cur * SZ;
  for (int e = threadIdx.x; e < NB * NB; e += blockDim.x) {
    const int r = e / NB, c = e % NB;
    const T v = a[r * LD + c];
    P[e] = v;
    A[(int64_t)(K0 + r) * kp + K0 + c] = -v;
  }
}

// D = A_JJ^-1 for the 32 x 32 block J of a 128 x 128 block whose column
// block J is stored transposed in colT (colT[c][r] = A[r][32 J + c]), by one
// warp: the element sweep above in registers, lane = row. Per pivot p lane p
// publishes its row in a shared buffer (two, alternating, so one warp
// barrier per pivot suffices) and every lane reads it back with 16-byte
// broadcast loads. Writes D and its transpose.
__device__ __noinline__ void warp_inv32(const float *colT, int J, float *D, float *DT, float *rowbuf) {
  const int l = threadIdx.x & 31;
  float d[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) d[c] = colT[c * 128 + 32 * J + l];
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    float *rb = rowbuf + (p & 1) * 32;
    if (l == p) {
#pragma unroll
      for (int c = 0; c < 32; c += 4)
        *reinterpret_cast<float4 *>(rb + c) = make_float4(d[c], d[c + 1], d[c + 2], d[c + 3]);
    }
    __syncwarp();
    const float piv = 1.0f / rb[p];
    const float f = d[p] * piv;  // a_lp / a_pp
#pragma unroll
    for (int c = 0; c < 32; c += 4) {
      const float4 v = *reinterpret_cast<const float4 *>(rb + c);
      const float vs[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) d[c + e] = (l == p) ? vs[e] * piv : fmaf(-f, vs[e], d[c + e]);
    }
    d[p] = (l == p) ? piv : -f;
  }
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    D[l * 32 + c] = d[c];
    DT[c * 32 + l] = d[c];
  }
}

// The same sweep for a 128 x 128 FP32 block, in four 32-wide block steps
// (the block form of the sweep: sweeping the 32 pivots of block J at once is
// D = A_JJ^-1, A_JL <- D A_JL, A_IJ <- -A_IJ D, A_IL <- A_IL - A_IJ D A_JL,
// A_JJ <- D, the same result as 32 single-pivot sweeps). The block lives in
// registers, a 4 x 8 tile per thread (512 threads): thread t owns rows
// 4 (t / 16) + i and columns 8 (t % 16) + j. Per block step the old row block
// J and the old column block J (transposed) go to shared memory, one warp
// inverts A_JJ, and every thread updates its tile with 32-term products
// (three 16-byte shared loads per 32 FMAs): four barriers per block step
// instead of one per pivot. Dynamic shared memory: DIAG128_SMEM bytes.
constexpr int DIAG128_THREADS = 512;
constexpr int DIAG128_SMEM = (3 * 32 * 128 + 2 * 32 * 32 + 64) * 4;
__device__ __forceinline__ void fac_diag128(int32_t kp, int32_t K0, float *__restrict__ A, float *__restrict__ P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  float *sRowJ = reinterpret_cast<float *>(smem_raw);  // [32][128] old rows of block J
  float *sColT = sRowJ + 32 * 128;                     // [32][128] old column block J, transposed
  float *sNewT = sColT + 32 * 128;                     // [32][128] new column block J, transposed
  float *sD = sNewT + 32 * 128;                        // [32][32] A_JJ^-1
  float *sDT = sD + 32 * 32;                           // [32][32] its transpose
  float *sPiv = sDT + 32 * 32;                         // [2][32] pivot rows of the warp inverse
  const int rb = threadIdx.x >> 4, cb = threadIdx.x & 15;
  float a[4][8];  // a[i][j] = row 4 rb + i, column 8 cb + j
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float *src = A + (int64_t)(K0 + 4 * rb + i) * kp + K0 + 8 * cb;
    const float4 v0 = *reinterpret_cast<const float4 *>(src), v1 = *reinterpret_cast<const float4 *>(src + 4);
    a[i][0] = v0.x; a[i][1] = v0.y; a[i][2] = v0.z; a[i][3] = v0.w;
    a[i][4] = v1.x; a[i][5] = v1.y; a[i][6] = v1.z; a[i][7] = v1.w;
  }
#pragma unroll 1
  for (int J = 0; J < 4; ++J) {
    const bool rowJ = (rb >> 3) == J, colJ = (cb >> 2) == J;
    const int ri = 4 * (rb & 7), ci = 8 * (cb & 3);  // offsets inside block J
    if (rowJ) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        float *dst = sRowJ + (ri + i) * 128 + 8 * cb;
        *reinterpret_cast<float4 *>(dst) = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
        *reinterpret_cast<float4 *>(dst + 4) = make_float4(a[i][4], a[i][5], a[i][6], a[i][7]);
      }
    }
    if (colJ) {
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4 *>(sColT + (ci + j) * 128 + 4 * rb) = make_float4(a[0][j], a[1][j], a[2][j], a[3][j]);
    }
    __syncthreads();
    if (threadIdx.x < 32) warp_inv32(sColT, J, sD, sDT, sPiv);
    __syncthreads();
    if (rowJ) {  // A_JL <- D A_JL (the pivot block itself becomes D)
      if (colJ) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) a[i][j] = sD[(ri + i) * 32 + ci + j];
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) a[i][j] = 0.0f;
#pragma unroll 4
        for (int t = 0; t < 32; ++t) {
          const float4 x = *reinterpret_cast<const float4 *>(sDT + t * 32 + ri);
          const float4 y0 = *reinterpret_cast<const float4 *>(sRowJ + t * 128 + 8 * cb);
          const float4 y1 = *reinterpret_cast<const float4 *>(sRowJ + t * 128 + 8 * cb + 4);
          const float xs[4] = {x.x, x.y, x.z, x.w};
          const float ys[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) a[i][j] = fmaf(xs[i], ys[j], a[i][j]);
        }
      }
    } else if (colJ) {  // A_IJ <- -A_IJ D, also published for the other tiles of the rows
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) a[i][j] = 0.0f;
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        const float4 x = *reinterpret_cast<const float4 *>(sColT + t * 128 + 4 * rb);
        const float4 y0 = *reinterpret_cast<const float4 *>(sD + t * 32 + ci);
        const float4 y1 = *reinterpret_cast<const float4 *>(sD + t * 32 + ci + 4);
        const float xs[4] = {x.x, x.y, x.z, x.w};
        const float ys[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) a[i][j] = fmaf(-xs[i], ys[j], a[i][j]);
      }
#pragma unroll
      for (int j = 0; j < 8; ++j)
        *reinterpret_cast<float4 *>(sNewT + (ci + j) * 128 + 4 * rb) = make_float4(a[0][j], a[1][j], a[2][j], a[3][j]);
    }
    __syncthreads();
    if (!rowJ && !colJ) {  // A_IL <- A_IL + (-A_IJ D) A_JL
#pragma unroll 4
      for (int t = 0; t < 32; ++t) {
        const float4 x = *reinterpret_cast<const float4 *>(sNewT + t * 128 + 4 * rb);
        const float4 y0 = *reinterpret_cast<const float4 *>(sRowJ + t * 128 + 8 * cb);
        const float4 y1 = *reinterpret_cast<const float4 *>(sRowJ + t * 128 + 8 * cb + 4);
        const float xs[4] = {x.x, x.y, x.z, x.w};
        const float ys[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) a[i][j] = fmaf(xs[i], ys[j], a[i][j]);
      }
    }
    __syncthreads();  // before the next block step restages
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = 4 * rb + i;
    float *p = P + r * 128 + 8 * cb;
    float *q = A + (int64_t)(K0 + r) * kp + K0 + 8 * cb;
    *reinterpret_cast<float4 *>(p) = make_float4(a[i][0], a[i][1], a[i][2], a[i][3]);
    *reinterpret_cast<float4 *>(p + 4) = make_float4(a[i][4], a[i][5], a[i][6], a[i][7]);
    *reinterpret_cast<float4 *>(q) = make_float4(-a[i][0], -a[i][1], -a[i][2], -a[i][3]);
    *reinterpret_cast<float4 *>(q + 4) = make_float4(-a[i][4], -a[i][5], -a[i][6], -a[i][7]);
  }
}

__global__ void __launch_bounds__(DIAG128_THREADS) k_fac_diag128(int32_t kp, int32_t K0, float *__restrict__ A,
                                                      float *__restrict__ P) {
  fac_diag128(kp, K0, A, P);
}


template <typename T>
struct V4;  // 4-vector load/store of T
template <>
struct V4<float> {
  __device__ static void ld(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ static void st(float *p, const float (&v)[4]) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <>
struct V4<double> {
  __device__ static void ld(const double *p, double (&v)[4]) {
    const double2 t0 = reinterpret_cast<const double2 *>(p)[0], t1 = reinterpret_cast<const double2 *>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
  }
  __device__ static void st(double *p, const double (&v)[4]) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
  }
};

// Operand layout of the tensor-core trailing update ("split canonical"): for
// a 128-row block B and a 16-wide chunk c of the inner dimension, the TF32
// high parts (x with its low 13 mantissa bits cleared) and the remainders
// (x - high) of the 128 x 16 chunk are two consecutive 8 KiB runs in the
// canonical no-swizzle K-major layout of tcgen05 (8-row x 16-byte core
// matrices: byte (r / 8) 512 + (k / 4) 128 + (r % 8) 16 + (k % 4) 4), at
// float offset (B 8 + c) 4096. A chunk's operands are then one contiguous
// 16 KiB copy. Four consecutive k (k % 4 == 0) are contiguous, so the writer
// stores float4s.
__device__ __forceinline__ void store_split4(float *X, int row, int k, const float (&v)[4]) {
  const int B = row >> 7, r = row & 127, c = k >> 4, kk = k & 15;
  float *blk = X + (int64_t)(B * 8 + c) * 4096;
  const int o = ((r >> 3) * 512 + (kk >> 2) * 128 + (r & 7) * 16) >> 2;
  float4 h, l;
  h.x = __uint_as_float(__float_as_uint(v[0]) & 0xFFFFE000u);
  h.y = __uint_as_float(__float_as_uint(v[1]) & 0xFFFFE000u);
  h.z = __uint_as_float(__float_as_uint(v[2]) & 0xFFFFE000u);
  h.w = __uint_as_float(__float_as_uint(v[3]) & 0xFFFFE000u);
  l.x = v[0] - h.x; l.y = v[1] - h.y; l.z = v[2] - h.z; l.w = v[3] - h.w;
  *reinterpret_cast<float4 *>(blk + o) = h;
  *reinterpret_cast<float4 *>(blk + 2048 + o) = l;
}
template <typename T>
__device__ __forceinline__ void store_split4(T *, int, int, const T (&)[4]) {}  // FP64: unused

// Panel of pivot block K for block I != K (NB rows): C_I = A_IK (from the
// stored upper triangle: A[i][K0 + s] for I < K, A[K0 + s][i] for I > K),
// U_I = C_I P. Writes C_I and U_I for the trailing update, transposed
// (Ct[t][i], Ut[t][i], the SIMT update's layout) or, with KM, in the split
// canonical layout of the tensor-core update (rows i of block I, inner index
// t), and stores U_I back as the new panel (A_IK for I < K, A_KI = U_I^T for
// I > K). 256 threads on a 16 x 16 grid, each an R x R block of U
// (R = NB / 16) accumulated in registers.
template <typename T, int NB, bool KM>
__device__ __forceinline__ void fac_panel(int32_t kp, int32_t K0, int I0, T *__restrict__ A, const T *__restrict__ P,
                                          T *__restrict__ Ct, T *__restrict__ Ut) {
  constexpr int R = NB / 16, LD = NB + 16 / (int)sizeof(T);
  if (I0 == K0) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T *sP = reinterpret_cast<T *>(smem_raw);  // [NB][NB]   sP[s][t]
  T *sC = sP + NB * NB;                     // [NB][LD]   sC[s][i] = C[i][s]
  const bool above = I0 < K0;
  // 4-vectors, several in flight per thread
#pragma unroll 4
  for (int e = 4 * threadIdx.x; e < NB * NB; e += 4 * blockDim.x) {
    T pv[4], cv[4];
    V4<T>::ld(P + e, pv);
    V4<T>::st(sP + e, pv);
    const int r = e / NB, c = e % NB;
    if (above) {  // i = r, s = c .. c + 3
      V4<T>::ld(A + (int64_t)(I0 + r) * kp + K0 + c, cv);
#pragma unroll
      for (int w = 0; w < 4; ++w) sC[(c + w) * LD + r] = cv[w];
    } else {      // s = r, i = c .. c + 3
      V4<T>::ld(A + (int64_t)(K0 + r) * kp + I0 + c, cv);
      V4<T>::st(sC + r * LD + c, cv);
    }
  }
  __syncthreads();
  if (KM) {  // C[i][t .. t + 3], split
    for (int e = threadIdx.x; e < NB * NB / 4; e += blockDim.x) {
      const int i = e / (NB / 4), t = (e % (NB / 4)) * 4;
      const T v[4] = {sC[t * LD + i], sC[(t + 1) * LD + i], sC[(t + 2) * LD + i], sC[(t + 3) * LD + i]};
      store_split4(Ct, I0 + i, t, v);
    }
  }
  for (int e = threadIdx.x; e < NB * NB && !KM; e += blockDim.x) {
    {          // Ct[t][I0 + i] = C[i][t]
      const int t = e / NB, i = e % NB;
      Ct[(int64_t)t * kp + I0 + i] = sC[t * LD + i];
    }
  }
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  T u[R][R];
#pragma unroll
  for (int x = 0; x < R; ++x)
#pragma unroll
    for (int y = 0; y < R; ++y) u[x][y] = T(0);
#pragma unroll 4
  for (int s = 0; s < NB; ++s) {
    T av[R], bv[R];
#pragma unroll
    for (int q = 0; q < R / 4; ++q) {
      T tmp[4];
      V4<T>::ld(sC + s * LD + ty * R + 4 * q, tmp);
#pragma unroll
      for (int w = 0; w < 4; ++w) av[4 * q + w] = tmp[w];
      V4<T>::ld(sP + s * NB + tx * R + 4 * q, tmp);
#pragma unroll
      for (int w = 0; w < 4; ++w) bv[4 * q + w] = tmp[w];
    }
#pragma unroll
    for (int x = 0; x < R; ++x)
#pragma unroll
      for (int y = 0; y < R; ++y) u[x][y] += av[x] * bv[y];
  }
  // u[x][y] = U[i = ty R + x][t = tx R + y]
  if (!KM || !above) {
#pragma unroll
    for (int y = 0; y < R; ++y) {
      const int t = tx * R + y;
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        T tmp[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) tmp[w] = u[4 * q + w][y];
        if (!KM) V4<T>::st(Ut + (int64_t)t * kp + I0 + ty * R + 4 * q, tmp);
        if (!above) V4<T>::st(A + (int64_t)(K0 + t) * kp + I0 + ty * R + 4 * q, tmp);
      }
    }
  }
  if (KM || above) {
#pragma unroll
    for (int x = 0; x < R; ++x) {
      const int i = ty * R + x;
#pragma unroll
      for (int q = 0; q < R / 4; ++q) {
        T tmp[4];
#pragma unroll
        for (int w = 0; w < 4; ++w) tmp[w] = u[x][4 * q + w];
        if (KM) store_split4(Ut, I0 + i, tx * R + 4 * q, tmp);
        if (above) V4<T>::st(A + (int64_t)(I0 + i) * kp + K0 + tx * R + 4 * q, tmp);
      }
    }
  }
}

template <typename T, int NB, bool KM>
__global__ void __launch_bounds__(256) k_fac_panel(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ P,
                                                   T *__restrict__ Ct, T *__restrict__ Ut) {
  fac_panel<T, NB, KM>(kp, K0, (int)blockIdx.x * NB, A, P, Ct, Ut);
}

// SIMT trailing update of the upper triangle (FP64, NB = 64):
// A[i][j] -= sum_t Ct[t][i] Ut[t][j] for i, j outside the pivot block with
// block(i) <= block(j). TM x TM tiles over the upper tile triangle; R x R
// outputs per thread in two SUB x SUB quadrants so that shared-memory reads
// are vectors.
template <typename T, int TM, int NB>
__global__ void __launch_bounds__(256)
k_fac_trailing(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ Ct, const T *__restrict__ Ut) {
  constexpr int R = TM / 16, SUB = R / 2, HALF = TM / 2;
  const int I0 = blockIdx.y * TM, J0 = blockIdx.x * TM;
  if (J0 < I0) return;  // lower tile triangle: not stored
  if ((I0 >= K0 && I0 + TM <= K0 + NB) || (J0 >= K0 && J0 + TM <= K0 + NB)) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  T *sA = reinterpret_cast<T *>(smem_raw);  // [NB][TM]  sA[t][i] = Ct[t][I0 + i]
  T *sB = sA + NB * TM;                     // [NB][TM]  sB[t][j] = Ut[t][J0 + j]
  for (int e = threadIdx.x; e < NB * TM; e += 256) {
    const int t = e / TM, x = e % TM;
    sA[e] = (I0 + x < kp) ? Ct[(int64_t)t * kp + I0 + x] : T(0);
    sB[e] = (J0 + x < kp) ? Ut[(int64_t)t * kp + J0 + x] : T(0);
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
  // Epilogue: each row's SUB consecutive columns lie in one block, so the
  // masks (pivot block, lower blocks, kp) are uniform over them.
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = I0 + (r / SUB) * HALF + ty * SUB + (r % SUB);
    if (i >= kp || (i >= K0 && i < K0 + NB)) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = J0 + h * HALF + tx * SUB;
      if (j >= kp || (j >= K0 && j < K0 + NB) || (i / NB) > (j / NB)) continue;
      T *p = A + (int64_t)i * kp + j;
#pragma unroll
      for (int s = 0; s < SUB; ++s) p[s] -= acc[r][h * SUB + s];
    }
  }
}

// ---------------------------------------------------------------------------
// Tensor-core trailing update (FP32 inverse): C_IJ -= A_I^T B_J with the
// 3xTF32 split (Ootomo & Yokota 2022; hi = x with the low 13 mantissa bits
// cleared): C ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, FP32 accumulation in
// tensor memory, 128 x 128 tiles, inner dimension 128 in 16-wide chunks.
// ---------------------------------------------------------------------------
namespace tc {
constexpr int TM = 128;                       // tile edge (M = N = 128)
constexpr int NB = 128;                       // pivot block = inner dimension
constexpr int KC = 16;                        // inner chunk per stage
constexpr uint32_t LBO = 128;                 // bytes to the next core matrix along K
constexpr uint32_t SBO = (KC / 4) * 128;      // bytes to the next 8-row group
constexpr int OPB = TM * KC * 4;              // one staged operand part (8 KiB)
constexpr int STAGE = 4 * OPB;                // A_hi, A_lo, B_hi, B_lo
constexpr int NST = 2;                        // stages (64 KiB: also the epilogue's tile)
constexpr int SMEM = NST * STAGE + 1024;      // stages (+ alignment); the epilogue reuses 64 KiB of them
constexpr long WAIT_LIMIT = 1L << 22;         // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::tf32: F32 accumulate, TF32 A and B, both K-major
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

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

// Chunk c of the operands of tile (I0, J0) into stage st: the 16 KiB split
// runs of Ct block I0 / 128 and Ut block J0 / 128, completing on bar.
__device__ __forceinline__ void issue_chunk(uint32_t st, uint64_t *bar, const float *Ct, const float *Ut, int I0,
                                            int J0, int c) {
  const uint32_t b = smem_u32(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(STAGE) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(st),
               "l"(Ct + (int64_t)((I0 / TM) * (NB / KC) + c) * 4096), "r"(2 * OPB), "r"(b)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   st + 2 * OPB),
               "l"(Ut + (int64_t)((J0 / TM) * (NB / KC) + c) * 4096), "r"(2 * OPB), "r"(b)
               : "memory");
}
}  // namespace tc

// Tiles of one launch: with k1 < 0, every upper tile outside the pivot block
// row and column (grid tg x tg, the others exit at once); with k1 >= 0 and
// !only_k1, the same without block row and column k1 (the next pivot's);
// with only_k1, just the tiles of block row and column k1 (grid nblk x 1:
// block b is tile (b, k1) for b < k1, else (k1, b)). The lookahead of the
// host loop updates block row and column k1 first, so that the next pivot's
// inverse and panel overlap the rest of the update.
// One thread streams the 8 inner chunks of the tile's operands (already
// split by the panel kernel) through NST shared-memory stages with bulk
// copies and issues the 3 x 2 MMAs of each chunk; a stage is refilled once
// the MMAs of the chunk before it have completed. 65 KiB of shared memory,
// 128 tensor-memory columns: three CTAs per SM, so that one CTA's epilogue
// (the read-modify-write of its C tile) overlaps the other's MMAs. Every
// mbarrier wait has an iteration limit (on expiry the CTA sets `err`, skips
// the update and still frees its tensor memory after bounded waits for its
// copies and MMAs).
// C tile (I0, J0) -= Ct_I^T Ut_J (the whole CTA; see k_fac_trailing_tc).
__device__ __forceinline__ void trailing_tc_tile(int32_t kp, int I0, int J0, float *__restrict__ A,
                                                 const float *__restrict__ Ct, const float *__restrict__ Ut,
                                                 int *__restrict__ err) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[NST], mmad[NST];
  __shared__ uint32_t tmem_sh;
  __shared__ int ok_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *sbuf = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // 1024-byte aligned
  const uint32_t sb = smem_u32(sbuf);
  // TMEM read-out: warp w takes lanes (rows) 32 (w % 4) .. + 31 and columns
  // 64 (w / 4) .. + 63 of the accumulator.
  const int lg = warp & 3, chalf = warp >> 2;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)), "r"(TM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mmad[q])));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  constexpr int NCH = NB / KC;
  if (tid == 0) {
    bool ok = true;
    int issued = 0, done = -1;  // chunks copied; last chunk whose MMAs were seen complete
    for (int c = 0; c < NST && c < NCH; ++c) issue_chunk(sb + c * STAGE, &full[c], Ct, Ut, I0, J0, c);
    issued = NST < NCH ? NST : NCH;
    int mmad_last = -1;
    for (int c = 0; c < NCH && ok; ++c) {
      const int s = c % NST;
      if (!mbar_wait(&full[s], (uint32_t)((c / NST) & 1))) {
        ok = false;
        break;
      }
      const uint32_t base = sb + s * STAGE;
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t pa = base + (pass == 2 ? OPB : 0);
        const uint32_t pb = base + 2 * OPB + (pass == 1 ? OPB : 0);
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint64_t da = desc(pa + ks * 2 * LBO);
          const uint64_t db = desc(pb + ks * 2 * LBO);
          const uint32_t acc = (c == 0 && pass == 0 && ks == 0) ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mmad[s])));
      mmad_last = c;
      // refill the stage of chunk c - 1 once its MMAs are done
      if (c >= 1 && c - 1 + NST < NCH) {
        const int sp = (c - 1) % NST;
        if (!mbar_wait(&mmad[sp], (uint32_t)(((c - 1) / NST) & 1))) {
          ok = false;
          break;
        }
        done = c - 1;
        issue_chunk(sb + sp * STAGE, &full[sp], Ct, Ut, I0, J0, c - 1 + NST);
        issued = c - 1 + NST + 1;
      }
    }
    // all MMAs complete (they complete in order)
    if (ok && !mbar_wait(&mmad[(NCH - 1) % NST], (uint32_t)(((NCH - 1) / NST) & 1))) ok = false;
    if (!ok) {
      atomicOr(err, 1);
      // bounded waits for the copies and MMAs this CTA issued
      for (int c = done + 1; c < issued; ++c) (void)mbar_wait(&full[c % NST], (uint32_t)((c / NST) & 1));
      for (int c = done + 1; c <= mmad_last; ++c) (void)mbar_wait(&mmad[c % NST], (uint32_t)((c / NST) & 1));
    }
    ok_sh = ok ? 1 : 0;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ok_sh) {
    // The product goes through shared memory (the stages are free once the
    // last MMA has completed) so that the read-modify-write of the C tile is
    // row-contiguous: warp w writes its 32 rows x 64 columns (TMEM lane = row),
    // 16-byte chunk c of row r at chunk slot c ^ (r % 32); then each warp
    // updates whole 512-byte rows.
    float *tile = reinterpret_cast<float *>(sbuf);  // 128 x 128
    const uint32_t tbase = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(64 * chalf);
    const int row = 32 * lg + lane;
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tbase + (uint32_t)(16 * q)));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int c4 = 16 * chalf + 4 * q + c;
        *reinterpret_cast<float4 *>(tile + row * TM + 4 * (c4 ^ (row & 31))) =
            make_float4(__uint_as_float(v[4 * c]), __uint_as_float(v[4 * c + 1]), __uint_as_float(v[4 * c + 2]),
                        __uint_as_float(v[4 * c + 3]));
      }
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = warp; rr < TM; rr += 8) {
      const float4 d = *reinterpret_cast<const float4 *>(tile + rr * TM + 4 * (lane ^ (rr & 31)));
      float4 *p = reinterpret_cast<float4 *>(A + (int64_t)(I0 + rr) * kp + J0) + lane;
      float4 x = *p;
      x.x -= d.x;
      x.y -= d.y;
      x.z -= d.z;
      x.w -= d.w;
      *p = x;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM));
}

__global__ void __launch_bounds__(256, 3)
k_fac_trailing_tc(int32_t kp, int32_t K0, int k1, int only_k1, float *__restrict__ A, const float *__restrict__ Ct,
                  const float *__restrict__ Ut, int *__restrict__ err) {
  using namespace tc;
  int I0, J0;
  if (only_k1) {
    const int b = blockIdx.x;
    I0 = (b < k1 ? b : k1) * TM;
    J0 = (b < k1 ? k1 : b) * TM;
  } else {
    I0 = blockIdx.y * TM;
    J0 = blockIdx.x * TM;
    if (k1 >= 0 && (I0 == k1 * TM || J0 == k1 * TM)) return;  // the lookahead's tiles
  }
  if (J0 < I0 || I0 == K0 || J0 == K0) return;  // lower triangle, pivot row and column
  trailing_tc_tile(kp, I0, J0, A, Ct, Ut, err);
}

// ---------------------------------------------------------------------------
// Persistent, warp-specialized tensor-core trailing update (single FP32
// inverse). One CTA per SM walks a static share of the launch's tiles:
//   warp 0 (one lane): streams each tile's 8 inner chunks (32 KiB: the split
//     high and low parts of Ct block I and Ut block J, bulk copies) through
//     NST shared-memory stages (full / empty mbarriers);
//   warp 1 (one lane): issues the 3 x 2 tcgen05.mma.kind::tf32 of each chunk
//     into one of two tensor-memory accumulators (128 columns each) and
//     commits the stage back to the producer and the accumulator to the
//     epilogue;
//   warps 4-7 (thread = tile row = TMEM lane): load their C rows by bulk
//     copies into a padded staging tile, subtract the accumulator (tcgen05.ld),
//     release it, and store the rows back by bulk copies.
// With two accumulators the epilogue of one tile overlaps the MMAs of the
// next, and the operand stream runs ahead by NST chunks. Every wait is bounded
// by a global-timer deadline: on expiry the CTA records the error, stops, waits
// (bounded) for its copies and MMAs in flight, and frees its tensor memory.
// `withhold` >= 0 makes CTA 0 skip that chunk's copies (a test of the expiry
// path; the wait for it then runs out); -1 in normal use.
// ---------------------------------------------------------------------------
namespace tcp {
constexpr int TM = 128, NB = 128, KC = 16;
constexpr int OPB = TM * KC * 4;            // 8 KiB: one split part of a 128 x 16 chunk
constexpr int CHUNK = 4 * OPB;              // A_hi, A_lo, B_hi, B_lo
constexpr int NST = 4;                      // operand stages
constexpr int NCH = NB / KC;                // chunks per tile
constexpr int CROW = TM * 4 + 16;           // staged C row stride: 528 B, conflict-free 16-byte accesses
constexpr int SMEM = NST * CHUNK + TM * CROW + 1024;
constexpr int THREADS = 256;
constexpr int SIDE_SMS = 8;                 // SMs left to the next pivot's inverse and panel
}  // namespace tcp

namespace {

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait for the phase `parity` of `bar`: false once the deadline
// passes or another role of the CTA has given up (abort set).
__device__ __forceinline__ bool pwait(uint64_t *bar, uint32_t parity, uint64_t limit_ns, volatile int *abort_f) {
  const uint32_t b = tc::smem_u32(bar);
  uint32_t done = 0;
  uint64_t t0 = 0;
  for (int it = 0;; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(b), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 63) == 0) {
      if (*abort_f) return false;
      const uint64_t t = gtimer();
      if (it == 0) t0 = t;
      else if (t - t0 > limit_ns) return false;
    }
  }
}

// Tiles of one launch in a fixed order. mode 0: the upper tiles (I <= J) of
// the blocks other than K and k1 (k1 < 0: only K excluded), row-major over the
// kept blocks; mode 1: the tiles of block row / column k1 other than K's.
struct TileWalk {
  int mode, m, i, j, e1, e2, k1, nblk;
  __device__ void init(int mode_, int nblk_, int K, int k1_, int t) {
    mode = mode_;
    nblk = nblk_;
    k1 = k1_;
    if (mode == 1) {
      m = nblk - 1;
      i = t;
      j = 0;
      e1 = K;
      return;
    }
    e1 = k1 < 0 ? K : min(K, k1);
    e2 = k1 < 0 ? 0x7fffffff : max(K, k1);
    m = nblk - (k1 < 0 ? 1 : 2);
    i = 0;
    while (i < m && t >= m - i) {
      t -= m - i;
      ++i;
    }
    j = i + t;
  }
  __device__ bool valid() const { return i < m; }
  __device__ void advance(int g) {
    if (mode == 1) {
      i += g;
      return;
    }
    j += g;
    while (i < m && j >= m) {
      j -= m - (i + 1);
      ++i;
    }
  }
  __device__ int blk(int x) const {
    int b = x;
    if (b >= e1) ++b;
    if (b >= e2) ++b;
    return b;
  }
  __device__ void tile(int &I0, int &J0) const {
    if (mode == 1) {
      const int b = i + (i >= e1 ? 1 : 0);
      I0 = min(b, k1) * tcp::TM;
      J0 = max(b, k1) * tcp::TM;
      return;
    }
    I0 = blk(i) * tcp::TM;
    J0 = blk(j) * tcp::TM;
  }
};

}  // namespace

__global__ void __launch_bounds__(tcp::THREADS, 1)
k_fac_trailing_pp(int32_t kp, int nblk, int K, int k1, int mode, float *__restrict__ A, const float *__restrict__ Ct,
                  const float *__restrict__ Ut, int *__restrict__ err, uint64_t limit_ns, int withhold) {
  using namespace tcp;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], accf[2], acce[2], cfull[4], fin;
  __shared__ uint32_t tmem_sh;
  __shared__ int abort_sh, prod_issued, mma_done, held;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *sbuf = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sb = tc::smem_u32(sbuf);
  unsigned char *cbuf = sbuf + NST * CHUNK;
  volatile int *abort_f = &abort_sh;
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::smem_u32(&tmem_sh)),
                 "r"(2 * TM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    for (int q = 0; q < NST; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&full[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&empty[q])));
    }
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&accf[q])));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;" ::"r"(tc::smem_u32(&acce[q])));
    }
    for (int q = 0; q < 4; ++q) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&cfull[q])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&fin)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    abort_sh = 0;
    prod_issued = 0;
    mma_done = 0;
    held = -1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const int G = (int)gridDim.x;

  if (warp == 0 && lane == 0) {
    // ---- producer
    TileWalk w;
    w.init(mode, nblk, K, k1, (int)blockIdx.x);
    int g = 0;
    bool ok = true;
    for (; ok && w.valid(); w.advance(G)) {
      int I0, J0;
      w.tile(I0, J0);
      for (int c = 0; c < NCH; ++c, ++g) {
        const int st = g % NST, n = g / NST;
        if (g >= NST && !pwait(&empty[st], (uint32_t)((n - 1) & 1), limit_ns, abort_f)) {
          ok = false;
          break;
        }
        if (withhold == g && blockIdx.x == 0) {
          held = g;  // this chunk's copies are not issued: the MMA warp's wait for it runs out
          continue;
        }
        const uint32_t dst = sb + st * CHUNK;
        const uint32_t b = tc::smem_u32(&full[st]);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(CHUNK) : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(Ct + (int64_t)((I0 / TM) * NCH + c) * 4096), "r"(2 * OPB), "r"(b)
            : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                dst + 2 * OPB),
            "l"(Ut + (int64_t)((J0 / TM) * NCH + c) * 4096), "r"(2 * OPB), "r"(b)
            : "memory");
      }
    }
    if (!ok) {
      atomicOr(err, 1);
      abort_sh = 1;
    }
    prod_issued = g;
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    TileWalk w;
    w.init(mode, nblk, K, k1, (int)blockIdx.x);
    int g = 0, li = 0;
    bool ok = true;
    for (; ok && w.valid(); w.advance(G), ++li) {
      const int ab = li & 1;
      if (li >= 2 && !pwait(&acce[ab], (uint32_t)(((li >> 1) - 1) & 1), limit_ns, abort_f)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dacc = tmem + (uint32_t)(ab * TM);
      for (int c = 0; c < NCH; ++c, ++g) {
        const int st = g % NST;
        if (!pwait(&full[st], (uint32_t)((g / NST) & 1), limit_ns, abort_f)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = sb + st * CHUNK;
#pragma unroll 1
        for (int pass = 0; pass < 3; ++pass) {
          const uint32_t pa = base + (pass == 2 ? OPB : 0);
          const uint32_t pb = base + 2 * OPB + (pass == 1 ? OPB : 0);
#pragma unroll
          for (int ks = 0; ks < KC / 8; ++ks) {
            const uint64_t da = tc::desc(pa + ks * 2 * tc::LBO);
            const uint64_t db = tc::desc(pb + ks * 2 * tc::LBO);
            const uint32_t accum = (c == 0 && pass == 0 && ks == 0) ? 0u : 1u;
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
                "l"(da), "l"(db), "r"(tc::IDESC), "r"(accum));
          }
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            tc::smem_u32(&empty[st])));
      }
      if (!ok) break;
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          tc::smem_u32(&accf[ab])));
    }
    if (!ok) {
      atomicOr(err, 1);
      abort_sh = 1;
    }
    mma_done = g;
    // every MMA this thread issued has completed before the tensor memory is freed
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        tc::smem_u32(&fin)));
    if (!pwait(&fin, 0u, limit_ns, abort_f)) {
      volatile int zero = 0;  // a second bounded wait that ignores abort
      (void)pwait(&fin, 0u, limit_ns, &zero);
    }
  } else if (warp >= 4) {
    // ---- epilogue: thread = tile row r = TMEM lane
    const int ew = warp & 3, r = 32 * ew + lane;
    unsigned char *crow = cbuf + r * CROW;
    const uint32_t crow_s = tc::smem_u32(crow);
    TileWalk w;
    w.init(mode, nblk, K, k1, (int)blockIdx.x);
    int li = 0;
    bool ok = true, cpending = false;
    for (; ok && w.valid(); w.advance(G), ++li) {
      int I0, J0;
      w.tile(I0, J0);
      const int ab = li & 1;
      float *grow = A + (int64_t)(I0 + r) * kp + J0;
      // the previous tile's store has read this row: load the new C row
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      __syncwarp();
      const uint32_t cb = tc::smem_u32(&cfull[ew]);
      if (lane == 0)
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cb), "r"(32 * TM * 4) : "memory");
      __syncwarp();
      asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                       crow_s),
                   "l"(grow), "r"(TM * 4), "r"(cb)
                   : "memory");
      cpending = true;
      // the warp decides together (tcgen05.ld below is warp-collective)
      if (!__all_sync(0xffffffffu, pwait(&accf[ab], (uint32_t)((li >> 1) & 1), limit_ns, abort_f))) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!__all_sync(0xffffffffu, pwait(&cfull[ew], (uint32_t)(li & 1), limit_ns, abort_f))) {
        ok = false;
        break;
      }
      cpending = false;
      const uint32_t tb = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(ab * TM);
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        uint32_t v[32];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
            "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(tb + (uint32_t)(32 * q)));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int t4 = 0; t4 < 8; ++t4) {
          float4 *cp = reinterpret_cast<float4 *>(crow + 4 * (32 * q + 4 * t4));
          float4 x = *cp;
          x.x -= __uint_as_float(v[4 * t4 + 0]);
          x.y -= __uint_as_float(v[4 * t4 + 1]);
          x.z -= __uint_as_float(v[4 * t4 + 2]);
          x.w -= __uint_as_float(v[4 * t4 + 3]);
          *cp = x;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc::smem_u32(&acce[ab])) : "memory");
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(grow), "r"(crow_s),
                   "r"(TM * 4)
                   : "memory");
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    }
    if (!ok) {
      atomicOr(err, 1);
      abort_sh = 1;
      if (cpending) {  // a C row load still in flight: let it land before the CTA exits
        volatile int zero = 0;
        (void)pwait(&cfull[ew], (uint32_t)(li & 1), limit_ns, &zero);
      }
    }
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (tid == 0 && abort_sh) {
    // operand copies issued but never consumed: let them land before exit
    volatile int zero = 0;
    for (int g = mma_done; g < prod_issued; ++g)
      if (g != held) (void)pwait(&full[g % NST], (uint32_t)((g / NST) & 1), limit_ns, &zero);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TM));
}

// A <- -A on the upper block triangle; with NB = 64 also the lower 64-block of
// every 128 x 128 diagonal tile filled from its mirror, giving M = A^-1 on the
// upper tile triangle with full diagonal tiles (what the layout reads).
template <typename T, int NB>
__global__ void k_fac_finish(int32_t kp, T *__restrict__ A) {
  const int64_t i = blockIdx.y;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < kp; j += (int64_t)gridDim.x * blockDim.x) {
    if (i / NB > j / NB) continue;
    const T v = -A[i * kp + j];
    A[i * kp + j] = v;
    if (NB < 128 && i / 128 == j / 128 && i / NB < j / NB) A[j * kp + i] = v;
  }
}

template <typename T>
static int spd_inverse(pprviz_ctx *ctx, int32_t kp, T *A, T *work) {
  constexpr bool TC = std::is_same<T, float>::value;  // FP32: 128-blocks, tensor-core trailing update
  constexpr int NB = TC ? 128 : 64;
  constexpr int TM = 64;                               // SIMT trailing tile (FP64)
  const size_t pan = (TC ? 2 : 1) * (size_t)NB * kp;         // one panel (split into high and low parts with TC)
  const size_t set = 2 * pan + (size_t)NB * NB;               // one parity's Ct, Ut, P
  T *Ct[2], *Ut[2], *P[2];
  for (int q = 0; q < 2; ++q) {
    Ct[q] = work + q * set;
    Ut[q] = Ct[q] + pan;
    P[q] = Ct[q] + 2 * pan;
  }
  int *err = reinterpret_cast<int *>(work + 2 * set);
  const size_t diag_smem = 2 * sizeof(T) * NB * (NB + 1);
  const size_t panel_smem = sizeof(T) * (NB * NB + NB * (NB + 16 / sizeof(T)));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_panel<T, NB, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)panel_smem));
  if constexpr (TC) {
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)tc::SMEM));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  } else {
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_diag<T, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)diag_smem));
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing<T, TM, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(2 * sizeof(T) * NB * TM)));
  }
  const int nblk = kp / NB;
  // per pivot: the NB^3 pivot inverse, (nblk - 1) panel products of 2 NB^3,
  // and 2 NB^3 flops for each of the (nblk - 1) nblk / 2 upper blocks
  const double b3 = (double)NB * NB * NB;
  const double nm1 = (double)(nblk - 1);
  ctx->stats.flops_factor += (double)nblk * (2.0 * b3 + nm1 * 2.0 * b3 + nm1 * (nm1 + 1.0) / 2.0 * 2.0 * b3);
  if constexpr (TC) {
    // Lookahead by one pivot on a second stream: step kb updates block row
    // and column kb + 1 first (T1, main stream); the side stream then inverts
    // pivot kb + 1 and forms its panel into the other parity's buffers while
    // the main stream runs the rest of step kb's update (T2). One profiling
    // interval covers the whole inverse on the main stream.
    if (!ctx->side) {
      // highest priority, so that the pivot's one-CTA inverse and the panel
      // are dispatched as soon as an SM frees up instead of after the queued
      // CTAs of the main stream's update
      int lo = 0, hi = 0;
      PPRVIZ_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&lo, &hi));
      PPRVIZ_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->side, cudaStreamNonBlocking, hi));
    }
    if (!ctx->ev_t1) PPRVIZ_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_t1, cudaEventDisableTiming));
    if (!ctx->ev_dp) PPRVIZ_CUDA(ctx, cudaEventCreateWithFlags(&ctx->ev_dp, cudaEventDisableTiming));
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_diag128, cudaFuncAttributeMaxDynamicSharedMemorySize, DIAG128_SMEM));
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing_pp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tcp::SMEM));
    int nsm = 0;
    PPRVIZ_CUDA(ctx, cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device));
    const uint64_t limit_ns = 2000000000ull;  // bounded waits: 2 s
    int withhold = ctx->test_expire_wait ? 0 : -1;  // consumed by the first main trailing launch
    ctx->test_expire_wait = false;
    PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR);
    float *Af = (float *)A;
    k_fac_diag128<<<1, DIAG128_THREADS, DIAG128_SMEM, ctx->stream>>>(kp, 0, Af, (float *)P[0]);
    PPRVIZ_LAUNCHED(ctx);
    if (nblk > 1) {
      k_fac_panel<T, NB, TC><<<nblk, 256, panel_smem, ctx->stream>>>(kp, 0, A, P[0], Ct[0], Ut[0]);
      PPRVIZ_LAUNCHED(ctx);
    }
    for (int kb = 0; nblk > 1 && kb < nblk; ++kb) {
      const int q = kb & 1, k1 = kb + 1 < nblk ? kb + 1 : -1;
      if (k1 >= 0) {
        // block row and column k1 first (nblk - 1 tiles), then the next
        // pivot's inverse and panel on the side stream, on the SMs that the
        // main update leaves free
        const int t1 = nblk - 1;
        k_fac_trailing_pp<<<(unsigned)std::min(t1, nsm), tcp::THREADS, tcp::SMEM, ctx->stream>>>(
            kp, nblk, kb, k1, 1, Af, (const float *)Ct[q], (const float *)Ut[q], err, limit_ns, -1);
        PPRVIZ_LAUNCHED(ctx);
        PPRVIZ_CUDA(ctx, cudaEventRecord(ctx->ev_t1, ctx->stream));
        PPRVIZ_CUDA(ctx, cudaStreamWaitEvent(ctx->side, ctx->ev_t1, 0));
        k_fac_diag128<<<1, DIAG128_THREADS, DIAG128_SMEM, ctx->side>>>(kp, k1 * NB, Af, (float *)P[q ^ 1]);
        PPRVIZ_LAUNCHED(ctx);
        k_fac_panel<T, NB, TC><<<nblk, 256, panel_smem, ctx->side>>>(kp, k1 * NB, A, P[q ^ 1], Ct[q ^ 1], Ut[q ^ 1]);
        PPRVIZ_LAUNCHED(ctx);
        PPRVIZ_CUDA(ctx, cudaEventRecord(ctx->ev_dp, ctx->side));
      }
      const int m = nblk - (k1 >= 0 ? 2 : 1);
      const int tiles = m * (m + 1) / 2;
      if (tiles > 0) {
        const int cap = k1 >= 0 ? std::max(1, nsm - tcp::SIDE_SMS) : nsm;
        k_fac_trailing_pp<<<(unsigned)std::min(tiles, cap), tcp::THREADS, tcp::SMEM, ctx->stream>>>(
            kp, nblk, kb, k1, 0, Af, (const float *)Ct[q], (const float *)Ut[q], err, limit_ns, withhold);
        PPRVIZ_LAUNCHED(ctx);
        withhold = -1;
      }
      if (k1 >= 0) PPRVIZ_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ctx->ev_dp, 0));
      if (k1 < 0) break;
    }
    k_fac_finish<T, NB><<<dim3((unsigned)std::min(8, (kp + 255) / 256), (unsigned)kp), 256, 0, ctx->stream>>>(kp, A);
    PPRVIZ_LAUNCHED(ctx);
  } else {
    for (int kb = 0; kb < nblk; ++kb) {
      const int K0 = kb * NB;
      { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_diag<T, NB><<<1, 512, diag_smem, ctx->stream>>>(kp, K0, A, P[0]); }
      PPRVIZ_LAUNCHED(ctx);
      if (nblk == 1) break;
      { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_panel<T, NB, TC><<<nblk, 256, panel_smem, ctx->stream>>>(kp, K0, A, P[0], Ct[0], Ut[0]); }
      PPRVIZ_LAUNCHED(ctx);
      const unsigned tg = (unsigned)((kp + TM - 1) / TM);
      { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_trailing<T, TM, NB><<<dim3(tg, tg), 256, 2 * sizeof(T) * NB * TM, ctx->stream>>>(kp, K0, A, Ct[0], Ut[0]); }
      PPRVIZ_LAUNCHED(ctx);
    }
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_finish<T, NB><<<dim3((unsigned)std::min(8, (kp + 255) / 256), (unsigned)kp), 256, 0, ctx->stream>>>(kp, A); }
    PPRVIZ_LAUNCHED(ctx);
  }
  if constexpr (TC) {
    int herr = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "tensor-core trailing update: a bounded wait expired");
  }
  return PPRVIZ_OK;
}

int spd_inverse_f32(pprviz_ctx *ctx, int32_t kp, float *A, float *work) { return spd_inverse<float>(ctx, kp, A, work); }
int spd_inverse_f64(pprviz_ctx *ctx, int32_t kp, double *A, double *work) {
  return spd_inverse<double>(ctx, kp, A, work);
}


// ---------------------------------------------------------------------------
// Batched FP32 inverses (the views of one batch): the same block sweep, pivot
// step by pivot step, each launch covering that step's work in every view that
// still has the pivot: one CTA per view for the pivot inverse, one per block
// for the panels, one per upper tile for the trailing update (the views'
// blocks and tiles concatenated; a CTA finds its view by binary search over
// the launch's offsets). No lookahead: the batch's views fill the GPU.
// ---------------------------------------------------------------------------
namespace {

struct FacJob {
  float *A, *Ct, *Ut, *P;
  int32_t kp, nblk;
};

// largest i < n with off[i] <= b (off non-decreasing, off[0] <= b)
__device__ __forceinline__ int find_slot(const int *__restrict__ off, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(DIAG128_THREADS) k_fac_diag128_batch(const FacJob *__restrict__ jobs, const int *__restrict__ act,
                                                            int32_t K0) {
  const FacJob j = jobs[act[blockIdx.x]];
  fac_diag128(j.kp, K0, j.A, j.P);
}

__global__ void __launch_bounds__(256) k_fac_panel_batch(const FacJob *__restrict__ jobs, const int *__restrict__ act,
                                                         const int *__restrict__ off, int nact, int32_t K0) {
  const int s = find_slot(off, nact, (int)blockIdx.x);
  const FacJob j = jobs[act[s]];
  fac_panel<float, 128, true>(j.kp, K0, ((int)blockIdx.x - off[s]) * 128, j.A, j.P, j.Ct, j.Ut);
}

// tile t of a view's upper tile triangle, row by row: (I, J), I <= J
__global__ void __launch_bounds__(256, 3)
k_fac_trailing_tc_batch(const FacJob *__restrict__ jobs, const int *__restrict__ act, const int *__restrict__ off,
                        int nact, int kb, int *__restrict__ err) {
  const int s = find_slot(off, nact, (int)blockIdx.x);
  const FacJob j = jobs[act[s]];
  int t = (int)blockIdx.x - off[s], I = 0;
  while (I < j.nblk && t >= j.nblk - I) {
    t -= j.nblk - I;
    ++I;
  }
  const int J = I + t;
  if (I >= j.nblk || J >= j.nblk || I == kb || J == kb) return;
  trailing_tc_tile(j.kp, I * tc::TM, J * tc::TM, j.A, j.Ct, j.Ut, err);
}

}  // namespace

size_t spd_inverse_batch_work(int32_t nviews, const int32_t *kp) {
  size_t total = 0;
  for (int32_t v = 0; v < nviews; ++v) total += (size_t)512 * kp[v] + 128 * 128;
  return total + 64;
}

int spd_inverse_batch_f32(pprviz_ctx *ctx, int32_t nviews, const int32_t *kp, float *const *A, float *work) {
  using namespace tc;
  std::vector<FacJob> jobs((size_t)nviews);
  size_t o = 0;
  int maxnb = 0;
  double flops = 0.0;
  for (int32_t v = 0; v < nviews; ++v) {
    const int nblk = kp[v] / 128;
    jobs[v] = FacJob{A[v], work + o, work + o + (size_t)256 * kp[v], work + o + (size_t)512 * kp[v], kp[v], nblk};
    o += (size_t)512 * kp[v] + 128 * 128;
    maxnb = std::max(maxnb, nblk);
    const double b3 = 128.0 * 128.0 * 128.0, nm1 = nblk - 1.0;
    flops += nblk * (2.0 * b3 + nm1 * 2.0 * b3 + nm1 * (nm1 + 1.0) / 2.0 * 2.0 * b3);
  }
  ctx->stats.flops_factor += flops;
  int *err = reinterpret_cast<int *>(work + o);
  // per step: the views with the pivot (all), those with panels and a trailing
  // update (more than one block), and the launches' offsets
  struct StepTab { size_t act_all, act_multi, pan, trl; int nall, nmulti, npan, ntrl; };
  std::vector<StepTab> steps((size_t)maxnb);
  std::vector<int> tab;
  for (int kb = 0; kb < maxnb; ++kb) {
    StepTab &st = steps[kb];
    st.act_all = tab.size();
    for (int32_t v = 0; v < nviews; ++v)
      if (jobs[v].nblk > kb) tab.push_back(v);
    st.nall = (int)(tab.size() - st.act_all);
    st.act_multi = tab.size();
    for (int32_t v = 0; v < nviews; ++v)
      if (jobs[v].nblk > kb && jobs[v].nblk > 1) tab.push_back(v);
    st.nmulti = (int)(tab.size() - st.act_multi);
    st.pan = tab.size();
    int acc = 0;
    for (int q = 0; q < st.nmulti; ++q) {
      tab.push_back(acc);
      acc += jobs[tab[st.act_multi + q]].nblk;
    }
    tab.push_back(acc);
    st.npan = acc;
    st.trl = tab.size();
    acc = 0;
    for (int q = 0; q < st.nmulti; ++q) {
      tab.push_back(acc);
      const int nb = jobs[tab[st.act_multi + q]].nblk;
      acc += nb * (nb + 1) / 2;
    }
    tab.push_back(acc);
    st.ntrl = acc;
  }
  const size_t jb = (sizeof(FacJob) * jobs.size() + 255) & ~(size_t)255;
  PPRVIZ_TRY(ws_ensure(ctx, WS_FACT, jb + sizeof(int) * tab.size()));
  FacJob *jobs_d = ctx->ws[WS_FACT].as<FacJob>();
  int *tab_d = reinterpret_cast<int *>(static_cast<unsigned char *>(ctx->ws[WS_FACT].p) + jb);
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(jobs_d, jobs.data(), sizeof(FacJob) * jobs.size(), cudaMemcpyHostToDevice,
                                   ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(tab_d, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice, ctx->stream));
  const size_t panel_smem = sizeof(float) * (128 * 128 + 128 * (128 + 4));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_panel_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_diag128_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        DIAG128_SMEM));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)SMEM));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  {
    PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR);
    for (int kb = 0; kb < maxnb; ++kb) {
      const StepTab &st = steps[kb];
      const int32_t K0 = kb * 128;
      k_fac_diag128_batch<<<(unsigned)st.nall, DIAG128_THREADS, DIAG128_SMEM, ctx->stream>>>(jobs_d, tab_d + st.act_all, K0);
      PPRVIZ_LAUNCHED(ctx);
      if (st.nmulti == 0) continue;
      k_fac_panel_batch<<<(unsigned)st.npan, 256, panel_smem, ctx->stream>>>(jobs_d, tab_d + st.act_multi,
                                                                              tab_d + st.pan, st.nmulti, K0);
      PPRVIZ_LAUNCHED(ctx);
      k_fac_trailing_tc_batch<<<(unsigned)st.ntrl, 256, SMEM, ctx->stream>>>(jobs_d, tab_d + st.act_multi,
                                                                             tab_d + st.trl, st.nmulti, kb, err);
      PPRVIZ_LAUNCHED(ctx);
    }
    for (int32_t v = 0; v < nviews; ++v) {
      k_fac_finish<float, 128><<<dim3((unsigned)std::min(8, (kp[v] + 255) / 256), (unsigned)kp[v]), 256, 0,
                                 ctx->stream>>>(kp[v], A[v]);
      PPRVIZ_LAUNCHED(ctx);
    }
  }
  int herr = 0;
  PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
  if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "tensor-core trailing update: MMA completion wait expired");
  return PPRVIZ_OK;
}

}  // namespace pprviz
