// P5 - inverse of the SPD matrix A = L^w + J/k for the Guttman solve of Eq. (10).
//
// Symmetric block sweep (Gauss-Jordan on an SPD matrix, no pivoting needed).
// With P = A_KK^-1 for pivot block K:
//   A_KK -> -P,   A_IK -> A_IK P (and A_KI -> P A_KI),   A_IJ -> A_IJ - A_IK P A_KJ;
// the matrix stays symmetric after every sweep and equals -A^-1 once every
// block has been swept. Only the upper block triangle (64 x 64 blocks I <= J,
// diagonal blocks in full) is stored and updated, which halves the O(k^3)
// trailing work. A final pass negates it and mirrors the lower 64-blocks that
// lie inside the 128 x 128 diagonal tiles read by the layout passes.
#include <math.h>

#include "common.cuh"

namespace pprviz {

constexpr int FNB = 64;  // pivot block

// P = A_KK^-1 by an in-place scalar sweep of the 64 x 64 block in shared memory
// (ping-pong buffers, one barrier per pivot); writes P to `P` and -P into A_KK.
template <typename T>
__global__ void __launch_bounds__(512) k_fac_diag(int32_t kp, int32_t K0, T *__restrict__ A, T *__restrict__ P) {
  extern __shared__ unsigned char smem_raw[];
  T *buf = reinterpret_cast<T *>(smem_raw);  // [2][FNB][FNB + 1]
  constexpr int LD = FNB + 1, SZ = FNB * LD;
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    const int r = e / FNB, c = e % FNB;
    buf[r * LD + c] = A[(int64_t)(K0 + r) * kp + K0 + c];
  }
  __syncthreads();
  int cur = 0;
  for (int p = 0; p < FNB; ++p) {
    const T *a = buf + cur * SZ;
    T *b = buf + (cur ^ 1) * SZ;
    const T piv = T(1) / a[p * LD + p];
    for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
      const int r = e / FNB, c = e % FNB;
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
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    const int r = e / FNB, c = e % FNB;
    const T v = a[r * LD + c];
    P[e] = v;
    A[(int64_t)(K0 + r) * kp + K0 + c] = -v;
  }
}

// Panel of pivot block K for block I != K (64 rows): C_I = A_IK (from the
// stored upper triangle: A[i][K0 + t] for I < K, A[K0 + t][i] for I > K),
// U_I = C_I P. Writes Ct[t][i] = C_I, Ut[t][i] = U_I and stores U_I back as
// the new panel (A_IK for I < K, A_KI = U_I^T for I > K).
template <typename T>
__global__ void __launch_bounds__(256) k_fac_panel(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ P,
                                                   T *__restrict__ Ct, T *__restrict__ Ut) {
  const int I0 = blockIdx.x * FNB;
  if (I0 == K0) return;
  extern __shared__ unsigned char smem_raw[];
  T *sP = reinterpret_cast<T *>(smem_raw);  // [FNB][FNB]
  T *sC = sP + FNB * FNB;                   // [FNB][FNB + 1]  sC[i][t]
  constexpr int LD = FNB + 1;
  const bool above = I0 < K0;
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    sP[e] = P[e];
    const int r = e / FNB, c = e % FNB;
    if (above) sC[r * LD + c] = A[(int64_t)(I0 + r) * kp + K0 + c];   // i = r, t = c
    else sC[c * LD + r] = A[(int64_t)(K0 + r) * kp + I0 + c];         // t = r, i = c
  }
  __syncthreads();
  for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
    const int t = e / FNB, i = e % FNB;  // consecutive threads: consecutive i
    T u = T(0);
#pragma unroll 8
    for (int s = 0; s < FNB; ++s) u += sC[i * LD + s] * sP[s * FNB + t];
    Ct[(int64_t)t * kp + I0 + i] = sC[i * LD + t];
    Ut[(int64_t)t * kp + I0 + i] = u;
    if (!above) A[(int64_t)(K0 + t) * kp + I0 + i] = u;
  }
  if (above) {
    __syncthreads();
    // A[I0 + i][K0 + t] = U[i][t]: reuse sC for a coalesced row-major store
    for (int e = threadIdx.x; e < FNB * FNB; e += blockDim.x) {
      const int i = e / FNB, t = e % FNB;
      T u = T(0);
#pragma unroll 8
      for (int s = 0; s < FNB; ++s) u += sC[i * LD + s] * sP[s * FNB + t];
      A[(int64_t)(I0 + i) * kp + K0 + t] = u;
    }
  }
}

// Trailing update of the upper triangle: A[i][j] -= sum_t Ct[t][i] Ut[t][j] for
// i, j outside the pivot block with block(i) <= block(j) (64-blocks). TM x TM
// tiles over the upper tile triangle; R x R outputs per thread in two
// SUB x SUB quadrants so that shared-memory reads are vectors.
template <typename T, int TM>
__global__ void __launch_bounds__(256)
k_fac_trailing(int32_t kp, int32_t K0, T *__restrict__ A, const T *__restrict__ Ct, const T *__restrict__ Ut) {
  constexpr int R = TM / 16, SUB = R / 2, HALF = TM / 2;
  const int I0 = blockIdx.y * TM, J0 = blockIdx.x * TM;
  if (J0 < I0) return;  // lower tile triangle: not stored
  if ((I0 >= K0 && I0 + TM <= K0 + FNB) || (J0 >= K0 && J0 + TM <= K0 + FNB)) return;
  extern __shared__ unsigned char smem_raw[];
  T *sA = reinterpret_cast<T *>(smem_raw);  // [FNB][TM]  sA[t][i] = Ct[t][I0 + i]
  T *sB = sA + FNB * TM;                    // [FNB][TM]  sB[t][j] = Ut[t][J0 + j]
  for (int e = threadIdx.x; e < FNB * TM; e += 256) {
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
  for (int t = 0; t < FNB; ++t) {
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
  // Epilogue: each row's SUB consecutive columns are one aligned vector; the
  // masks (pivot block, lower blocks, kp) are uniform over it since blocks are
  // 64-aligned and kp is a multiple of 128.
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int i = I0 + (r / SUB) * HALF + ty * SUB + (r % SUB);
    if (i >= kp || (i >= K0 && i < K0 + FNB)) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = J0 + h * HALF + tx * SUB;
      if (j >= kp || (j >= K0 && j < K0 + FNB) || (i / FNB) > (j / FNB)) continue;
      T *p = A + (int64_t)i * kp + j;
      if constexpr (sizeof(T) == 4 && SUB == 4) {
        float4 v = *reinterpret_cast<float4 *>(p);
        v.x -= acc[r][h * SUB + 0];
        v.y -= acc[r][h * SUB + 1];
        v.z -= acc[r][h * SUB + 2];
        v.w -= acc[r][h * SUB + 3];
        *reinterpret_cast<float4 *>(p) = v;
      } else {
#pragma unroll
        for (int s = 0; s < SUB; ++s) p[s] -= acc[r][h * SUB + s];
      }
    }
  }
}

// A <- -A on the upper block triangle, and the lower 64-block of every 128 x 128
// diagonal tile filled from its mirror, giving M = A^-1 where the layout reads it.
template <typename T>
__global__ void k_fac_finish(int32_t kp, T *__restrict__ A) {
  const int64_t i = blockIdx.y;
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < kp; j += (int64_t)gridDim.x * blockDim.x) {
    if (i / FNB > j / FNB) continue;
    const T v = -A[i * kp + j];
    A[i * kp + j] = v;
    if (i / 128 == j / 128 && i / FNB < j / FNB) A[j * kp + i] = v;
  }
}

template <typename T>
static int spd_inverse(pprviz_ctx *ctx, int32_t kp, T *A, T *work) {
  constexpr int TM = sizeof(T) == 4 ? 128 : 64;
  T *Ct = work, *Ut = work + (size_t)FNB * kp, *P = work + (size_t)2 * FNB * kp;
  const size_t diag_smem = 2 * sizeof(T) * FNB * (FNB + 1);
  const size_t panel_smem = sizeof(T) * (FNB * FNB + FNB * (FNB + 1));
  const size_t trail_smem = 2 * sizeof(T) * FNB * TM;
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing<T, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)trail_smem));
  const int nblk = kp / FNB;
  const unsigned tgrid = (unsigned)((kp + TM - 1) / TM);
  // per pivot: the 64^3 pivot inverse, (nblk - 1) panel products of 2 * 64^3,
  // and 2 * 64 flops for each of the (nblk - 1) nblk / 2 upper blocks of 64^2
  const double b3 = (double)FNB * FNB * FNB;
  const double nm1 = (double)(nblk - 1);
  ctx->stats.flops_factor += (double)nblk * (2.0 * b3 + nm1 * 2.0 * b3 + nm1 * (nm1 + 1.0) / 2.0 * 2.0 * b3);
  for (int kb = 0; kb < nblk; ++kb) {
    const int K0 = kb * FNB;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_diag<T><<<1, 512, diag_smem, ctx->stream>>>(kp, K0, A, P); }
    PPRVIZ_LAUNCHED(ctx);
    if (nblk == 1) break;
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_panel<T><<<nblk, 256, panel_smem, ctx->stream>>>(kp, K0, A, P, Ct, Ut); }
    PPRVIZ_LAUNCHED(ctx);
    { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_trailing<T, TM><<<dim3(tgrid, tgrid), 256, trail_smem, ctx->stream>>>(kp, K0, A, Ct, Ut); }
    PPRVIZ_LAUNCHED(ctx);
  }
  { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_finish<T><<<dim3((unsigned)std::min(8, (kp + 255) / 256), (unsigned)kp), 256, 0, ctx->stream>>>(kp, A); }
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

int spd_inverse_f32(pprviz_ctx *ctx, int32_t kp, float *A, float *work) { return spd_inverse<float>(ctx, kp, A, work); }
int spd_inverse_f64(pprviz_ctx *ctx, int32_t kp, double *A, double *work) {
  return spd_inverse<double>(ctx, kp, A, work);
}

}  // namespace pprviz
