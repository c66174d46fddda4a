// P3 - PDist (Sec. 3.1, Eq. (1)):
//   Delta[i][j] = min(max(1 - ln(z_ij), 2), 2 ln n_clamp),  z_ij = pi_d(i,j) + pi_d(j,i),
// with the natural logarithm, z <= 0 mapped to the upper clamp, and a zero
// diagonal. Each block owns one 32x32 output tile; the mirrored input tile
// is staged transposed in shared memory so every global access is coalesced.
#include <math.h>

#include "common.cuh"

namespace pprviz {

template <typename T>
__device__ __forceinline__ T pdist_of(T z, double upper);

template <>
__device__ __forceinline__ float pdist_of<float>(float z, double upper) {
  float raw;
  if (!(z > 0.0f)) raw = INFINITY;
  else if (z < 1e-30f) raw = (float)(1.0 - log((double)z));  // log of tiny z taken in FP64
  else raw = 1.0f - logf(z);
  return fminf(fmaxf(raw, 2.0f), (float)upper);
}
template <>
__device__ __forceinline__ double pdist_of<double>(double z, double upper) {
  double raw = (z > 0.0) ? 1.0 - log(z) : INFINITY;
  return fmin(fmax(raw, 2.0), upper);
}

template <typename T>
__global__ void k_pdist(int32_t k, const T *__restrict__ D, T *__restrict__ out, double upper) {
  __shared__ T tr[32][33];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  // tr[jj][ii] = D[j0 + jj][i0 + ii]  (the mirrored tile)
  for (int jj = ty; jj < 32; jj += 8) {
    const int j = j0 + jj, i = i0 + tx;
    tr[jj][tx] = (j < k && i < k) ? D[(int64_t)j * k + i] : T(0);
  }
  __syncthreads();
  for (int ii = ty; ii < 32; ii += 8) {
    const int i = i0 + ii, j = j0 + tx;
    if (i < k && j < k) {
      const T z = D[(int64_t)i * k + j] + tr[tx][ii];
      out[(int64_t)i * k + j] = (i == j) ? T(0) : pdist_of<T>(z, upper);
    }
  }
}

int pdist_launch(pprviz_ctx *ctx, const void *dppr_d, int32_t k, int64_t n_clamp, void *pdist_d, bool f64) {
  const double upper = 2.0 * log((double)n_clamp);
  dim3 grid((unsigned)((k + 31) / 32), (unsigned)((k + 31) / 32));
  dim3 block(32, 8);
  if (f64)
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PDIST); k_pdist<double><<<grid, block, 0, ctx->stream>>>(k, (const double *)dppr_d, (double *)pdist_d, upper); }
  else
    { PPRVIZ_PROF(ctx, PPRVIZ_K_PDIST); k_pdist<float><<<grid, block, 0, ctx->stream>>>(k, (const float *)dppr_d, (float *)pdist_d, upper); }
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

}  // namespace pprviz
