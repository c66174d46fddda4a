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

#include <algorithm>
#include <type_traits>

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

// ---------------------------------------------------------------------------
// Tensor-core trailing update (FP32 path): the same A[i][j] -= sum_t
// Ct[t][i] Ut[t][j] on 128 x 128 tiles, as tcgen05.mma kind::tf32 products
// with split operands (x = x_hi + x_lo, x_hi = x with the low 13 mantissa bits
// cleared): C ~ A_hi B_hi + A_hi B_lo + A_lo B_hi (error-compensated TF32,
// Ootomo & Yokota 2022), FP32 accumulation in tensor memory.
// Operands are staged by the CTA into the canonical no-swizzle K-major shared
// layout (8-row x 16-byte core matrices, LBO = 128 B along K, SBO = 16 core
// matrices per 8-row group); one thread issues the 24 MMAs and commits them to
// an mbarrier, which every thread waits on with an iteration limit (on expiry
// the CTA sets `err`, skips the update and still frees its tensor memory).
// ---------------------------------------------------------------------------
namespace tc {
constexpr int TM = 128;                       // tile edge (M = N = 128)
constexpr int KD = FNB;                       // inner dimension (pivot block)
constexpr uint32_t LBO = 128;                 // bytes to the next core matrix along K
constexpr uint32_t SBO = (KD / 4) * 128;      // bytes to the next 8-row group
constexpr int OPB = TM * KD * 4;              // bytes of one staged operand (32 KiB)
constexpr int SMEM = 4 * OPB;                 // A_hi, A_lo, B_hi, B_lo
constexpr long WAIT_LIMIT = 1L << 22;         // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint32_t canon(int r, int k) {
  return (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor, kind::tf32: F32 accumulate, TF32 A and B, both K-major
constexpr uint32_t IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TM >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ float hi_part(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }
}  // namespace tc

__global__ void __launch_bounds__(256)
k_fac_trailing_tc(int32_t kp, int32_t K0, float *__restrict__ A, const float *__restrict__ Ct,
                  const float *__restrict__ Ut, int *__restrict__ err) {
  using namespace tc;
  const int I0 = blockIdx.y * TM, J0 = blockIdx.x * TM;
  if (J0 < I0) return;  // lower tile triangle: not stored
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  unsigned char *sAh = smem_raw, *sAl = smem_raw + OPB, *sBh = smem_raw + 2 * OPB, *sBl = smem_raw + 3 * OPB;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // Epilogue ownership: warp w updates tile rows 32 (w % 4) + lane (its TMEM
  // lanes) and columns 64 (w / 4) .. +63. Those 64 values of A are read from
  // HBM first, so their latency overlaps the staging and the MMAs.
  const int lg = warp & 3, ch = warp >> 2;
  const int i_row = I0 + 32 * lg + lane;
  const bool row_ok = !(i_row >= K0 && i_row < K0 + FNB);
  float4 pre[16];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int j = J0 + 64 * ch + 8 * c;
    const bool ok = row_ok && !(j >= K0 && j < K0 + FNB) && (i_row / FNB) <= (j / FNB);
    const float4 *p = reinterpret_cast<const float4 *>(A + (int64_t)i_row * kp + j);
    pre[2 * c] = ok ? p[0] : make_float4(0.f, 0.f, 0.f, 0.f);
    pre[2 * c + 1] = ok ? p[1] : make_float4(0.f, 0.f, 0.f, 0.f);
  }
  // stage: thread (row r, quad q of 4 inner indices) reads Ct[4q .. 4q+3][I0 + r]
  // (coalesced across the warp) and writes one 16-byte chunk per operand part
  static_assert((TM * (KD / 4)) % 256 == 0, "staging assumes 256 threads");
#pragma unroll 4
  for (int it = 0; it < TM * (KD / 4) / 256; ++it) {
    const int idx = tid + 256 * it;
    const int r = idx % TM, q = idx / TM;
    float a[4], b[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      a[s] = Ct[(int64_t)(4 * q + s) * kp + I0 + r];
      b[s] = Ut[(int64_t)(4 * q + s) * kp + J0 + r];
    }
    float4 ah, al, bh, bl;
    ah.x = hi_part(a[0]); ah.y = hi_part(a[1]); ah.z = hi_part(a[2]); ah.w = hi_part(a[3]);
    al.x = a[0] - ah.x; al.y = a[1] - ah.y; al.z = a[2] - ah.z; al.w = a[3] - ah.w;
    bh.x = hi_part(b[0]); bh.y = hi_part(b[1]); bh.z = hi_part(b[2]); bh.w = hi_part(b[3]);
    bl.x = b[0] - bh.x; bl.y = b[1] - bh.y; bl.z = b[2] - bh.z; bl.w = b[3] - bh.w;
    const uint32_t o = canon(r, 4 * q);
    *reinterpret_cast<float4 *>(sAh + o) = ah;
    *reinterpret_cast<float4 *>(sAl + o) = al;
    *reinterpret_cast<float4 *>(sBh + o) = bh;
    *reinterpret_cast<float4 *>(sBl + o) = bl;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)), "r"(TM));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  if (tid == 0) {
    int first = 1;
#pragma unroll 1
    for (int pass = 0; pass < 3; ++pass) {
      const unsigned char *pa = (pass == 2) ? sAl : sAh;
      const unsigned char *pb = (pass == 1) ? sBl : sBh;
#pragma unroll 1
      for (int ks = 0; ks < KD / 8; ++ks) {
        const uint64_t da = desc(smem_u32(pa) + ks * 2 * LBO);
        const uint64_t db = desc(smem_u32(pb) + ks * 2 * LBO);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(IDESC), "r"(first ? 0u : 1u));
        first = 0;
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(&mbar)));
  }
  uint32_t done = 0;
  for (long it = 0; it < WAIT_LIMIT && !done; ++it) {
    asm volatile(
        "{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], 0;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(&mbar))
        : "memory");
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!done) {
    if (lane == 0) atomicOr(err, 1);
  } else {
    // the warp's 32 lanes x 64 columns of the product, 4 x 16 columns per load
    uint32_t v[64];
    const uint32_t tbase = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)(64 * ch);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[16 * q + 0]), "=r"(v[16 * q + 1]), "=r"(v[16 * q + 2]), "=r"(v[16 * q + 3]), "=r"(v[16 * q + 4]),
            "=r"(v[16 * q + 5]), "=r"(v[16 * q + 6]), "=r"(v[16 * q + 7]), "=r"(v[16 * q + 8]), "=r"(v[16 * q + 9]),
            "=r"(v[16 * q + 10]), "=r"(v[16 * q + 11]), "=r"(v[16 * q + 12]), "=r"(v[16 * q + 13]),
            "=r"(v[16 * q + 14]), "=r"(v[16 * q + 15])
          : "r"(tbase + (uint32_t)(16 * q)));
    }
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int j = J0 + 64 * ch + 8 * c;
      if (!row_ok || (j >= K0 && j < K0 + FNB) || (i_row / FNB) > (j / FNB)) continue;
      float4 *p = reinterpret_cast<float4 *>(A + (int64_t)i_row * kp + j);
      float4 x = pre[2 * c], y = pre[2 * c + 1];
      x.x -= __uint_as_float(v[8 * c + 0]); x.y -= __uint_as_float(v[8 * c + 1]);
      x.z -= __uint_as_float(v[8 * c + 2]); x.w -= __uint_as_float(v[8 * c + 3]);
      y.x -= __uint_as_float(v[8 * c + 4]); y.y -= __uint_as_float(v[8 * c + 5]);
      y.z -= __uint_as_float(v[8 * c + 6]); y.w -= __uint_as_float(v[8 * c + 7]);
      p[0] = x;
      p[1] = y;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TM));
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
  constexpr bool TC = std::is_same<T, float>::value;  // FP32: tensor-core trailing update
  T *Ct = work, *Ut = work + (size_t)FNB * kp, *P = work + (size_t)2 * FNB * kp;
  int *err = reinterpret_cast<int *>(P + FNB * FNB);
  const size_t diag_smem = 2 * sizeof(T) * FNB * (FNB + 1);
  const size_t panel_smem = sizeof(T) * (FNB * FNB + FNB * (FNB + 1));
  const size_t trail_smem = TC ? (size_t)tc::SMEM : 2 * sizeof(T) * FNB * TM;
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_diag<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)diag_smem));
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_panel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)panel_smem));
  if constexpr (TC) {
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)trail_smem));
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  } else {
    PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_fac_trailing<T, TM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)trail_smem));
  }
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
    if constexpr (TC) {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_trailing_tc<<<dim3(tgrid, tgrid), 256, trail_smem, ctx->stream>>>(kp, K0, A, Ct, Ut, err); }
    } else {
      { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_trailing<T, TM><<<dim3(tgrid, tgrid), 256, trail_smem, ctx->stream>>>(kp, K0, A, Ct, Ut); }
    }
    PPRVIZ_LAUNCHED(ctx);
  }
  { PPRVIZ_PROF(ctx, PPRVIZ_K_FACTOR); k_fac_finish<T><<<dim3((unsigned)std::min(8, (kp + 255) / 256), (unsigned)kp), 256, 0, ctx->stream>>>(kp, A); }
  PPRVIZ_LAUNCHED(ctx);
  if constexpr (TC) {
    int herr = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (herr) return set_err(ctx, PPRVIZ_E_TIMEOUT, "tensor-core trailing update: MMA completion wait expired");
  }
  return PPRVIZ_OK;
}

int spd_inverse_f32(pprviz_ctx *ctx, int32_t kp, float *A, float *work) { return spd_inverse<float>(ctx, kp, A, work); }
int spd_inverse_f64(pprviz_ctx *ctx, int32_t kp, double *A, double *work) {
  return spd_inverse<double>(ctx, kp, A, work);
}

}  // namespace pprviz
