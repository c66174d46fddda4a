// P1d - propagation sweeps on the tensor cores for dense views.
//
// When a view's walk matrix is dense (a weighted supergraph view), one sweep
// of the propagation over a group of G sources is a true dense contraction:
// in the degree-scaled node-major state of the sparse path (y = x / dw,
// [n][G]), (x P)_j = sum_i w_ij y_i for every source column, i.e.
//   ACC = W Y   (W the n x n symmetric weight matrix, Y the n x G state),
// 2 n^2 G flop per sweep (Sec. 3.1 in matrix form). The sweep then applies
// the same update as the CSR sweep,
//   y_out = om1 * y_old + om * (b + c * ACC) / dw,
// so the Chebyshev recurrence, the FP64 residual certificate and the
// refinement passes of the sparse path are reused unchanged; only the
// gather sweep is replaced.
//
// Arithmetic: tcgen05.mma kind::tf32 with split operands (x = hi + lo, hi = x
// with its low 13 mantissa bits cleared, lo = x - hi exactly;
// W Y ~ W_hi Y_hi + W_hi Y_lo + W_lo Y_hi, the error-compensated TF32 scheme
// of Ootomo & Yokota 2022), accumulated in FP32 in tensor memory: FP32-level
// products, which is what the sweeps need (the certificate comes from the
// FP64 residual over the CSR, not from these products).
//
// BF16 mode (PPRVIZ_FP32_BF16TC): the same sweep with the operands rounded to
// BF16 while they are staged (W and Y each to 8 significant bits) and one
// tcgen05.mma kind::f16 (BF16 x BF16, FP32 accumulation in tensor memory)
// per 16-wide inner step instead of the three TF32 products. A sweep is then
// accurate to ~2^-9 of its products only; the refinement passes, driven by
// the same FP64 residual over the CSR, restore the eps bound (each pass
// gains what one BF16 solve resolves).
//
// Tiling: one CTA per 128 (target rows j) x NT (sources q) output tile, the
// inner dimension i streamed in 32-wide chunks through two shared-memory
// stages. Both operands are staged K-major in the canonical no-swizzle layout
// (8-row x 16-byte core matrices): W rows are K-contiguous in memory; the state
// Y[i][q] is source-contiguous and is transposed while staging (lanes run over
// q, each thread packs 4 consecutive i). The global loads of chunk c + 1 are
// issued before the MMAs of chunk c are waited on, and every mbarrier wait has
// an iteration limit: on expiry the CTA sets the error word, skips its output
// and still frees its tensor memory.
#include <math.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "common.cuh"

namespace pprviz {

namespace dtc {
constexpr int TM = 128;                  // target rows per tile (MMA M)
constexpr int KC = 32;                   // inner-dimension chunk per stage
constexpr uint32_t LBO = 128;            // bytes to the next core matrix along K
constexpr int THREADS = 256;
constexpr long WAIT_LIMIT = 1L << 22;

// BF: BF16 operands (2 bytes, one product per step), else split TF32 (4 bytes,
// high and low parts: three products per step).
template <int NT, bool BF>
struct Cfg {
  static constexpr int EB = BF ? 2 : 4;                  // operand element bytes
  static constexpr uint32_t SBO = (KC * EB / 16) * 128;  // bytes to the next 8-row group
  static constexpr int A_BYTES = TM * KC * EB;  // one (split part of the) W chunk
  static constexpr int B_BYTES = NT * KC * EB;  // one (split part of the) Y chunk
  static constexpr int STAGE = BF ? A_BYTES + B_BYTES : 2 * A_BYTES + 2 * B_BYTES;
  // a CTA holds NT tensor-memory columns, so at most 512 / NT CTAs fit on an
  // SM; the BF16 stages are small, so their request is padded to keep the
  // scheduler from placing more CTAs than that (232,448 bytes per SM)
  static constexpr int MAXC = 512 / NT;
  static constexpr int SMEM = BF ? (2 * STAGE > 232448 / (MAXC + 1) + 1024 ? 2 * STAGE : 232448 / (MAXC + 1) + 1024)
                                 : 2 * STAGE;
  static constexpr int B_ITEMS = NT * (KC / 4) / THREADS;  // float4 groups of Y per thread
  // kind::tf32: A, B format 2 (TF32); kind::f16: A, B format 1 (BF16); F32 accumulator
  static constexpr uint32_t IDESC = (1u << 4) | ((BF ? 1u : 2u) << 7) | ((BF ? 1u : 2u) << 10) |
                                    ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
  static constexpr int K_STEP = BF ? 16 : 8;  // inner extent of one MMA
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
// byte offset of element (row r, inner index k) in the canonical no-swizzle
// K-major layout: 8-row x 16-byte core matrices, LBO along K, SBO along rows
template <bool BF>
__device__ __forceinline__ uint32_t canon(int r, int k) {
  constexpr uint32_t SBO = (KC * (BF ? 2 : 4) / 16) * 128;
  return BF ? (uint32_t)((r >> 3) * SBO + (k >> 3) * LBO + (r & 7) * 16 + (k & 7) * 2)
            : (uint32_t)((r >> 3) * SBO + (k >> 2) * LBO + (r & 7) * 16 + (k & 3) * 4);
}
template <bool BF>
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  constexpr uint32_t SBO = (KC * (BF ? 2 : 4) / 16) * 128;
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((LBO >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((SBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ float hi_part(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

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

// four consecutive inner elements rounded to BF16 (round to nearest even), 8 bytes
__device__ __forceinline__ void put_bf16(unsigned char *dst, uint32_t off, float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t *>(&a);
  u.y = *reinterpret_cast<const uint32_t *>(&b);
  *reinterpret_cast<uint2 *>(dst + off) = u;
}

__device__ __forceinline__ void put_split(unsigned char *hi, unsigned char *lo, uint32_t off, float4 v) {
  float4 h, l;
  h.x = hi_part(v.x); h.y = hi_part(v.y); h.z = hi_part(v.z); h.w = hi_part(v.w);
  l.x = v.x - h.x; l.y = v.y - h.y; l.z = v.z - h.z; l.w = v.w - h.w;
  *reinterpret_cast<float4 *>(hi + off) = h;
  *reinterpret_cast<float4 *>(lo + off) = l;
}

// Raw operand values of one inner chunk, held in registers between the
// global loads and the split stores into a stage.
template <int NT>
struct Chunk {
  float4 a[4];                          // W: 128 rows x 32 -> 1024 float4, 4 per thread
  float4 b[Cfg<NT, false>::B_ITEMS];    // Y: NT sources x 8 quads of i
};

// W chunk mapping: 8 lanes of a warp cover 8 rows at one 16-byte column quad,
// the 4 lane octets 4 consecutive quads (64 contiguous bytes per row), which
// keeps the canonical-layout stores at the 4-wavefront minimum.
__device__ __forceinline__ void a_coords(int tid, int it, int &r, int &kq) {
  const int lane = tid & 31, w = tid >> 5;
  const int g = w * 4 + it;  // 0 .. 31
  r = 8 * (g >> 1) + (lane & 7);
  kq = 4 * (g & 1) + (lane >> 3);
}

template <int NT>
__device__ __forceinline__ void load_chunk(Chunk<NT> &ch, const float *__restrict__ W, int64_t nw, int64_t j0,
                                           const float *__restrict__ Y, int64_t ld, int64_t q0, int64_t n,
                                           int64_t k0, int tid) {
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    int r, kq;
    a_coords(tid, it, r, kq);
    ch.a[it] = __ldg(reinterpret_cast<const float4 *>(W + (j0 + r) * nw + k0 + 4 * kq));
  }
#pragma unroll
  for (int it = 0; it < Cfg<NT, false>::B_ITEMS; ++it) {
    const int item = tid + THREADS * it;
    const int q = item % NT, kq = item / NT;
    const int64_t i = k0 + 4 * kq;
    const float *p = Y + i * ld + q0 + q;
    float4 v;
    v.x = (i + 0 < n) ? __ldg(p) : 0.0f;
    v.y = (i + 1 < n) ? __ldg(p + ld) : 0.0f;
    v.z = (i + 2 < n) ? __ldg(p + 2 * ld) : 0.0f;
    v.w = (i + 3 < n) ? __ldg(p + 3 * ld) : 0.0f;
    ch.b[it] = v;
  }
}

template <int NT, bool BF>
__device__ __forceinline__ void store_chunk(const Chunk<NT> &ch, unsigned char *st, int tid) {
  using C = Cfg<NT, BF>;
  if (BF) {
    unsigned char *a = st, *b = st + C::A_BYTES;
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      int r, kq;
      a_coords(tid, it, r, kq);
      put_bf16(a, canon<true>(r, 4 * kq), ch.a[it]);
    }
#pragma unroll
    for (int it = 0; it < C::B_ITEMS; ++it) {
      const int item = tid + THREADS * it;
      put_bf16(b, canon<true>(item % NT, 4 * (item / NT)), ch.b[it]);
    }
    return;
  }
  unsigned char *a_hi = st, *a_lo = st + C::A_BYTES;
  unsigned char *b_hi = st + 2 * C::A_BYTES, *b_lo = b_hi + C::B_BYTES;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    int r, kq;
    a_coords(tid, it, r, kq);
    put_split(a_hi, a_lo, canon<false>(r, 4 * kq), ch.a[it]);
  }
#pragma unroll
  for (int it = 0; it < C::B_ITEMS; ++it) {
    const int item = tid + THREADS * it;
    put_split(b_hi, b_lo, canon<false>(item % NT, 4 * (item / NT)), ch.b[it]);
  }
}
}  // namespace dtc

// One Chebyshev sweep of a source group on the tensor cores:
//   ACC[j][q] = sum_i W[j][i] ycur[i][q]
//   yout[j][q] = om1 * yold[j][q] + om * (b_jq + c * ACC[j][q]) * invdw[j]
// with b_jq = alpha [j == src[q]], or rhs[j][q] when RHS. yout may alias
// yold (each element is read and written by the same thread).
// W: mw x nw FP32 (mw = n rounded up to 128, nw = n rounded up to 32, zero
// padded); the state has n rows of ld floats; grid (ld / NT, mw / 128).
template <int NT, bool RHS, bool BF>
__global__ void __launch_bounds__(dtc::THREADS, BF ? 2 : 1)
k_dsweep_tc(int64_t n, int64_t nw, int64_t ld, const float *__restrict__ W, const float *__restrict__ invdw,
            const int32_t *__restrict__ src, const float *__restrict__ rhs, const float *__restrict__ ycur,
            const float *yold, float *yout, float alpha, float c, float om, float om1, int *__restrict__ err) {
  using namespace dtc;
  using C = Cfg<NT, BF>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t q0 = (int64_t)blockIdx.x * NT, j0 = (int64_t)blockIdx.y * TM;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_sh)),
                 "r"(NT));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_sh;
  const int64_t nchunks = nw / KC;
  bool ok = true;
  int64_t issued = -1;  // last chunk whose MMAs were committed
  Chunk<NT> ch;
  load_chunk<NT>(ch, W, nw, j0, ycur, ld, q0, n, 0, tid);
  for (int64_t cidx = 0; cidx < nchunks; ++cidx) {
    const int buf = (int)(cidx & 1);
    unsigned char *st = smem_raw + buf * C::STAGE;
    // the MMAs of chunk cidx - 2 read this stage: wait for their commit
    if (cidx >= 2 && !mbar_wait(&mbar[buf], (uint32_t)(((cidx - 2) >> 1) & 1))) ok = false;
    if (__syncthreads_and(ok) == 0) {
      ok = false;
      break;
    }
    store_chunk<NT, BF>(ch, st, tid);
    if (cidx + 1 < nchunks) load_chunk<NT>(ch, W, nw, j0, ycur, ld, q0, n, (cidx + 1) * KC, tid);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0) {
      const uint32_t base = smem_u32(st);
      if (BF) {
        // one BF16 product per 16-wide inner step (32 bytes = two core matrices)
#pragma unroll
        for (int ks = 0; ks < KC / C::K_STEP; ++ks) {
          const uint64_t da = desc<true>(base + ks * 2 * LBO);
          const uint64_t db = desc<true>(base + C::A_BYTES + ks * 2 * LBO);
          const uint32_t acc = (cidx == 0 && ks == 0) ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(C::IDESC), "r"(acc));
        }
      } else {
#pragma unroll 1
      for (int pass = 0; pass < 3; ++pass) {
        // hi*hi, hi*lo (W_hi Y_lo), lo*hi (W_lo Y_hi)
        const uint32_t pa = base + (pass == 2 ? C::A_BYTES : 0);
        const uint32_t pb = base + 2 * C::A_BYTES + (pass == 1 ? C::B_BYTES : 0);
#pragma unroll
        for (int ks = 0; ks < KC / C::K_STEP; ++ks) {
          const uint64_t da = desc<false>(pa + ks * 2 * LBO);
          const uint64_t db = desc<false>(pb + ks * 2 * LBO);
          const uint32_t acc = (cidx == 0 && pass == 0 && ks == 0) ? 0u : 1u;
          asm volatile(
              "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
              "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
              "l"(da), "l"(db), "r"(C::IDESC), "r"(acc));
        }
      }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(&mbar[buf])));
    }
    issued = cidx;
  }
  // the commit of the last issued chunk covers every MMA this CTA issued
  if (ok && !mbar_wait(&mbar[issued & 1], (uint32_t)((issued >> 1) & 1))) ok = false;
  ok = __syncthreads_and(ok) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (!ok) {
    if (tid == 0) {
      atomicOr(err, 1);
      // give MMAs still in flight a second bounded wait before the tensor
      // memory is released
      if (issued >= 0) (void)mbar_wait(&mbar[issued & 1], (uint32_t)((issued >> 1) & 1));
    }
  } else {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows j) and the column half w / 4
    const int lg = warp & 3, half = warp >> 2;
    const int64_t j = j0 + 32 * lg + lane;
    const bool valid = j < n;
    const float invd = valid ? invdw[j] : 0.0f;
#pragma unroll 1
    for (int cb = 0; cb < NT / 2; cb += 32) {
      const int col0 = half * (NT / 2) + cb;
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * lg) << 16) + (uint32_t)col0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(taddr));
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
            "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
            "=r"(v[30]), "=r"(v[31])
          : "r"(taddr + 16u));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (valid) {
        const int64_t q = q0 + col0;
        const int64_t off = j * ld + q;
#pragma unroll
        for (int t4 = 0; t4 < 8; ++t4) {
          const float4 o = *reinterpret_cast<const float4 *>(yold + off + 4 * t4);
          float4 bq;
          if (RHS) {
            bq = __ldg(reinterpret_cast<const float4 *>(rhs + off + 4 * t4));
          } else {
            const int4 s4 = __ldg(reinterpret_cast<const int4 *>(src + q + 4 * t4));
            bq.x = (s4.x == (int32_t)j) ? alpha : 0.0f;
            bq.y = (s4.y == (int32_t)j) ? alpha : 0.0f;
            bq.z = (s4.z == (int32_t)j) ? alpha : 0.0f;
            bq.w = (s4.w == (int32_t)j) ? alpha : 0.0f;
          }
          float4 r;
          r.x = om1 * o.x + om * ((bq.x + c * __uint_as_float(v[4 * t4 + 0])) * invd);
          r.y = om1 * o.y + om * ((bq.y + c * __uint_as_float(v[4 * t4 + 1])) * invd);
          r.z = om1 * o.z + om * ((bq.z + c * __uint_as_float(v[4 * t4 + 2])) * invd);
          r.w = om1 * o.w + om * ((bq.w + c * __uint_as_float(v[4 * t4 + 3])) * invd);
          *reinterpret_cast<float4 *>(yout + off + 4 * t4) = r;
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

// W[j][col] = w_j,col (1 on unweighted graphs); W[j][j] = 1 for a node without
// edges (its walk stays put). W is zeroed beforehand. One warp per row.
__global__ void k_dense_w(int64_t n, int64_t nw, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                          const float *__restrict__ w, float *__restrict__ W) {
  const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (j >= n) return;
  const int64_t b = rp[j], e = rp[j + 1];
  if (b == e) {
    if (lane == 0) W[j * nw + j] = 1.0f;
    return;
  }
  for (int64_t p = b + lane; p < e; p += 32) W[j * nw + col[p]] = w ? w[p] : 1.0f;
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------

bool dense_eligible(const pprviz_graph *g) {
  // a dense contraction pays once the view holds ~5 % of all pairs: one
  // tensor-core sweep costs ~6 n^2 G flop at ~1 PFLOP/s, a CSR sweep gathers
  // nnz G 4-byte values at L2 speed (~10 TB/s); above 5 % the former wins
  // by more than 1.5x
  return !g->directed && g->n >= 512 && (double)g->nnz >= 0.05 * (double)g->n * (double)g->n;
}

int64_t dense_group(int32_t k) {
  // wide groups keep the grid's last wave nearly full (152 SMs, one CTA each)
  const int64_t kk = ((int64_t)k + 127) / 128 * 128;
  return std::min<int64_t>(kk, 2048);
}

int dense_prepare(pprviz_ctx *ctx, const pprviz_graph *g) {
  const int64_t n = g->n;
  const int64_t nw = (n + 31) / 32 * 32, mw = (n + 127) / 128 * 128;
  if (g->dense.p && g->dense_nw == nw) return PPRVIZ_OK;
  const size_t bytes = sizeof(float) * (size_t)mw * (size_t)nw;
  cudaError_t e = g->dense.ensure(bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    g->dense.release();
    return set_err(ctx, PPRVIZ_E_OOM, "dense weight matrix for the tensor-core sweeps does not fit");
  }
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(g->dense.p, 0, bytes, ctx->stream));
  {
    PPRVIZ_PROF(ctx, PPRVIZ_K_OTHER);
    k_dense_w<<<(unsigned)((n * 32 + 255) / 256), 256, 0, ctx->stream>>>(
        n, nw, g->rp.as<int64_t>(), g->col.as<int32_t>(), g->weighted ? g->w.as<float>() : nullptr,
        g->dense.as<float>());
  }
  PPRVIZ_LAUNCHED(ctx);
  g->dense_nw = nw;
  return PPRVIZ_OK;
}

template <int NT, bool RHS, bool BF>
static int dsweep_launch(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src,
                         const float *rhs, const float *ycur, float *yold, double alpha, double om, int *err) {
  using C = dtc::Cfg<NT, BF>;
  PPRVIZ_CUDA(ctx, cudaFuncSetAttribute(k_dsweep_tc<NT, RHS, BF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        C::SMEM));
  const int64_t mw = (g->n + 127) / 128 * 128;
  const dim3 grid((unsigned)(ld / NT), (unsigned)(mw / dtc::TM));
  const double c = 1.0 - alpha;
  PPRVIZ_PROF(ctx, PPRVIZ_K_SWEEP);
  k_dsweep_tc<NT, RHS, BF><<<grid, dtc::THREADS, C::SMEM, ctx->stream>>>(
      g->n, g->dense_nw, ld, g->dense.as<float>(), g->invdw_f.as<float>(), src, rhs, ycur, yold, yold,
      (float)alpha, (float)c, (float)om, (float)(1.0 - om), err);
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

template <bool BF>
static int dense_sweep_t(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src, const float *rhs,
                         const float *ycur, float *yold, double alpha, double om, int *err) {
  if (ld % 256 == 0)
    return rhs ? dsweep_launch<256, true, BF>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err)
               : dsweep_launch<256, false, BF>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err);
  return rhs ? dsweep_launch<128, true, BF>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err)
             : dsweep_launch<128, false, BF>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err);
}

int dense_sweep(pprviz_ctx *ctx, const pprviz_graph *g, int64_t ld, const int32_t *src, const float *rhs,
                const float *ycur, float *yold, double alpha, double om, int *err, bool bf16) {
  return bf16 ? dense_sweep_t<true>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err)
              : dense_sweep_t<false>(ctx, g, ld, src, rhs, ycur, yold, alpha, om, err);
}

}  // namespace pprviz
