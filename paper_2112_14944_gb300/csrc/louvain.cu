// Louvain+ supergraph hierarchy on the GPU (Sec. 5, the preprocessing step;
// Appendix A, the Louvain+ merge rules).
//
// Level l+1 groups the nodes of level l (level 0: the leaves). Every node
// starts as its own group; a group S merges into a neighbouring group T by
// rule (i), when T is S's only neighbour, or by rule (ii), into the T of the
// largest modularity gain Q^(S, T) = sum_{V_i in S} q(V_i, T). With w(.) and
// w_cr counted as ordered leaf pairs (both directions of each edge, the count
// under which q is the change of modularity), (2m)^2 Q^(S, T) / 2 equals
//   G(S, T) = 2m c(S, T) - w_in(S) w_in(T),
// c(S, T) the CSR entries u -> v with u in S and v in T and w_in the degree
// sums, an exact integer: no decision depends on rounding.
//
// Schedule (synchronous rounds; the appendix gives the rules, not their
// order): in a round every group picks its target from the state at the
// start of the round (rule (i) if it has one neighbour, else the largest
// G among the neighbours whose merge keeps at most k children, ties to the
// smaller id, taken only if G > 0 until a round merges nothing, then any
// G). S moves when its target does not (T proposes nothing, or T proposes
// S back and T has the smaller id); a target takes its movers in increasing
// id order while its size stays within k. A level ends with a round that
// merges nothing after that switch; the next level's nodes are the groups,
// numbered by their smallest member. The hierarchy ends when a level has at
// most k nodes or merged nothing.
//
// Data per level: the degree sum of every node, the group of every node (a
// representative: the id of a member; targets never move in their round, so
// one relabelling step applies a round), and the list of the current groups'
// pairs (S, T, c(S, T)), S != T, each once. After every round that merged,
// the list is mapped through the merges and summed per distinct pair in an
// open-addressing table keyed by (S, T) (integer atomics), so it shrinks as
// the groups grow; at the end of a level its representatives are relabelled
// to the next level's ids. The round's per-group maxima and minima are
// integer atomics too: the result does not depend on the order of any atomic.
#include <cstdio>
#include <cstring>

#include "common.cuh"

namespace pprviz {

namespace {

constexpr unsigned long long kLpEmpty = ~0ull;
constexpr int kLpTpb = 256;
constexpr int kLpMaxLevels = 64;
constexpr int kLpMaxRounds = 100000;

__device__ __forceinline__ unsigned long long lp_hash(unsigned long long x) {
  // splitmix64 finaliser (Steele, Lea, Flood 2014)
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

// c(S, T) += w in the table (mask + 1 slots, at least twice the pairs that
// can be inserted, so a free slot is always found; a full table sets bit 0
// of *err and drops the pair).
__device__ __forceinline__ void lp_pair_add(unsigned long long *keys, int32_t *vals, unsigned long long mask,
                                            uint32_t S, uint32_t T, int32_t w, int *err) {
  const unsigned long long key = ((unsigned long long)S << 32) | T;
  unsigned long long h = lp_hash(key) & mask;
  for (unsigned long long probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(&keys[h], kLpEmpty, key);
    if (prev == kLpEmpty || prev == key) {
      atomicAdd(&vals[h], w);
      return;
    }
    h = (h + 1) & mask;
  }
  atomicOr(err, 1);
}

// level-0 pairs: one ordered pair per CSR entry u -> v
__global__ void k_lp_edges0(int64_t n, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                            int32_t *__restrict__ eA, int32_t *__restrict__ eB, int32_t *__restrict__ ew,
                            int64_t *__restrict__ win) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = rp[u], e = rp[u + 1];
    win[u] = e - b;
    for (int64_t t = b; t < e; ++t) {
      eA[t] = (int32_t)u;
      eB[t] = col[t];
      ew[t] = 1;
    }
  }
}

__global__ void k_lp_round_init(int32_t nl, int32_t *__restrict__ gsize, long long *__restrict__ gwin,
                                int32_t *__restrict__ nbr, long long *__restrict__ bgain, int32_t *__restrict__ bt,
                                int32_t *__restrict__ prop, int32_t *__restrict__ mcnt, int32_t *__restrict__ mcur,
                                int32_t *__restrict__ acc) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x) {
    gsize[a] = 0;
    gwin[a] = 0;
    nbr[a] = 0;
    bgain[a] = LLONG_MIN;
    bt[a] = INT32_MAX;
    prop[a] = -1;
    mcnt[a] = 0;
    mcur[a] = 0;
    acc[a] = 0;
  }
}

// group sizes (children) and degree sums
__global__ void k_lp_gstats(int32_t nl, const int32_t *__restrict__ grp, const long long *__restrict__ win,
                            int32_t *__restrict__ gsize, long long *__restrict__ gwin) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = grp[a];
    atomicAdd(&gsize[g], 1);
    atomicAdd(reinterpret_cast<unsigned long long *>(&gwin[g]), (unsigned long long)win[a]);
  }
}

// c(S, T) summed over the pair list, its ends mapped by `map` (the group of
// each node within a level; the parent of each node for the next level's
// pairs)
__global__ void k_lp_pairs(int64_t E, const int32_t *__restrict__ eA, const int32_t *__restrict__ eB,
                           const int32_t *__restrict__ ew, const int32_t *__restrict__ map,
                           unsigned long long *__restrict__ keys, int32_t *__restrict__ vals, unsigned long long mask,
                           int *__restrict__ err) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t S = map[eA[e]], T = map[eB[e]];
    if (S != T) lp_pair_add(keys, vals, mask, (uint32_t)S, (uint32_t)T, ew[e], err);
  }
}

__device__ __forceinline__ long long lp_gain(long long m2, int32_t c, long long wS, long long wT) {
  return m2 * (long long)c - wS * wT;
}

// per group: distinct neighbours, and the largest gain among the neighbours
// it fits with (the pair list holds each (S, T) of the current groups once)
__global__ void k_lp_best(int64_t E, const int32_t *__restrict__ eA, const int32_t *__restrict__ eB,
                          const int32_t *__restrict__ ew, const int32_t *__restrict__ gsize,
                          const long long *__restrict__ gwin, int32_t k, long long m2, int32_t *__restrict__ nbr,
                          long long *__restrict__ bgain) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t S = eA[e], T = eB[e];
    atomicAdd(&nbr[S], 1);
    if (gsize[S] + gsize[T] <= k) atomicMax(&bgain[S], lp_gain(m2, ew[e], gwin[S], gwin[T]));
  }
}

// per group: the smallest neighbour id that reaches the largest gain
__global__ void k_lp_argbest(int64_t E, const int32_t *__restrict__ eA, const int32_t *__restrict__ eB,
                             const int32_t *__restrict__ ew, const int32_t *__restrict__ gsize,
                             const long long *__restrict__ gwin, int32_t k, long long m2,
                             const long long *__restrict__ bgain, int32_t *__restrict__ bt) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t S = eA[e], T = eB[e];
    if (gsize[S] + gsize[T] <= k && lp_gain(m2, ew[e], gwin[S], gwin[T]) == bgain[S]) atomicMin(&bt[S], T);
  }
}

// the group of every current group after the round: its target if it moved
__global__ void k_lp_gmap(int32_t nl, const int32_t *__restrict__ acc, const int32_t *__restrict__ prop,
                          int32_t *__restrict__ gmap) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    gmap[a] = acc[a] ? prop[a] : (int32_t)a;
}

// the level's final pair list relabelled to the next level's ids (distinct
// groups have distinct parents, so no two pairs merge)
__global__ void k_lp_relabel(int64_t E, int32_t *__restrict__ eA, int32_t *__restrict__ eB,
                             const int32_t *__restrict__ parent) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
    eA[e] = parent[eA[e]];
    eB[e] = parent[eB[e]];
  }
}

// proposals: rule (i) (one neighbour), or rule (ii) (positive gain, or any
// gain once relaxed)
__global__ void k_lp_propose(int32_t nl, const int32_t *__restrict__ gsize, const int32_t *__restrict__ nbr,
                             const long long *__restrict__ bgain, const int32_t *__restrict__ bt, int relaxed,
                             int32_t *__restrict__ prop) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nl; s += (int64_t)gridDim.x * blockDim.x) {
    if (gsize[s] == 0 || bt[s] == INT32_MAX) continue;
    if (nbr[s] == 1 || relaxed || bgain[s] > 0) prop[s] = bt[s];
  }
}

// movers: S moves when its target stays (no proposal, or a mutual proposal
// in which the target has the smaller id); counted per target
__global__ void k_lp_movers(int32_t nl, const int32_t *__restrict__ prop, int32_t *__restrict__ mover,
                            int32_t *__restrict__ mcnt) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nl; s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t t = prop[s];
    int mv = 0;
    if (t >= 0) {
      const int32_t pt = prop[t];
      mv = pt < 0 || (pt == (int32_t)s && (int32_t)s > t);
    }
    mover[s] = mv;
    if (mv) atomicAdd(&mcnt[t], 1);
  }
}

__global__ void k_lp_scatter(int32_t nl, const int32_t *__restrict__ prop, const int32_t *__restrict__ mover,
                             const int64_t *__restrict__ moff, int32_t *__restrict__ mcur, int32_t *__restrict__ mlist) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nl; s += (int64_t)gridDim.x * blockDim.x) {
    if (!mover[s]) continue;
    const int32_t t = prop[s];
    mlist[moff[t] + atomicAdd(&mcur[t], 1)] = (int32_t)s;
  }
}

// one warp per target: its movers in increasing id order, each taken while
// the target's size stays within k
__global__ void k_lp_accept(int32_t nl, int32_t k, const int32_t *__restrict__ mcnt, const int64_t *__restrict__ moff,
                            const int32_t *__restrict__ mlist, const int32_t *__restrict__ gsize,
                            int32_t *__restrict__ acc, int *__restrict__ naccepted) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); t < nl; t += warps) {
    const int32_t cnt = mcnt[t];
    if (cnt == 0) continue;
    const int32_t *seg = mlist + moff[t];
    int32_t room = k - gsize[t];
    int32_t last = -1;
    int taken = 0;
    for (int32_t step = 0; step < cnt && room > 0; ++step) {
      int32_t best = INT32_MAX;
      for (int32_t i = lane; i < cnt; i += 32) {
        const int32_t s = seg[i];
        if (s > last && s < best) best = s;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (best == INT32_MAX) break;
      const int32_t sz = gsize[best];
      if (sz <= room) {
        if (lane == 0) acc[best] = 1;
        room -= sz;
        ++taken;
      }
      last = best;
    }
    if (lane == 0 && taken) atomicAdd(naccepted, taken);
  }
}

__global__ void k_lp_apply(int32_t nl, int32_t *__restrict__ grp, const int32_t *__restrict__ acc,
                           const int32_t *__restrict__ prop) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g = grp[a];
    if (acc[g]) grp[a] = prop[g];
  }
}

__global__ void k_lp_fill(int32_t nl, int32_t *__restrict__ x, int32_t v) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    x[a] = v;
}

__global__ void k_lp_iota(int32_t nl, int32_t *__restrict__ x) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    x[a] = (int32_t)a;
}

__global__ void k_lp_minmember(int32_t nl, const int32_t *__restrict__ grp, int32_t *__restrict__ minm) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    atomicMin(&minm[grp[a]], (int32_t)a);
}

__global__ void k_lp_first(int32_t nl, const int32_t *__restrict__ grp, const int32_t *__restrict__ minm,
                           int32_t *__restrict__ flag) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    flag[a] = minm[grp[a]] == (int32_t)a;
}

// parent[a] = rank of a's group among the groups ordered by smallest member
__global__ void k_lp_parent(int32_t nl, const int32_t *__restrict__ grp, const int32_t *__restrict__ minm,
                            const int64_t *__restrict__ rank, int32_t *__restrict__ parent) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    parent[a] = (int32_t)rank[minm[grp[a]]];
}

__global__ void k_lp_lift_win(int32_t nl, const int32_t *__restrict__ parent, const long long *__restrict__ win,
                              long long *__restrict__ win2) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < nl; a += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(reinterpret_cast<unsigned long long *>(&win2[parent[a]]), (unsigned long long)win[a]);
}

__global__ void k_lp_zero64(int64_t n, long long *__restrict__ x) {
  for (int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x)
    x[a] = 0;
}

// the table's pairs as a pair list (any order), each emitted slot cleared
// so that the table is empty again for the next contraction; one counter
// atomic per warp (H is a power of two >= 1,024 and the grid a multiple of
// 32 threads, so every lane of a warp is in range together)
__global__ void k_lp_compact(unsigned long long H, unsigned long long *__restrict__ keys,
                             int32_t *__restrict__ vals, int32_t *__restrict__ eA, int32_t *__restrict__ eB,
                             int32_t *__restrict__ ew, unsigned long long *__restrict__ count) {
  const int lane = threadIdx.x & 31;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long h = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; h < H; h += stride) {
    const unsigned long long key = keys[h];
    const bool has = key != kLpEmpty;
    const unsigned mask = __ballot_sync(0xffffffffu, has);
    unsigned long long first = 0;
    if (lane == 0 && mask) first = atomicAdd(count, (unsigned long long)__popc(mask));
    first = __shfl_sync(0xffffffffu, first, 0);
    if (has) {
      const unsigned long long i = first + (unsigned long long)__popc(mask & ((1u << lane) - 1u));
      eA[i] = (int32_t)(key >> 32);
      eB[i] = (int32_t)(key & 0xffffffffu);
      ew[i] = vals[h];
      keys[h] = kLpEmpty;
      vals[h] = 0;
    }
  }
}

// exclusive prefix sum of n int32 counts into int64 (three passes: 1,024-entry
// blocks, their totals in one block, then the block offsets added)
constexpr int kScanB = 1024;
__global__ void k_scan_blocks(int64_t n, const int32_t *__restrict__ in, int64_t *__restrict__ out,
                              int64_t *__restrict__ bsum) {
  __shared__ int64_t wsum[32];
  const int64_t i = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t v = i < n ? (int64_t)in[i] : 0;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t s = wsum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    wsum[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int64_t before = warp ? wsum[warp - 1] : 0;
  if (i < n) out[i] = before + x - v;
  if (threadIdx.x == kScanB - 1) bsum[blockIdx.x] = wsum[31];
}

__global__ void k_scan_top(int64_t nb, int64_t *__restrict__ bsum, int64_t *__restrict__ total) {
  // one block: exclusive scan of the block totals, chunk by chunk
  __shared__ int64_t wsum[32];
  __shared__ int64_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < nb; base += kScanB) {
    const int64_t i = base + threadIdx.x;
    const int64_t v = i < nb ? bsum[i] : 0;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int64_t s = wsum[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, s, o);
        if (lane >= o) s += y;
      }
      wsum[lane] = s;
    }
    __syncthreads();
    const int64_t before = (warp ? wsum[warp - 1] : 0) + carry;
    if (i < nb) bsum[i] = before + x - v;
    __syncthreads();
    if (threadIdx.x == 0) carry += wsum[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(int64_t n, int64_t *__restrict__ out, const int64_t *__restrict__ bsum) {
  const int64_t i = (int64_t)blockIdx.x * kScanB + threadIdx.x;
  if (i < n) out[i] += bsum[blockIdx.x];
}

unsigned grid_for(int64_t n) {
  const int64_t b = (n + kLpTpb - 1) / kLpTpb;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

}  // namespace

// Exclusive scan helper: out[i] = sum_{j < i} in[j]; total (device, one
// int64) = the sum. bsum: ceil(n / 1024) int64 of scratch.
static int lp_scan(pprviz_ctx *ctx, int64_t n, const int32_t *in, int64_t *out, int64_t *bsum, int64_t *total) {
  const int64_t nb = std::max<int64_t>(1, (n + kScanB - 1) / kScanB);
  k_scan_blocks<<<(unsigned)nb, kScanB, 0, ctx->stream>>>(n, in, out, bsum);
  PPRVIZ_LAUNCHED(ctx);
  k_scan_top<<<1, kScanB, 0, ctx->stream>>>(nb, bsum, total);
  PPRVIZ_LAUNCHED(ctx);
  k_scan_add<<<(unsigned)nb, kScanB, 0, ctx->stream>>>(n, out, bsum);
  PPRVIZ_LAUNCHED(ctx);
  return PPRVIZ_OK;
}

int louvain_plus_solve(pprviz_ctx *ctx, const pprviz_graph *g, int32_t k, std::vector<int32_t> &parents,
                       std::vector<int64_t> &level_n, pprviz_louvain_info *info) {
  parents.clear();
  level_n.assign(1, g->n);
  memset(info, 0, sizeof(*info));
  const int64_t n = g->n, E0 = g->nnz;
  if (n <= k || E0 == 0) return PPRVIZ_OK;
  const long long m2 = (long long)E0;
  // pair table: a power of two of at least twice the level-0 pairs (every
  // contraction uses the leading power of two its own pairs need)
  unsigned long long H = 1024;
  while (H < 2ull * (unsigned long long)E0) H <<= 1;
  const size_t ni = (size_t)n;
  // node arrays (sized for level 0; later levels are smaller), each starting
  // on a 16-byte boundary
  const size_t a32 = (sizeof(int32_t) * ni + 15) & ~(size_t)15, a64 = (sizeof(long long) * ni + 15) & ~(size_t)15;
  PPRVIZ_TRY(ws_ensure(ctx, WS_LPNODE, 13 * a32 + 4 * a64));
  char *base = ctx->ws[WS_LPNODE].as<char>();
  auto take = [&](size_t bytes) {
    char *p = base;
    base += (bytes + 15) & ~(size_t)15;
    return p;
  };
  int32_t *grp = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *gsize = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *nbr = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *bt = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *prop = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *mcnt = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *mcur = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *mover = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *mlist = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *acc = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *minm = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *parent = (int32_t *)take(sizeof(int32_t) * ni);
  int32_t *gmap = (int32_t *)take(sizeof(int32_t) * ni);
  long long *gwin = (long long *)take(sizeof(long long) * ni);
  long long *bgain = (long long *)take(sizeof(long long) * ni);
  long long *win = (long long *)take(sizeof(long long) * ni);
  long long *win2 = (long long *)take(sizeof(long long) * ni);
  // scan scratch: offsets (n + 1 int64), block totals, counters
  PPRVIZ_TRY(ws_ensure(ctx, WS_LPSCAN, sizeof(int64_t) * (ni + 1 + (ni + kScanB) / kScanB + 8)));
  int64_t *moff = ctx->ws[WS_LPSCAN].as<int64_t>();
  int64_t *bsum = moff + ni + 1;
  int64_t *misc = bsum + (ni + kScanB) / kScanB + 1;  // [0] scan total, [1] pair count, [2] accepted + error
  int *flags = reinterpret_cast<int *>(misc + 2);      // [0] accepted in the round, [1] table error
  // pair lists (two, ping-pong) and the table
  const size_t eb = (sizeof(int32_t) * 3) * (size_t)E0;
  PPRVIZ_TRY(ws_ensure(ctx, WS_LPEDGE, 2 * eb + 64));
  int32_t *eA = ctx->ws[WS_LPEDGE].as<int32_t>();
  int32_t *eB = eA + E0, *ew = eB + E0;
  int32_t *fA = ew + E0, *fB = fA + E0, *fw = fB + E0;
  PPRVIZ_TRY(ws_ensure(ctx, WS_LPHASH, (sizeof(unsigned long long) + sizeof(int32_t)) * (size_t)H));
  unsigned long long *keys = ctx->ws[WS_LPHASH].as<unsigned long long>();
  int32_t *vals = reinterpret_cast<int32_t *>(keys + H);
  int64_t E = E0;

  // the pair list mapped through `map` and summed per distinct (S, T), S != T
  auto contract = [&](const int32_t *map) -> int {
    unsigned long long Hl = 1024;
    while (Hl < 2ull * (unsigned long long)E) Hl <<= 1;
    info->slot_visits += (int64_t)Hl;
    info->pair_visits += E;
    // the table is empty here: cleared once below, then by every compaction
    PPRVIZ_CUDA(ctx, cudaMemsetAsync(misc + 1, 0, 2 * sizeof(int64_t), ctx->stream));
    k_lp_pairs<<<grid_for(E), kLpTpb, 0, ctx->stream>>>(E, eA, eB, ew, map, keys, vals, Hl - 1, flags + 1);
    PPRVIZ_LAUNCHED(ctx);
    k_lp_compact<<<grid_for((int64_t)Hl), kLpTpb, 0, ctx->stream>>>(
        Hl, keys, vals, fA, fB, fw, reinterpret_cast<unsigned long long *>(misc + 1));
    PPRVIZ_LAUNCHED(ctx);
    int64_t count = 0;
    int full = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&count, misc + 1, sizeof(count), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&full, flags + 1, sizeof(full), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (full) return set_err(ctx, PPRVIZ_E_CUDA, "Louvain+: pair table full (internal error)");
    std::swap(eA, fA);
    std::swap(eB, fB);
    std::swap(ew, fw);
    E = count;
    return PPRVIZ_OK;
  };

  PPRVIZ_CUDA(ctx, cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * H, ctx->stream));
  PPRVIZ_CUDA(ctx, cudaMemsetAsync(vals, 0, sizeof(int32_t) * H, ctx->stream));
  int32_t nl = (int32_t)n;
  k_lp_edges0<<<grid_for(n), kLpTpb, 0, ctx->stream>>>(n, pull_rp(g), pull_col(g), eA, eB, ew, (int64_t *)win);
  PPRVIZ_LAUNCHED(ctx);
  {
    // level-0 pairs: each (u, v), u != v, once with its multiplicity
    PPRVIZ_PROF(ctx, PPRVIZ_K_HIER);
    k_lp_iota<<<grid_for(nl), kLpTpb, 0, ctx->stream>>>(nl, gmap);
    PPRVIZ_LAUNCHED(ctx);
    PPRVIZ_TRY(contract(gmap));
  }
  int rounds = 0;
  bool done = false;  // a level reached at most k nodes
  for (int level = 0; !done; ++level) {
    if (level == kLpMaxLevels) return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "Louvain+: level cap reached");
    const unsigned gn = grid_for(nl);
    k_lp_iota<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp);
    PPRVIZ_LAUNCHED(ctx);
    bool relaxed = false;
    int merges = 0;
    for (;;) {
      if (++rounds > kLpMaxRounds)
        return set_err(ctx, PPRVIZ_E_NOT_CONVERGED, "Louvain+: round cap reached");
      info->list_visits += E;
      info->node_visits += nl;
      PPRVIZ_PROF(ctx, PPRVIZ_K_HIER);
      k_lp_round_init<<<gn, kLpTpb, 0, ctx->stream>>>(nl, gsize, gwin, nbr, bgain, bt, prop, mcnt, mcur, acc);
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_CUDA(ctx, cudaMemsetAsync(flags, 0, 2 * sizeof(int), ctx->stream));
      k_lp_gstats<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp, win, gsize, gwin);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_best<<<grid_for(E), kLpTpb, 0, ctx->stream>>>(E, eA, eB, ew, gsize, gwin, k, m2, nbr, bgain);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_argbest<<<grid_for(E), kLpTpb, 0, ctx->stream>>>(E, eA, eB, ew, gsize, gwin, k, m2, bgain, bt);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_propose<<<gn, kLpTpb, 0, ctx->stream>>>(nl, gsize, nbr, bgain, bt, relaxed ? 1 : 0, prop);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_movers<<<gn, kLpTpb, 0, ctx->stream>>>(nl, prop, mover, mcnt);
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_TRY(lp_scan(ctx, nl, mcnt, moff, bsum, misc));
      k_lp_scatter<<<gn, kLpTpb, 0, ctx->stream>>>(nl, prop, mover, moff, mcur, mlist);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_accept<<<grid_for((int64_t)nl * 32), kLpTpb, 0, ctx->stream>>>(nl, k, mcnt, moff, mlist, gsize, acc, flags);
      PPRVIZ_LAUNCHED(ctx);
      k_lp_apply<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp, acc, prop);
      PPRVIZ_LAUNCHED(ctx);
      int accepted = 0;
      PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&accepted, flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
      if (accepted == 0) {
        if (relaxed) break;
        relaxed = true;
        continue;
      }
      merges += accepted;
      // the pair list of the merged groups
      k_lp_gmap<<<gn, kLpTpb, 0, ctx->stream>>>(nl, acc, prop, gmap);
      PPRVIZ_LAUNCHED(ctx);
      PPRVIZ_TRY(contract(gmap));
    }
    if (merges == 0) break;  // nothing merged: the hierarchy ends below this level
    // number the groups by smallest member
    PPRVIZ_PROF(ctx, PPRVIZ_K_HIER);
    k_lp_fill<<<gn, kLpTpb, 0, ctx->stream>>>(nl, minm, INT32_MAX);
    PPRVIZ_LAUNCHED(ctx);
    k_lp_minmember<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp, minm);
    PPRVIZ_LAUNCHED(ctx);
    k_lp_first<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp, minm, mcnt);
    PPRVIZ_LAUNCHED(ctx);
    PPRVIZ_TRY(lp_scan(ctx, nl, mcnt, moff, bsum, misc));
    k_lp_parent<<<gn, kLpTpb, 0, ctx->stream>>>(nl, grp, minm, moff, parent);
    PPRVIZ_LAUNCHED(ctx);
    int64_t nl2h = 0;
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(&nl2h, misc, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int32_t nl2 = (int32_t)nl2h;
    const size_t off = parents.size();
    parents.resize(off + (size_t)nl);
    PPRVIZ_CUDA(ctx, cudaMemcpyAsync(parents.data() + off, parent, sizeof(int32_t) * (size_t)nl, cudaMemcpyDeviceToHost,
                                     ctx->stream));
    PPRVIZ_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    level_n.push_back(nl2);
    if (nl2 <= k) {
      done = true;
      break;
    }
    // the next level: degree sums lifted, the pair list (already one entry
    // per pair of final groups, keyed by their representatives, whose parent
    // is the group's new id) relabelled
    k_lp_zero64<<<grid_for(nl2), kLpTpb, 0, ctx->stream>>>(nl2, win2);
    PPRVIZ_LAUNCHED(ctx);
    k_lp_lift_win<<<gn, kLpTpb, 0, ctx->stream>>>(nl, parent, win, win2);
    PPRVIZ_LAUNCHED(ctx);
    k_lp_relabel<<<grid_for(E), kLpTpb, 0, ctx->stream>>>(E, eA, eB, parent);
    PPRVIZ_LAUNCHED(ctx);
    std::swap(win, win2);
    nl = nl2;
  }
  info->levels = (int32_t)level_n.size() - 1;
  info->rounds = rounds;
  info->parent_need = (int64_t)parents.size();
  return PPRVIZ_OK;
}

}  // namespace pprviz
