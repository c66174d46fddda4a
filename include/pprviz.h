/*
 * pprviz.h - C ABI of the GB300 (sm_103a) PPRviz hot path.
 *
 * The library computes, on one GPU, the distance-matrix and positioning
 * phases of PPRviz (Zhang et al., "Effective and Efficient PageRank-based
 * Positioning for Graph Visualization", SIGMOD 2023, arXiv 2112.14944):
 *
 *   1. personalized PageRank pi(s, .) for every node s of a view
 *      (Sec. 3.1: random walk with restart probability alpha);
 *   2. DPPR pi_d(s, t) = d(s) pi(s, t) (Definition 1) and PDist
 *      Delta[i,j] = min(max(1 - ln(pi_d(i,j) + pi_d(j,i)), 2), 2 ln n)
 *      (Sec. 3.1, Eq. (1));
 *   3. the stress energy L(X | Delta) = sum_{i<j} (1 - |X_i - X_j| / Delta_ij)^2
 *      (Sec. 5, Eq. (7)), its gradients, and stress majorization
 *      X <- (L^w)^+ L^Y(X) X (Appendix A.1, Eq. (10)).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Every call returns an int status (PPRVIZ_OK = 0 or a PPRVIZ_E_* code);
 *    no C++ exception crosses the ABI. pprviz_last_error() gives a message
 *    owned by the context, valid until the next call on that context.
 *  - The caller owns every input and output buffer. By default they are host
 *    pointers: the call copies inputs to the device, runs, copies outputs back
 *    and returns when the results are in place. With PPRVIZ_DEVICE_PTRS in
 *    `mem_flags` they are device pointers on the context's device, and the
 *    call only enqueues work on the context stream (pprviz_sync waits).
 *    Scalar report outputs (cert_out, stress_out, e_out) are always host
 *    pointers and are written before the call returns (the call waits for the
 *    values they need).
 *  - The library owns the context, graph objects and its device workspace.
 *  - Dense matrices are row-major with leading dimension k. Node and view ids
 *    are 0-based. A view lists distinct node ids of the graph.
 *  - A context is used by one host thread at a time.
 */
#ifndef PPRVIZ_H
#define PPRVIZ_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PPRVIZ_OK 0
#define PPRVIZ_E_INVALID_ARG 1   /* bad scalar, size, pointer or flag */
#define PPRVIZ_E_BAD_GRAPH 2     /* CSR fails validation (see pprviz_graph_upload) */
#define PPRVIZ_E_OOM 3           /* device allocation failed */
#define PPRVIZ_E_CUDA 4          /* a CUDA runtime call or kernel launch failed */
#define PPRVIZ_E_NOT_CONVERGED 5 /* iteration cap hit; outputs valid, cert_out states the bound */
#define PPRVIZ_E_TIMEOUT 6       /* a bounded device wait expired */

/* graph flags */
#define PPRVIZ_UNDIRECTED 1u     /* CSR stores both directions (checked); without it: directed */
#define PPRVIZ_VALIDATE 2u       /* accepted for clarity; validation always runs */
#define PPRVIZ_DEGREE_COUNT 4u   /* weighted graph, but d(v) = edge count instead of strength */

/* memory / output flags */
#define PPRVIZ_DEVICE_PTRS 1u    /* buffers are device pointers; calls are asynchronous */
#define PPRVIZ_OUT_FP64 2u       /* matrices and coordinates are double instead of float */

/* propagation precision (pprviz_dppr) and layout precision (pprviz_layout) */
#define PPRVIZ_FP64 0            /* plain FP64: power iteration / FP64 layout arithmetic */
#define PPRVIZ_FP32 1            /* FP32 Chebyshev sweeps + FP64 residual + refinement; FP32 layout.
                                  * pprviz_dppr picks the sweep kernel: dense tensor-core sweeps when
                                  * n >= 512 and nnz >= n^2 / 20 (and the n x n matrix fits), CSR
                                  * gather sweeps otherwise */
#define PPRVIZ_FP32_CSR 2        /* pprviz_dppr only: PPRVIZ_FP32 with CSR gather sweeps always */
#define PPRVIZ_FP32_TC 3         /* pprviz_dppr only: PPRVIZ_FP32 with every sweep a dense
                                  * tensor-core contraction (3xTF32 tcgen05.mma); E_OOM if the
                                  * n x n weight matrix does not fit */
#define PPRVIZ_FP32_BF16TC 4     /* pprviz_dppr only: as PPRVIZ_FP32_TC, but every sweep is one
                                  * BF16 x BF16 tcgen05.mma (kind::f16) with FP32 accumulation;
                                  * the FP64 residual and up to 16 FP32 refinement passes
                                  * restore eps (E_NOT_CONVERGED if they do not) */

typedef struct pprviz_ctx pprviz_ctx;
typedef struct pprviz_graph pprviz_graph;

/* Counters of the last pprviz_dppr / pprviz_layout call on a context. */
typedef struct pprviz_stats {
    int32_t groups;            /* source groups processed */
    int32_t sweeps_main;       /* propagation sweeps of the main solve, summed over groups */
    int32_t sweeps_refine;     /* refinement sweeps, summed over groups */
    int32_t refine_passes;     /* refinement passes, summed over groups */
    int32_t residual_passes;   /* FP64 residual passes, summed over groups */
    int32_t kernel_launches;   /* kernels this library launched in the call */
    double max_cert;           /* max over sources of the final certificate */
    int32_t layout_iters;      /* layout iterations run */
    int32_t source_group;      /* sources per group (state tile width) */
    /* Algorithmic bytes of the call, per kernel class: the bytes each launch
     * must move for the entries it computes (valid sources only; a gathered
     * state row counts once, CSR and caches excluded). Sweep: 12 bytes per
     * (node, source) for a Chebyshev sweep (read y_k, y_k-1, write y_k+1),
     * 16 with a dense right-hand side, 16 per FP64 power sweep; L^Y and apply
     * passes: one k x k matrix read each. */
    double bytes_sweep;
    double bytes_ly;
    double bytes_apply;
    /* Algorithmic FP flops of the L^w inverse (symmetric block sweep: pivot
     * inverses, panels and the upper-triangle trailing updates). */
    double flops_factor;
    /* Algorithmic flops of the dense tensor-core sweeps: 2 n^2 per (sweep,
     * valid source); the 3xTF32 split executes three times as many. */
    double flops_dense;
    /* 1 when the layout updates of the call ran as one CUDA graph (batched
     * views: the updates are recorded once and launched as a graph), else 0.
     * With kernel timing on (pprviz_profile) they are launched one by one. */
    int32_t graph_launched;
} pprviz_stats;

/* Kernel classes for per-class device timing (pprviz_profile). */
#define PPRVIZ_K_GRAPH 0         /* CSR validation, degrees, view checks */
#define PPRVIZ_K_SWEEP 1         /* propagation sweeps (Chebyshev / power) */
#define PPRVIZ_K_RESIDUAL 2      /* FP64 residual certificate passes */
#define PPRVIZ_K_EXTRACT 3       /* DPPR row extraction (transpose + scaling) */
#define PPRVIZ_K_PDIST 4         /* PDist transform */
#define PPRVIZ_K_FACTOR 5        /* L^w build and Gauss-Jordan inversion */
#define PPRVIZ_K_LY 6            /* all-pairs L^Y(X) X pass */
#define PPRVIZ_K_APPLY 7         /* X = (L^w)^+ b pass */
#define PPRVIZ_K_ENERGY 8        /* energy / gradient passes and reductions */
#define PPRVIZ_K_OTHER 9         /* initialisation, casts, small helpers */
#define PPRVIZ_K_PUSH 10         /* Tau-Push rounds and the DPR power iterations */
#define PPRVIZ_K_HIER 11         /* Louvain+ merge rounds and level lifts */
#define PPRVIZ_NKCLASS 12

/* Create a context on CUDA device `device`. `cuda_stream` is a cudaStream_t
 * to run on (borrowed, not destroyed), or NULL for a stream the context owns.
 * Errors: E_INVALID_ARG (out == NULL, bad device), E_CUDA. */
int pprviz_create(pprviz_ctx **out, int device, void *cuda_stream);
void pprviz_destroy(pprviz_ctx *ctx);
/* Cap the device workspace of a context (a library convenience; the paper
 * has no counterpart): the buffers the context allocates for its calls
 * (staging, propagation state, matrices of the layout) may hold at most
 * `bytes` in all; 0 removes the cap. A call whose workspace would exceed it
 * fails with PPRVIZ_E_OOM before allocating, and the context stays usable
 * (buffers already held are kept). Graph objects and caller buffers are not
 * counted. Errors: E_INVALID_ARG (ctx NULL, bytes < 0). */
int pprviz_set_workspace_limit(pprviz_ctx *ctx, int64_t bytes);
/* Test aid for the bounded-wait error path (the paper has no counterpart).
 * The tensor-core kernels bound every wait on a copy or an MMA completion by
 * a deadline (2 s) and report PPRVIZ_E_TIMEOUT instead of hanging. This call
 * makes the next FP32 L^w inverse on the context (pprviz_layout with
 * PPRVIZ_FP32) leave out one operand copy of one tile, so that the wait for
 * it runs out: that call returns PPRVIZ_E_TIMEOUT after about 2 s, its
 * outputs are undefined, and the context stays usable for the next call.
 * Nothing faults. Errors: E_INVALID_ARG (ctx NULL). */
int pprviz_test_expire_wait(pprviz_ctx *ctx);
const char *pprviz_last_error(const pprviz_ctx *ctx);
/* Wait for all work enqueued on the context stream. */
int pprviz_sync(pprviz_ctx *ctx);
int pprviz_get_stats(const pprviz_ctx *ctx, pprviz_stats *out);
/* Device timing per kernel class, by CUDA events on the context stream
 * around launches. enable = 0: off; 1: every launch is timed; N > 1: every
 * launch of the classes launched a few times per call, and one launch in N
 * of the sweep, L^Y, apply and other classes (launched hundreds of times per
 * call; events between every launch would serialise them). The totals
 * accumulate until read; pprviz_profile resets them. */
int pprviz_profile(pprviz_ctx *ctx, int enable);
/* Waits for the context stream, then writes, per class (PPRVIZ_NKCLASS
 * entries; NULL arrays are skipped) since the last reset: the total device
 * milliseconds of the timed launches, the number of launches, and the number
 * of timed launches (the ones in ms_out). Launch counts are kept even when
 * timing is off. A pair of events that cannot be timed is left out of both
 * ms_out and timed_out, every event goes back to the context's pool, the
 * arrays are still written, and the call returns E_CUDA. */
int pprviz_kernel_times(pprviz_ctx *ctx, double *ms_out, int64_t *launches_out, int64_t *timed_out);

/* P0 - graph ingest (Sec. 2.1; Table 1: n nodes, out-degree d(v)).
 * row_ptr: n+1 int64, row_ptr[0] = 0, non-decreasing, row_ptr[n] = nnz.
 * col_idx: nnz int32 out-neighbour ids, strictly increasing within a row
 *          (no duplicate edges), no self-loops.
 * weights: nnz float edge weights (> 0, finite) or NULL for unit weights;
 *          weighted walks step to v_j with probability w_ij / sum_j w_ij and
 *          d(v) is that sum (the strength) unless PPRVIZ_DEGREE_COUNT.
 * flags:   PPRVIZ_UNDIRECTED: the CSR stores both directions of every edge;
 *          the symmetry (including equal weights both ways) is checked.
 *          Without it the graph is directed (Sec. 2.1's general setting):
 *          row v lists v's out-neighbours, the walk steps along out-edges,
 *          d(v) is the out-degree (or out-strength), and a node without
 *          out-edges (dangling) keeps its walk; the library builds the
 *          in-neighbour CSR the pull-form sweeps need. Directed graphs take
 *          the CSR sweeps only (no tensor-core sweeps, no batched views);
 *          their FP32 propagation runs power sweeps with the same FP64
 *          certificate and refinement (a directed walk has a complex
 *          spectrum, outside the Chebyshev recurrence's interval). Every rule
 *          above is always checked on the device before the graph is
 *          accepted.
 * Host pointers unless mem_flags has PPRVIZ_DEVICE_PTRS. The library copies
 * the arrays; the caller may free them on return. A node with no edges is
 * kept: its walk stays on it and its d(v) = 0.
 * Errors: E_INVALID_ARG, E_BAD_GRAPH (validation failed; message says which
 * rule), E_OOM, E_CUDA. */
int pprviz_graph_upload(pprviz_ctx *ctx, int64_t n, const int64_t *row_ptr,
                        const int32_t *col_idx, const float *weights, uint32_t flags,
                        uint32_t mem_flags, pprviz_graph **out);
/* Frees a graph's device memory; valid before or after its context is destroyed. */
void pprviz_graph_free(pprviz_graph *g);
/* Copy the n degrees d(v) (double) computed on the device into deg_out (host
 * or device per mem_flags) and report n, nnz and m = sum_v d(v). */
int pprviz_graph_degrees(pprviz_ctx *ctx, const pprviz_graph *g, double *deg_out,
                         int64_t *n_out, int64_t *nnz_out, double *m_out, uint32_t mem_flags);

/* P1-P3 - DPPR and PDist of a view (Sec. 3.1, Definition 1 and Eq. (1)).
 * view:      k distinct node ids (int32). Row q of the outputs is source view[q].
 * alpha:     restart probability, 0 < alpha < 1.
 * eps:       absolute DPPR error bound. Each source s is certified by the FP64
 *            residual res = alpha e_s - x (I - (1 - alpha) P) of the computed
 *            row x: cert(s) = d(s) ||res||_1 / alpha bounds max_t |error| of
 *            d(s) x_t (Eq. (3) with 0 <= pi <= 1). The FP64 path runs power
 *            iteration for the a-priori sweep count; the FP32 path runs
 *            Chebyshev sweeps and FP32 refinement passes until every source
 *            has cert(s) <= eps, or returns E_NOT_CONVERGED after 6 passes.
 *            The FP32 path keeps each row as an exact sum of two floats, so it
 *            certifies down to about d(s) * 1e-13; tighter eps needs PPRVIZ_FP64.
 *            Through Eq. (1) the certificates bound the PDist error too:
 *            |dDelta_ij| <= (c_i + c_j) / max(z_ij - c_i - c_j, e / n_clamp^2).
 * precision: PPRVIZ_FP64, PPRVIZ_FP32 (sweep kernel chosen by density),
 *            PPRVIZ_FP32_CSR, PPRVIZ_FP32_TC or PPRVIZ_FP32_BF16TC (sweep
 *            kernel and operand precision forced). The
 *            tensor-core sweeps (P1d, Sec. 3.1 in matrix form: one sweep is the
 *            dense product W Y of the n x n weights and the n x G state) change
 *            only how a sweep is computed: the certificate and the refinement
 *            are the same FP64 residual over the CSR.
 * dppr_out:  k*k DPPR, row q = pi_d(view[q], view[.]); may be NULL.
 * pdist_out: k*k PDist with Delta[q][r] from pi_d(q,r) + pi_d(r,q), the upper
 *            clamp 2 ln n_clamp (n_clamp = 0 means the graph's n) and a zero
 *            diagonal; may be NULL.
 * cert_out:  k doubles, the final certificate per source (host); may be NULL.
 * Float outputs unless PPRVIZ_OUT_FP64 (then double). The certificate bounds
 * the computed row before the output is rounded to the output type.
 * Errors: E_INVALID_ARG (k < 1, k > n, bad id, duplicate id, alpha or eps out
 * of range, a tensor-core precision on a directed graph), E_NOT_CONVERGED,
 * E_OOM, E_CUDA. */
int pprviz_dppr(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view, int32_t k,
                double alpha, double eps, int precision, void *dppr_out, void *pdist_out,
                int64_t n_clamp, double *cert_out, uint32_t mem_flags);

/* Level-l DPPR and PDist between supernodes (Sec. 3.2, Definition 2, Eq. (2)):
 *   pi_d(V_i, V_j) = sum_{s in F(V_i), t in F(V_j)} pi_d(s, t) / (|F(V_i)| |F(V_j)|)
 * for the nsup children V_0 .. V_{nsup-1} of a supernode, each given by its
 * leaf set F(V_i) (CSR: leaf_ptr[nsup + 1] int64 with leaf_ptr[0] = 0 and
 * every set non-empty, leaf_idx[leaf_ptr[nsup]] int32 node ids; the sets are
 * disjoint). One FP32 propagation per supernode from the group start
 * alpha d(s) / |F(V_i)| on its leaves (the initial residues of GFP,
 * Algorithm 2), certified by the FP64 residual and refined until
 * cert_i = ||res_i||_1 / alpha <= eps; every entry of row i is then within
 * cert_i of Eq. (2). With singleton leaf sets this is pprviz_dppr's DPPR.
 * ldppr_out: nsup*nsup, row i = pi_d(V_i, .); may be NULL.
 * pdist_out: nsup*nsup, Eq. (1) on the level-l DPPR (upper clamp 2 ln n_clamp,
 *            n_clamp = 0 means the graph's n; zero diagonal); may be NULL.
 * cert_out:  nsup doubles (host); may be NULL.
 * Float outputs unless PPRVIZ_OUT_FP64; host or device buffers (leaf arrays
 * and outputs) per PPRVIZ_DEVICE_PTRS.
 * Errors: E_INVALID_ARG (nsup < 1 or > n, empty or overlapping leaf sets, a
 * leaf id out of range, alpha / eps / n_clamp out of range), E_NOT_CONVERGED,
 * E_OOM, E_CUDA. */
int pprviz_level_dppr(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr,
                      const int32_t *leaf_idx, double alpha, double eps, void *ldppr_out, void *pdist_out,
                      int64_t n_clamp, double *cert_out, uint32_t mem_flags);

/* Frontier profile of the view's propagation (a diagnostic for the threshold
 * of Algorithm 2, GFP). Runs `sweeps` FP64 power-iteration sweeps
 * x_{t+1} = alpha e_s + (1 - alpha) x_t P from every view source (Forward-Push
 * with every node pushed once per sweep) and writes to active_out[t] (host,
 * `sweeps` int64) the number of (node v, source s) entries whose push residue
 * after sweep t, r = d(s) (x_{t+1} - x_t)_v / alpha (Eq. (3)), exceeds
 * d(v) r_max with r_max = eps / max_{t in view} d(t): the entries that GFP
 * would still push. The fraction active_out[t] / (n k) is the share of a sweep
 * that a frontier-thresholded sweep could skip no more than. view: as in
 * pprviz_dppr (host or device per mem_flags).
 * Errors: E_INVALID_ARG (k, sweeps outside [1, 100000], alpha, eps), E_OOM, E_CUDA. */
int pprviz_frontier_profile(pprviz_ctx *ctx, const pprviz_graph *g, const int32_t *view, int32_t k, double alpha,
                            double eps, int32_t sweeps, int64_t *active_out, uint32_t mem_flags);

/* The DPR index of Tau-Push (Sec. 4, Eq. (dnpr-dnppr) with single-node
 * leaf sets; Sec. 4.3, indexing scheme): per node t
 *   tau_t = (1 / m) sum_k pi_d(v_k, v_t),
 * computed as the paper's global PageRank whose start vector has entry
 * d(v_k) / m at v_k: FP64 power iterations
 *   x_0 = alpha s,  x_{t+1} = alpha s + (1 - alpha) x_t P,  s = d / m,
 * until the walk mass not yet ended, (1 - alpha)^(T + 1), is at most eps.
 * (An undirected graph has tau_t = d(t) / m exactly.)
 * dpr_out:  n doubles (host or device per PPRVIZ_DEVICE_PTRS).
 * cert_out: host double, (1 - alpha)^(T + 1), the L1 bound on the error of
 *           dpr_out before rounding; may be NULL.
 * Errors: E_INVALID_ARG (dpr_out NULL, alpha outside (0, 1), eps outside
 * (0, 1), a graph without edges), E_OOM, E_CUDA. */
int pprviz_dpr(pprviz_ctx *ctx, const pprviz_graph *g, double alpha, double eps, double *dpr_out, double *cert_out,
               uint32_t mem_flags);

/* What one pprviz_tau_push call did (host struct). */
typedef struct pprviz_tau_info {
    double tau;               /* DPR threshold used */
    double r_max;             /* forward residue threshold, Eq. (rmax) */
    int32_t backward_targets; /* supernodes V_j with tau_j > tau (refined by GBP) */
    int32_t fwd_rounds;       /* synchronous push rounds of the forward phase */
    int32_t bwd_rounds;       /* and of the backward phase */
    int32_t pad0;
    int64_t fwd_pushes;       /* (node, source supernode) pushes, forward */
    int64_t bwd_pushes;       /* (node, target supernode) pushes, backward */
    int64_t fwd_edges;        /* residue shares sent along edges, forward */
    int64_t bwd_edges;        /* and backward */
} pprviz_tau_info;

/* Tau-Push (Sec. 4, Algorithm 1 with GFP, Algorithm 2, and GBP, Algorithm 3):
 * (eps, delta)-approximate level-l DPPR (Definition 3) between the nsup
 * children V_0 .. V_{nsup-1} of a supernode, leaf sets as in
 * pprviz_level_dppr (leaf_ptr / leaf_idx, disjoint, non-empty).
 *   tau    = the DPR threshold; tau <= 0 selects the paper's 1 / sqrt(nsup n);
 *   r_max  = eps delta / (m tau)  (Eq. (rmax));
 *   row i  = GFP from V_i: initial residue d(v) / |F(V_i)| on its leaves,
 *            pushes while some residue exceeds d(v) r_max, the reserve kept at
 *            the leaves of the children only;
 *   col j  = for every V_j with tau_j = mean over F(V_j) of dpr > tau: GBP
 *            towards V_j (initial residue 1 / |F(V_j)| on its leaves, pushes
 *            along in-edges while a residue exceeds
 *            rb_max = eps delta / max_{i != j} mean_{F(V_i)} d  (Eq. (brmax))),
 *            replacing the GFP estimates of that column.
 * The pushes run as synchronous rounds: every residue above its threshold is
 * pushed at once and shares arrive by FP64 atomic adds, so the order of the
 * pushes (which the paper leaves open) differs from a sequential push; the
 * stopping rule, and with it the error bounds of Lemmas 2 and 3 and
 * Theorem 3, are those of Algorithms 2 and 3. Every estimate is at most the
 * exact value; forward columns miss by at most r_max m tau_j, refined columns
 * by at most rb_max times the source's mean leaf degree. A node without
 * out-edges keeps the walk: its push takes the sum of its endless repeats.
 * dpr:       n doubles, the DPR index (pprviz_dpr), host or device.
 * ldppr_out: nsup*nsup estimates, row i = source V_i; may be NULL.
 * pdist_out: nsup*nsup, Eq. (1) on the estimates (Algorithm 1, conversion
 *            step; upper clamp 2 ln n_clamp, n_clamp = 0 means n); may be NULL.
 * info:      host struct; may be NULL.
 * Float outputs unless PPRVIZ_OUT_FP64; leaf arrays, dpr and outputs host or
 * device per PPRVIZ_DEVICE_PTRS.
 * Errors: E_INVALID_ARG (leaf sets as in pprviz_level_dppr, nsup * n at or
 * above 2^31, a graph of 2^31 or more stored edges, dpr NULL or with a negative or non-finite entry, alpha outside
 * (0, 1), eps or delta not finite and > 0, tau not finite, n_clamp < 2),
 * E_NOT_CONVERGED (a phase still had residues above its threshold after
 * 65,535 rounds), E_OOM, E_CUDA. */
int pprviz_tau_push(pprviz_ctx *ctx, const pprviz_graph *g, int32_t nsup, const int64_t *leaf_ptr,
                    const int32_t *leaf_idx, const double *dpr, double alpha, double eps, double delta, double tau,
                    void *ldppr_out, void *pdist_out, int64_t n_clamp, pprviz_tau_info *info, uint32_t mem_flags);

/* What one pprviz_louvain_plus call did (host struct). */
typedef struct pprviz_louvain_info {
    int32_t levels;           /* L: levels above the leaves */
    int32_t rounds;           /* merge rounds, all levels */
    int64_t parent_need;      /* sum_{l < L} level_n[l]: the parent entries needed */
    int64_t slot_visits;      /* pair-table slots cleared and scanned, all contractions */
    int64_t pair_visits;      /* pairs summed into the table, all contractions */
    int64_t list_visits;      /* pairs scanned for the gains, all rounds */
    int64_t node_visits;      /* level nodes processed, all rounds */
} pprviz_louvain_info;

/* Louvain+ supergraph hierarchy (Sec. 5, the preprocessing step; Appendix A,
 * "Louvain+"): level l+1 groups the supernodes of level l (level 0: the
 * leaves) so that no supernode has more than k children, and levels are added
 * until one has at most k supernodes. A supernode S is merged into a
 * neighbouring T by rule (i), T being S's only neighbour, or rule (ii), the T
 * of the largest modularity gain Q^(S, T) = sum_{V_i in S} q(V_i, T), with
 * w(.) and w_cr counted as ordered leaf pairs (the count under which q is the
 * change of modularity). Decisions use exact integer gains. Schedule (the
 * appendix fixes the rules, not their order): synchronous rounds; every
 * supernode proposes its target from the round's starting state (rule (ii)
 * only on a positive gain until a round of the level merges nothing, then on
 * any gain; ties to the smaller id); S moves when its target does not; a
 * target takes its movers in increasing id order while it keeps at most k
 * children. A level ends with a round that merges nothing; the hierarchy ends
 * when a level has at most k supernodes or merged nothing (so a graph of more
 * than k connected components keeps more than k supernodes at the top).
 * g:          an undirected graph; weights are ignored (edges are counted);
 *             fewer than 2^31 stored edges.
 * k:          children per supernode and supernodes at the top, at most; >= 2.
 * level_n:    host, level_cap + 1 int64: level_n[0] = n, level_n[l] = the
 *             number of level-l supernodes, l = 1..L.
 * parent:     host, parent_cap int32: for l = 1..L in turn, the level-l
 *             supernode of every level-(l-1) node (level_n[l - 1] entries),
 *             supernodes numbered from 0 in the order of their smallest child.
 * info:       host, required: what the call did (pprviz_louvain_info); its
 *             levels and parent_need are written also when parent_cap or
 *             level_cap is too small (E_INVALID_ARG, level_n and parent
 *             untouched).
 * Scratch (kept by the context): about 80 B per node, 24 B per stored edge
 * and a pair table of 12 B x the power of two >= 2 x the stored edges (each
 * contraction of the pair list clears and scans only the power of two it
 * needs).
 * Errors: E_INVALID_ARG (NULL, k < 2, a directed graph, short outputs),
 * E_NOT_CONVERGED (100,000 rounds or 64 levels), E_OOM, E_CUDA. */
int pprviz_louvain_plus(pprviz_ctx *ctx, const pprviz_graph *g, int32_t k, int64_t *level_n, int32_t level_cap,
                        int32_t *parent, int64_t parent_cap, pprviz_louvain_info *info);

/* P3 alone - PDist from a k*k DPPR matrix (Sec. 3.1, Eq. (1)):
 * Delta[i][j] = min(max(1 - ln(D[i][j] + D[j][i]), 2), 2 ln n_clamp), zero
 * diagonal, z = 0 mapped to the upper clamp. Types per PPRVIZ_OUT_FP64.
 * Errors: E_INVALID_ARG (k < 1, n_clamp < 2), E_OOM, E_CUDA. */
int pprviz_pdist(pprviz_ctx *ctx, const void *dppr, int32_t k, int64_t n_clamp,
                 void *pdist_out, uint32_t mem_flags);

/* P4-P5 - stress-majorization layout (Sec. 5, Eq. (7); Appendix A.1, Eq. (10)).
 * pdist:     k*k symmetric target distances, off-diagonal finite and > 0
 *            (the diagonal is ignored).
 * x0:        k*2 initial coordinates; x_out: k*2 result (may alias x0).
 * iters:     number of updates X <- (L^w)^+ L^Y(X) X, each the exact solve
 *            of Eq. (10) with the Moore-Penrose inverse of L^w; the result
 *            is centred (column means 0). iters = 0 only centres x0.
 * precision: PPRVIZ_FP64 (FP64 arithmetic throughout) or PPRVIZ_FP32.
 * stress_out: Eq. (7) at the final X, accumulated in FP64 (host); may be NULL.
 * Types per PPRVIZ_OUT_FP64 (pdist, x0, x_out).
 * Errors: E_INVALID_ARG (k < 1, iters < 0, a non-finite or non-positive
 * off-diagonal distance), E_OOM, E_CUDA. */
int pprviz_layout(pprviz_ctx *ctx, const void *pdist, int32_t k, const void *x0,
                  int32_t iters, int precision, void *x_out, double *stress_out,
                  uint32_t mem_flags);

/* P6 - stress energy and its gradients by pair recomputation (Sec. 5, Eq. (7)).
 * e_out:      L(X | Delta) summed over i < j in FP64 (host); may be NULL.
 * grad_x:     k*2, grad_scale * dL/dX_i = grad_scale * sum_j 2 (d_ij - Delta_ij)
 *             / (Delta_ij^2 d_ij) (X_i - X_j), 0 for coincident points; may be NULL.
 * grad_pdist: k*k, grad_scale * (1 - d_ij / Delta_ij) d_ij / Delta_ij^2 for
 *             i != j (the derivative of (1/2) sum_{i != j}, equal to Eq. (7) for
 *             symmetric Delta), 0 on the diagonal; may be NULL.
 * Float buffers (FP32 arithmetic, FP64 energy accumulation), or double with
 * PPRVIZ_OUT_FP64 (FP64 arithmetic).
 * Errors: E_INVALID_ARG, E_OOM, E_CUDA. */
int pprviz_energy(pprviz_ctx *ctx, const void *pdist, int32_t k, const void *x,
                  double grad_scale, double *e_out, void *grad_x, void *grad_pdist,
                  uint32_t mem_flags);

/* P7 - many independent views in one call (Sec. 2.2: the multi-level
 * mechanism visits the children of many supernodes). View v is its own
 * undirected graph (uploaded with pprviz_graph_upload); every node of it is a
 * source (k_v = n_v, n_clamp = n_v). For each view: DPPR (FP32 path, eps, the
 * same certificate as pprviz_dppr), PDist, then `iters` FP32
 * stress-majorization updates from its x0.
 * The propagation runs the views, largest first, as the disjoint union of
 * their graphs: consecutive views of similar size form a wave whose sources
 * advance together in every sweep launch; the layouts of all views share one
 * launch per pass.
 * nviews:      1 .. 65,535; the views hold at most 2^31 - 1 nodes in all.
 * offsets:     nviews+1 int64 prefix sums of n_v (host).
 * x0_packed:   sum n_v * 2 floats (view v at offsets[v]*2).
 * pdist_packed: sum n_v^2 floats (view v at the prefix sum of n_u^2, u < v);
 *              may be NULL.
 * x_packed:    sum n_v * 2 floats, the final layouts.
 * stress_out:  nviews doubles (host), final stress per view; may be NULL.
 * cert_out:    sum n_v doubles (host, packed like offsets): the DPPR
 *              certificate of each view's source rows; may be NULL.
 * Errors: as pprviz_dppr and pprviz_layout. */
int pprviz_views_batch(pprviz_ctx *ctx, int32_t nviews, const pprviz_graph *const *views,
                       const int64_t *offsets, double alpha, double eps, int32_t iters,
                       const float *x0_packed, float *pdist_packed, float *x_packed,
                       double *stress_out, double *cert_out, uint32_t mem_flags);

/* Layout quality metrics (Sec. 2, visualization quality assessment):
 *   ND(X)   = sum_{i<j} 1 / |X_i - X_j|^2 (node distribution; +inf when two
 *             points coincide);
 *   ULCV(X) = l_sigma / l_mu of the edge lengths (uniform length coefficient
 *             variance; population standard deviation; each undirected edge
 *             once; NaN when the view holds no edge).
 * x:        k*2 coordinates (float, or double with PPRVIZ_OUT_FP64), host or
 *           device per PPRVIZ_DEVICE_PTRS; sums are accumulated in FP64 in a
 *           fixed order.
 * g, view:  the graph whose edges ULCV measures and the k node ids of the rows
 *           of x (NULL view: k = n and row i is node i); the edges are those
 *           of g between view nodes. g may be NULL when ulcv_out is NULL.
 * nd_out, ulcv_out: host doubles; either may be NULL.
 * Errors: E_INVALID_ARG (k < 1, no graph for ULCV, k != n without a view, a
 * bad view id), E_OOM, E_CUDA. */
int pprviz_layout_metrics(pprviz_ctx *ctx, const void *x, int32_t k, const pprviz_graph *g, const int32_t *view,
                          double *nd_out, double *ulcv_out, uint32_t mem_flags);

/* Stress energy and gradients without allocating anything (no counterpart in
 * the paper; a library convenience). Same results as pprviz_energy with FP32
 * device buffers, for callers that may not allocate device memory when they
 * call: code whose device memory is all owned by its own pool or a
 * framework's allocator, code under a hard memory cap, or code that may only
 * enqueue work on a stream it was handed.
 * pdist, x:   device pointers (k*k and k*2 float), as in pprviz_energy.
 * grad_x, grad_pdist: device outputs or NULL; e_out: host double or NULL.
 * cuda_stream: the stream to run on (NULL = the legacy default stream); the
 *             call waits for that stream before it returns, to read back the
 *             energy and the status word. No context is needed: the call runs
 *             on the current device, in its primary context (the one the CUDA
 *             runtime API uses).
 * Scratch: a fixed device array inside the library (about 528 KiB, held by
 * every GPU that loads the library until the process exits), so k is limited
 * to 65,536. The first call on a device looks up the array's device address
 * in that device's primary context (once per device, with that device
 * current); make that first call on each device before any stream capture.
 * Every call shares the array and the calls clear what must start at zero,
 * but calls that overlap on the GPU (two streams, two threads) race on it
 * and must be serialised by the caller.
 * Returns PPRVIZ_OK, PPRVIZ_E_INVALID_ARG (NULL input, k outside [1, 65536],
 * a non-positive off-diagonal distance) or PPRVIZ_E_CUDA; no error message is
 * kept since there is no context. */
int pprviz_energy_noalloc(const float *pdist, int32_t k, const float *x, double grad_scale, double *e_out,
                          float *grad_x, float *grad_pdist, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PPRVIZ_H */
