/*
 * gazecut.h -- C ABI of the GB300 (sm_103a) exact min-cut for the gaze-line /
 * depth-number stereo formulation of Oguri & Shibata, "A new stereo
 * formulation not using pixel and disparity models" (arXiv 1803.01516).
 *
 * Pipeline (one stereo pair):
 *   gs_stereo_cost_volume   data term g_v at every cross point        (§4.3, §3)
 *   gs_build_graph          chain graph of the convex prior, with the
 *                           terminal arcs folded into node excess     (§2 Eq. 1, §3, Fig. 4, §4.4)
 *   gs_maxflow_solve        push-relabel with global relabelling      (§4.4)
 *   gs_extract_labels       the cut as one depth number per gaze line (§3 "real cross points")
 *
 * Geometry.  The paper leaves the cuboid offsets out (§4.1); this library
 * fixes them so that every cross point lies inside both images:
 *   depth numbers S in [0, D), disparity dis(S) = dis0 - 2S, dis0 >= 2(D-1);
 *   sites (gaze lines) W in [0, n_g), n_g = w - dis0, rows y in [0, h);
 *   cross point (W, S, y) pairs right pixel x_r = W + S with left pixel
 *   x_l = W + dis0 - S.
 *
 * Energy (§2, §3):  E(X) = sum_v C_v(X_v) + sum_(u,v) h~(X_u - X_v),
 *   h~(d) = lambda |d| + inhibit (|d| - 1) [|d| > 1]
 * over 4-connected sites; vertical pairs carry the inhibit term only when
 * vertical_inhibit != 0.  The solve is exact: the flow value equals min E and
 * the labels are the component-wise smallest minimiser (read from the
 * minimal source set of the cut), so they do not depend on the schedule.
 *
 * Conventions shared by every call:
 *   - All array pointers are DEVICE pointers owned by the caller unless a
 *     parameter says "host".  The library allocates nothing; the caller sizes
 *     buffers with the *_bytes() queries.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call is stream-ordered and asynchronous unless stated.
 *   - Host return value: GS_OK, GS_ERR_INVAL (bad sizes, NULL or misaligned
 *     pointer; nothing was launched) or GS_ERR_CUDA (a launch failed).
 *     Errors found on the device (overflow, non-converged solve) are written
 *     to the caller's device status word instead, so no call needs a host
 *     synchronisation.
 *   - Device buffers must be 256-byte aligned (cudaMalloc / torch give this).
 */
#ifndef GAZECUT_H
#define GAZECUT_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (host return values and device status words). */
#define GS_OK            0
#define GS_ERR_INVAL     1   /* bad argument; or a negative data cost seen on the device */
#define GS_ERR_OVERFLOW  2   /* capacities / flow would not fit the int32 state */
#define GS_ERR_TIMEOUT   3   /* max_iters reached, or the idle limit ran out, before the cut was
                                exact; the state stays a valid preflow and the solve resumes */
#define GS_ERR_CUDA      4   /* a CUDA launch or copy failed */
#define GS_ERR_LABELS    5   /* the cut was not one depth number per gaze line (internal check) */
#define GS_ERR_TOO_LARGE 6   /* the problem needs more scratch than gs_noalloc_scratch_bytes() */

/* Problem description.  tau is used by the cost-volume call only. */
typedef struct gs_params {
    int32_t w, h;              /* image size in pixels (both images) */
    int32_t D;                 /* number of depth numbers (labels), D >= 2 */
    int32_t dis0;              /* disparity of depth number 0, dis0 >= 2(D-1), w - dis0 >= 1 */
    int32_t tau;               /* truncation of the absolute-difference data term, >= 0 */
    int32_t lambda;            /* penalty h~1 (smoothness), 0 <= lambda <= 2^28 */
    int32_t inhibit;           /* inhibit h~2 (visibility), 0 <= inhibit <= 2^29 */
    int32_t vertical_inhibit;  /* 1: inhibit on vertical pairs too; 0: horizontal pairs only */
    int32_t direction;         /* max-flow direction: 0 auto, 1 as given, 2 label-reversed
                                  (the reversed graph; same min energy and canonical labels).
                                  Auto takes the side with the smaller source capacity. */
} gs_params;

/* Solve modes. */
#define GS_MODE_EXACT        0  /* iterate until no active node can reach the sink */
#define GS_MODE_FIXED_SWEEPS 1  /* stop after fixed_sweeps local sweeps (approximate cut) */

/* Solver engines.  Both compute the same exact cut; they differ in schedule.
 *   TILED   one persistent cooperative launch: shared-memory tiles of whole
 *           depth chains, local push/relabel iterations, tile-local relabel
 *           passes, tiles claimed per step from device-side queues, no host
 *           synchronisation (default)
 *   SIMPLE  one thread per node, one kernel per sweep / relabel pass, host loop
 *           (a second, independent schedule kept for cross-checking) */
#define GS_ENGINE_TILED  0
#define GS_ENGINE_SIMPLE 1

typedef struct gs_solve_opts {
    int32_t mode;                /* GS_MODE_* */
    int32_t sweeps_per_relabel;  /* sweep rounds between global relabels (>= 1) */
    int32_t fixed_sweeps;        /* GS_MODE_FIXED_SWEEPS: total sweeps */
    int32_t engine;              /* GS_ENGINE_* */
    int64_t max_iters;           /* cap on global relabels in exact mode (> 0) */
    int32_t local_iters;         /* TILED: push/relabel iterations per tile visit (0: 8) */
    int32_t relabel_passes;      /* TILED: tile passes of an intermediate global relabel
                                    (0: 8); the relabel that decides termination always
                                    runs to its fixed point */
    int32_t tail_iters;          /* TILED: local iterations per tile visit once few nodes
                                    are active (0: 4 x local_iters) */
    int32_t tile_w, tile_h;      /* TILED: sites per tile along W (4, 8, 16 or 32) and
                                    rows per tile (1..8); 0, 0: chosen by the library.
                                    A shape that does not fit shared memory is refused
                                    (GS_ERR_INVAL). */
    int32_t idle_limit_us;       /* TILED: a block of the persistent launch that finds no
                                    work for this long gives up, and the pairs still
                                    running end with GS_ERR_TIMEOUT (state valid,
                                    resumable); 0: 60 s.  In a batch the smallest
                                    non-zero value among the descriptors applies. */
    int32_t cta_threads;         /* TILED: threads per block of the persistent launch,
                                    0 or 512 (one block per SM) or 256 (two blocks per
                                    SM when two tiles fit its shared memory, each
                                    tile on half the threads).  A batch runs 256 only
                                    when every descriptor asks for it. */
} gs_solve_opts;

/* Host-side check of solve options (the same checks gs_maxflow_solve and
 * gs_solve_batched apply): GS_OK or GS_ERR_INVAL (unknown mode or engine,
 * sweeps_per_relabel < 1, max_iters < 1, a negative count, fixed_sweeps < 0 in
 * GS_MODE_FIXED_SWEEPS, idle_limit_us < 0, cta_threads not 0, 256 or 512). */
GS_API int gs_check_solve_opts(const gs_solve_opts *o);

/* Derived sizes (0 when the params are invalid). */
GS_API int32_t gs_num_sites_w(const gs_params *p);           /* n_g = w - dis0 */
GS_API size_t  gs_cost_volume_bytes(const gs_params *p);     /* int32 [h][n_g][D] */
GS_API size_t  gs_graph_bytes(const gs_params *p);           /* opaque solver state */
GS_API size_t  gs_workspace_bytes(const gs_params *p, const gs_solve_opts *o);
GS_API int64_t gs_num_nodes(const gs_params *p);             /* graph nodes without s, t: n_g*h*(D-1) */

/*
 * Data term g_v (§4.3, grayscale form, truncated as the workloads specify):
 *   cost[(y*n_g + W)*D + S] = min(|L[y*pitch + W+dis0-S] - R[y*pitch + W+S]|, tau)
 * L, R: uint8 images, row pitch `pitch` bytes (>= w).  cost: int32, layout
 * [h][n_g][D] (one contiguous depth chain per site), gs_cost_volume_bytes().
 * Rows are staged with 128-bit loads when both images and the pitch are
 * 16-byte aligned; no byte outside a row's first w is read.
 */
GS_API int gs_stereo_cost_volume(const uint8_t *L, const uint8_t *R, int32_t pitch, const gs_params *p,
                          int32_t *cost, void *stream);

/*
 * Colour data term of §4.3, the form the paper uses:
 *   cost[(y*n_g + W)*D + S] = min(|L_R - R_R| + |L_G - R_G| + |L_B - R_B|, tau)
 * with (L_R, L_G, L_B) the left pixel (x_l, y) = (W+dis0-S, y) and
 * (R_R, R_G, R_B) the right pixel (x_r, y) = (W+S, y); each sum lies in
 * [0, 765], so tau >= 765 gives the paper's plain sum of absolute differences.
 * L, R: interleaved 8-bit RGB (3 bytes per pixel, R first), row pitch `pitch`
 * bytes (>= 3w); rows are staged with 128-bit loads when both images and the
 * pitch are 16-byte aligned.  cost: layout and size as gs_stereo_cost_volume.
 */
GS_API int gs_stereo_cost_volume_rgb(const uint8_t *L, const uint8_t *R, int32_t pitch,
                                     const gs_params *p, int32_t *cost, void *stream);

/*
 * Chain graph of §3 / Fig. 4 (Ishikawa construction for the convex h~ of Eq. 1):
 *   chain node n(v, k), k in [1, D-1]; data arc n(v,k) -> n(v,k+1) carries
 *   C_v(k) with an infinite reverse arc; penalty arcs u_k <-> v_k carry lambda;
 *   inhibit arcs u_k -> v_(k-1), k >= 2, carry inhibit.  The source arc C_v(0)
 *   and sink arc C_v(D-1) are folded into positive / negative node excess
 *   (§4.4); heights start at 0.
 * Initial flow (the stand-in for the paper's undisclosed "wave front fetch"
 * pre-pass, §4.4): every chain starts with its own largest flow already pushed
 * down it, node n_k holding min C(0..k-1) - min C(0..k) and the data arcs
 * carrying the prefix minima; the max-flow only routes what the interaction
 * terms change.  The cut is the same with or without it (see
 * gs_build_graph_flags).
 * cost: int32 [h][n_g][D], every entry >= 0.  graph: gs_graph_bytes() bytes,
 * written entirely.  status: device int32[1], set to GS_OK, GS_ERR_INVAL
 * (negative cost) or GS_ERR_OVERFLOW (sum of source capacities > 2^30 or a
 * cost > 2^30).
 */
#define GS_BUILD_CHAIN_PREFLOW 1   /* chain-local initial flow (gs_build_graph's default) */

/* gs_build_graph with explicit build flags (0 or GS_BUILD_CHAIN_PREFLOW).  With
 * flags = 0 only the source arcs start saturated (n_1 holds C(0), the last node
 * a deficit of C(D-1), every data arc unused): the textbook initial preflow,
 * kept to measure what the pre-pass saves.  GS_ERR_INVAL for unknown flags. */
GS_API int gs_build_graph_flags(const int32_t *cost, const gs_params *p, int32_t flags,
                                void *graph, int32_t *status, void *stream);

GS_API int gs_build_graph(const int32_t *cost, const gs_params *p, void *graph, int32_t *status,
                   void *stream);

/*
 * Max-flow on the graph state in place (§4.4): local push/relabel sweeps with
 * a periodic global relabel (breadth-first distances to the remaining sink
 * capacity), until no node with excess can reach the sink (GS_MODE_EXACT) or
 * for a fixed number of sweeps (GS_MODE_FIXED_SWEEPS).
 * workspace: gs_workspace_bytes() bytes of scratch, contents ignored on entry.
 * status: device int32[1]; left as is when it already holds an error,
 * otherwise set to GS_OK or GS_ERR_TIMEOUT (max_iters reached: the state is a
 * valid preflow and the call can be repeated to continue) or GS_ERR_OVERFLOW.
 */
GS_API int gs_maxflow_solve(void *graph, const gs_params *p, const gs_solve_opts *o, void *workspace,
                     int32_t *status, void *stream);

/*
 * Labels and flow value from the solved state.
 * GS_MODE_EXACT: S_min = nodes reachable from a node with positive excess in
 *   the residual graph; labels[y*n_g + W] = |S_min ∩ chain(W, y)|, the
 *   smallest minimiser of E.  flow = value of the maximum flow = min E.
 * GS_MODE_FIXED_SWEEPS: the source side is the set of nodes that cannot reach
 *   the sink (valid for any preflow); flow = flow routed so far (a lower
 *   bound on min E).
 * labels: int32 [h][n_g].  flow: device int64[1].  status as above
 * (GS_ERR_LABELS if a chain's source side is not a prefix).
 */
GS_API int gs_extract_labels(void *graph, const gs_params *p, const gs_solve_opts *o, void *workspace,
                      int32_t *labels, int64_t *flow, int32_t *status, void *stream);

/*
 * Learned data term (the paper's g_v generalised to a trainable matching cost;
 * the paper tunes h~1 by grid search, §4.3): at every cross point
 *   c = w1 |L - R| + w2 |dxL - dxR|,  dx = central difference with replicated
 *   border,  cost = rint(scale * min(c, tau))   (round half to even)
 * computed in FP32 with every product and sum rounded separately (no fused
 * multiply-add).  Layout and arguments as gs_stereo_cost_volume; w1, w2,
 * tau >= 0, scale > 0; GS_ERR_OVERFLOW when scale * tau > 2^30.
 */
GS_API int gs_stereo_cost_volume_f32(const uint8_t *L, const uint8_t *R, int32_t pitch,
                                     const gs_params *p, float w1, float w2, float tau, float scale,
                                     int32_t *cost, void *stream);

/*
 * Adjoint of the minimum energy E* (§2) at a minimiser X (int32 [h][n_g]):
 *   dE/dC[v][l] = [X_v = l]; written as grad * one-hot into dcost (float
 *   [h][n_g][D]) when dcost is not NULL;
 *   counts (device int64[2]) = { sum |X_u - X_v| = dE/dlambda,
 *                                sum (|X_u - X_v| - 1)_+ = dE/dinhibit }
 *   over the 4-connected pairs (vertical pairs in the second sum only when
 *   vertical_inhibit).  E* is concave and piecewise linear in the costs and
 *   weights: these are its gradients where the minimiser is unique.
 */
GS_API int gs_energy_backward(const int32_t *labels, const gs_params *p, float grad, float *dcost,
                              int64_t *counts, void *stream);

/*
 * Chain rule through gs_stereo_cost_volume_f32 at the labels X: device
 * int64[3] = { sum_v |L - R| [c < tau], sum_v 2 |dxL - dxR| [c < tau],
 *              sum_v [c >= tau] }, c taken at (v, X_v).  With the quantiser
 * treated as the identity, dE/dw1 = sums[0], dE/dw2 = sums[1] / 2,
 * dE/dtau = sums[2] (energy in cost units).
 */
GS_API int gs_cost_volume_f32_backward(const uint8_t *L, const uint8_t *R, int32_t pitch,
                                       const gs_params *p, float w1, float w2, float tau,
                                       const int32_t *labels, int64_t *sums, void *stream);

/* cost[v][labels[v]] += value for every site (labels outside [0, D) are
 * skipped): the loss augmentation of structured learning, where adding a
 * constant to the ground-truth label's cost equals subtracting the Hamming
 * loss up to a constant. */
GS_API int gs_cost_add_at_labels(int32_t *cost, const int32_t *labels, const gs_params *p,
                                 int32_t value, void *stream);

/* E(X) of §2 for labels int32 [h][n_g] over cost [h][n_g][D]; energy: device int64[1],
 * negative if a label lies outside [0, D). */
GS_API int gs_energy(const int32_t *cost, const int32_t *labels, const gs_params *p, int64_t *energy,
              void *stream);

/* Diagnostics of the last solve on this workspace: host int64[10] =
 * {global relabels, sweep rounds, relabel passes, label-extraction passes (0
 *  when the extraction read the finished solve's exact distances),
 *  active nodes at exit, device time of the sweep rounds in ns, device time
 *  of the global relabels in ns, kernel launches of the solve, tile visits of
 *  the sweep rounds, tile visits of the relabel passes}.  The times come from
 * the device's global timer (TILED) or CUDA events on the solve's stream
 * (SIMPLE); the visit counts are 0 for the SIMPLE engine.  Synchronises
 * `stream`. */
GS_API int gs_solve_stats(const void *workspace, int64_t *host_stats, void *stream);

/*
 * Batched solve: n stereo pairs of any sizes and depth ranges (n <= 64), each
 * through the whole path (data term, graph, exact max-flow, labels), with the
 * max-flows of all pairs in ONE persistent cooperative launch and the label
 * extractions in one more.  Pairs advance through their own relabel / sweep
 * schedule inside the shared launch, so tiles of pairs still working fill
 * the grid while others are done.  Every launch is stream-ordered with no host
 * synchronisation, so the call can be captured in a CUDA graph.
 * descs: HOST array of n descriptors whose pointers are device buffers sized
 * by the single-pair queries; opts.engine must be GS_ENGINE_TILED.
 * batch_workspace: gs_batch_workspace_bytes(n) device bytes (256-aligned).
 * Results per pair as for gs_extract_labels; statistics via gs_solve_stats on
 * the pair's workspace.
 */
typedef struct gs_pair_desc {
    gs_params p;
    gs_solve_opts o;
    const uint8_t *L, *R;      /* device images, row pitch = p.w bytes */
    int32_t *cost;             /* gs_cost_volume_bytes(&p) */
    void *graph;               /* gs_graph_bytes(&p) */
    void *workspace;           /* gs_workspace_bytes(&p, &o) */
    int32_t *labels;           /* int32 [h][n_g] */
    int64_t *flow;             /* int64 [1] */
    int32_t *status;           /* int32 [1] */
} gs_pair_desc;

GS_API size_t gs_batch_workspace_bytes(int32_t n);
GS_API int gs_solve_batched(const gs_pair_desc *descs, int32_t n, void *batch_workspace,
                            void *stream);

/*
 * Level-1 hierarchical approximation (§4.5).  The paper combines b x b x b
 * neighbouring cross points into a delegate point, cuts the delegate graph,
 * then cuts exactly among the cross points of a thin skin around that cut.
 * It leaves the delegate terms and the skin open; this library fixes them:
 *
 *   delegate site (Wc, yc) = sites W in [b Wc, b Wc + b), y in [b yc, b yc + b)
 *   delegate depth number Lc = depth numbers [b Lc, b Lc + b)   (fewer at the
 *     far edges); n_gc = ceil(n_g / b), h_c = ceil(h / b), D_c = ceil(D / b)
 *   delegate data term  Cc(Wc, yc, Lc) = sum over the block's sites of the
 *     smallest data term in the depth bin
 *   delegate interaction  h~ of §3 with lambda and inhibit multiplied by b
 *   thin skin  a site whose delegate has label Lc keeps the depth numbers
 *     [b Lc - b, b Lc + 2b - 1] clipped to [0, D-1]
 *   second cut  the exact minimum of E (§2) over labelings inside the skin;
 *     its canonical (smallest) minimiser
 *
 * b = 1 gives the exact cut.  A caller runs: gs_delegate_params,
 * gs_delegate_cost, the exact path on the delegate problem (gs_build_graph,
 * gs_maxflow_solve, gs_extract_labels), gs_skin_bounds on the delegate labels,
 * gs_build_graph_skin, then gs_maxflow_solve and gs_extract_labels with the
 * fine params.
 */

/* Params of the delegate problem for block size b (host; 1 <= b < D):
 * w = n_gc + dis0_c, h = h_c, D = D_c, dis0 = 2 (D_c - 1), lambda and inhibit
 * times b, the rest copied.  GS_ERR_INVAL for bad params or b, GS_ERR_OVERFLOW
 * when the scaled weights leave their range. */
GS_API int gs_delegate_params(const gs_params *p, int32_t b, gs_params *out);

/* Delegate data term: coarse[(yc*n_gc + Wc)*D_c + Lc] (int32, layout of a cost
 * volume of the delegate problem) from cost (layout of gs_stereo_cost_volume).
 * status: device int32[1], set to GS_OK, GS_ERR_INVAL (a negative cost) or
 * GS_ERR_OVERFLOW (a delegate term above 2^30). */
GS_API int gs_delegate_cost(const int32_t *cost, const gs_params *p, int32_t b, int32_t *coarse,
                            int32_t *status, void *stream);

/* Skin bounds lo, hi (int32 [h][n_g] each, device) from the delegate labels
 * (int32 [h_c][n_gc], device).  status: device int32[1], GS_ERR_LABELS when a
 * delegate label is outside [0, D_c), else left as is. */
GS_API int gs_skin_bounds(const int32_t *coarse_labels, const gs_params *p, int32_t b, int32_t *lo,
                          int32_t *hi, int32_t *status, void *stream);

/*
 * Graph of the second cut: the chain graph of gs_build_graph for the problem
 * as given (p->direction is ignored; the label-reversed twin is never taken)
 * with every site's labels held in [lo, hi] (int32 [h][n_g] each, device,
 * 0 <= lo <= hi <= D-1).  X >= lo holds n_1..n_lo on the source side and
 * X <= hi holds n_hi+1..n_(D-1) on the sink side; held nodes are contracted
 * into the terminals (arcs from source-held into free nodes become source
 * capacity of the free node, arcs from free into sink-held nodes sink
 * capacity), so only the nodes of the skin carry flow.  Solve with
 * GS_MODE_EXACT.  The flow value gs_extract_labels reports for this graph is
 * that of the contracted graph; the energy of the labels (gs_energy) is the
 * restricted minimum.  status as gs_build_graph, plus GS_ERR_INVAL for bounds
 * out of order.
 */
GS_API int gs_build_graph_skin(const int32_t *cost, const gs_params *p, const int32_t *lo,
                               const int32_t *hi, void *graph, int32_t *status, void *stream);

/*
 * Level-2 hierarchical approximation (§4.5).  The paper's level 2 keeps the
 * level-1 delegate cut and thin skin, but its push-relabel loop cuts each
 * block separately while an undisclosed wave-front pass covers the skin as a
 * whole.  This library fixes that reading as block-coordinate descent inside
 * the skin:
 *
 *   start labels  each site's first argmin of the data term inside its
 *                 delegate's depth bin [b Xc, min(b Xc + b, D) - 1]
 *   block cut     block (bx, by) = sites W in [b bx, b bx + b), y in
 *                 [b by, b by + b); with every other site held at its current
 *                 label, the block's labels become the exact minimum of E (§2)
 *                 inside lo <= X <= hi, canonical (smallest) minimiser; the
 *                 pairs leaving the block act as data terms h~(l - X_u)
 *   order         a pass cuts every block with (bx + by) even, then every
 *                 block with (bx + by) odd against the new labels (blocks of
 *                 one colour share no pair, so E never increases)
 *
 * A caller runs the level-1 steps up to gs_skin_bounds, then gs_level2_start
 * on the delegate labels, then gs_block_descent.  The labels are read from
 * `labels` (no flow value: the result is not a cut of the whole graph); its
 * energy is gs_energy.
 */

/* Start labels (int32 [h][n_g], device) from the delegate labels (int32
 * [h_c][n_gc], device) of block size b (1 <= b < D) over the data term cost.
 * status: device int32[1], GS_ERR_LABELS when a delegate label is outside
 * [0, D_c), else left as is. */
GS_API int gs_level2_start(const int32_t *cost, const gs_params *p, int32_t b,
                           const int32_t *coarse_labels, int32_t *labels, int32_t *status,
                           void *stream);

/* `passes` two-colour passes of exact block cuts (block size 1 <= b <= 3) on
 * labels (int32 [h][n_g], device, updated in place; every label inside its
 * bounds lo, hi on entry).  One warp solves a block by dynamic programming over
 * row states, so a block's label range (the union of its sites' bounds) may
 * hold at most min(3b, D) labels -- what gs_skin_bounds gives; a wider one
 * sets GS_ERR_INVAL in status and leaves that block as it is.  2 passes = 4
 * launches, stream-ordered, no host synchronisation. */
GS_API int gs_block_descent(const int32_t *cost, const gs_params *p, int32_t b,
                            const int32_t *lo, const int32_t *hi, int32_t *labels,
                            int32_t passes, int32_t *status, void *stream);

/* Tile shape the TILED engine uses for these params and options: host
 * int32[4] = {sites per tile along W, rows per tile, number of tiles, shared
 * bytes}.  GS_ERR_INVAL if the requested shape does not fit. */
GS_API int gs_tile_info(const gs_params *p, const gs_solve_opts *o, int32_t *out);

/* Number of kernels this library has launched in this process so far. */
GS_API int64_t gs_kernel_launches(void);

/*
 * gs_maxflow_solve without a workspace argument (the paper has no
 * counterpart: this is an interface for callers of the library).
 *
 * For callers that cannot allocate device memory when they solve, e.g. a
 * real-time loop that reserves all its memory at start-up, or a plug-in whose
 * host application owns the device allocator.  The solver's scratch lives in
 * a library-owned static device array of gs_noalloc_scratch_bytes() bytes
 * (16 MiB) that every GPU loading this library holds until the process exits.
 * The call itself allocates nothing.
 *
 * graph, p, o, status, stream: as for gs_maxflow_solve; o->engine must be
 * GS_ENGINE_TILED.  Returns GS_ERR_TOO_LARGE, before any device work, when the
 * problem needs more scratch than the array holds (about 6.5 bytes per graph
 * node: 384x288 with 16 depth numbers fits, 1920x1080 with 128 does not).
 * The first call on each device looks up the array's device address with that
 * device current; make that first call before any stream capture.  All calls
 * share the one array (it keeps the last call's contents; the solve clears
 * what must start at zero), so calls that overlap on the GPU race: issue them
 * on one stream or serialise them.  gs_extract_labels still takes its own
 * workspace.  The solve's statistics land in the shared array too:
 * gs_solve_stats has no workspace to read them from for this call, and the
 * next call overwrites them.
 *
 * The graph must live on the current device (the device whose array and
 * stream the call uses); the Python binding refuses a tensor on another one.
 */
GS_API size_t gs_noalloc_scratch_bytes(void);
GS_API int gs_maxflow_solve_noalloc(void *graph, const gs_params *p, const gs_solve_opts *o,
                                    int32_t *status, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GAZECUT_H */
