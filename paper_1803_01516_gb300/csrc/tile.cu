// Persistent, tiled push-relabel with global relabelling (§4.4) for the chain
// graph of §3 / Fig. 4.
//
// One cooperative launch runs the whole solve.  The node grid is cut into
// tiles of TW sites x TH rows x all K chain layers (whole chains, so the data
// arcs and their infinite reverse arcs never leave a tile).  A CTA stages a
// tile plus a one-site halo in shared memory and works on it locally; tiles
// exchange flow only through atomics on global memory, and a pair's steps
// (see "the solve loop" below) separate its phases:
//
//   global relabel  heights = breadth-first distance to the nearest node with
//                   sink capacity left, computed as a monotone relaxation:
//                   every tile relaxes to its local fixed point in shared
//                   memory, passes repeat until a whole pass changes nothing
//                   (the exact distances); the pass also counts active nodes
//                   (positive excess, finite height); zero active nodes means
//                   the preflow is maximum and the solve ends.
//   sweep rounds    every tile with active nodes runs up to `local_iters`
//                   push/relabel iterations in shared memory; pushes to halo
//                   nodes go to global memory at once, and the tile writes its
//                   own changes back as deltas, so concurrent tiles compose.
//
// Correctness does not depend on the interleaving: every push moves at most
// the excess and the residual its tile can see, and both only grow under
// other tiles' updates, so the state stays a valid preflow; heights only steer
// pushes.  The exit test is the exact reachability computed by the relabel.
#include <cstring>
#include <mutex>

#include "arcs.cuh"

namespace gs {

constexpr int kTileThreads = 512;            // threads per block (256 on request: two per SM)
constexpr int kInitOuter = 2;                 // relaxation rounds of a first relabel pass
constexpr int kMaxTileNodes = 4096;           // own nodes per tile (8 per thread at most)

struct TileGeom {
    int TW, TH;        // sites per tile along W and y
    int PW;            // padded row length TW + 2
    int SJ;            // shared-memory stride of one chain layer (= PW)
    int SYs;           // shared-memory stride of one row of sites: K * PW, padded
                       // to SYs = TW (mod 32) when R > 0
    int PN;            // padded nodes per tile (TH + 2) * SYs
    int TN;            // own nodes per tile TH * K * TW
    int R;             // rows of sites one warp covers (32 / TW), 0: layers instead
    int spread;        // R > 0: warp group g of the tile holds row group (g * spread) mod
                       // (TN / 32), so a warp's groups lie far apart in the tile
    int tiles_w, tiles_h, T;
};

struct SolveArgs {
    Geom g;
    TileGeom t;
    State s;
    uint16_t *amask;     // per node: residual-arc bits (14) | has-excess bit (15)
    int32_t *tile_act;   // [2][T] tiles with work in the current / next sweep round
    int32_t *tile_dirty; // [2][T] tiles whose halo heights changed in the last relabel pass
    int32_t *tile_cnt;   // [T] active nodes per tile after its last relabel pass
    int32_t *tile_list;  // [3][T] tiles queued for a step (slot = step mod 3)
    int32_t *hgt;        // distances the relabel passes compute (state heights, or marks)
    int dir;             // 0: distance to sink capacity over out-arcs (heights);
                         // 1: distance from positive excess over in-arcs (reachability);
                         // 2: label extraction of an exact solve, 1 unless the state is
                         //    the label-reversed problem, then 0
    Ctrl *ctrl;          // the pair's control block (statistics)
    int32_t *status;     // the caller's device status word
    int32_t *labels;     // label extraction output [h][n_g]
    int64_t *flow;       // label extraction output [1]
    int mode, sweeps_per_relabel, local_iters, relabel_passes, tail_iters;
    long long fixed_sweeps, max_iters;
    int npt;             // own nodes per thread of the pair's tile shape (4 or 8)
};

// Every read of solver state inside the persistent kernel bypasses L1: other
// SMs update the same words during the launch, and L1 is not coherent.
template <class T>
__device__ __forceinline__ T ld(const T *p) { return __ldcg(p); }

// Block-wide sum (all threads get the total).
__device__ __forceinline__ long long block_sum(long long v) {
    __shared__ unsigned long long s_sum;
    __syncthreads();
    if (threadIdx.x == 0) s_sum = 0;
    __syncthreads();
    if (v) atomicAdd(&s_sum, (unsigned long long)v);
    __syncthreads();
    return (long long)s_sum;
}

__device__ __forceinline__ bool aborted(Ctrl *ctrl) {
    return *(volatile int32_t *)&ctrl->abort != 0;
}

__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Atomics with acquire / release semantics at GPU scope (one instruction in
// place of a fence and a relaxed atomic).
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v) {
    unsigned r;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "r"(v) : "memory");
    return r;
}
__device__ __forceinline__ unsigned long long atom_add_acquire(unsigned long long *p,
                                                             unsigned long long v) {
    unsigned long long r;
    asm volatile("atom.acquire.gpu.global.add.u64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
    return r;
}
__device__ __forceinline__ unsigned long long atom_exch_release(unsigned long long *p,
                                                              unsigned long long v) {
    unsigned long long r;
    asm volatile("atom.release.gpu.global.exch.b64 %0, [%1], %2;" : "=l"(r) : "l"(p), "l"(v) : "memory");
    return r;
}

// ------------------------------------------------------- tile addressing ---

struct TileSmem {
    int32_t *ht, *ex, *rc, *rr, *rd, *ri0, *ri1, *ri2, *ri3;
};

__device__ __forceinline__ TileSmem tile_smem(int32_t *base, int PN) {
    TileSmem m;
    m.ht = base;
    m.ex = base + PN;
    m.rc = base + 2 * PN;
    m.rr = base + 3 * PN;
    m.rd = base + 4 * PN;
    m.ri0 = base + 5 * PN;
    m.ri1 = base + 6 * PN;
    m.ri2 = base + 7 * PN;
    m.ri3 = base + 8 * PN;
    return m;
}

// shared-memory index of tile position (yl, j, wl), yl in [-1, TH], wl in [-1, TW]
__device__ __forceinline__ int pidx(const TileGeom &t, int yl, int j, int wl) {
    return (yl + 1) * t.SYs + j * t.SJ + (wl + 1);
}

// slot -> (dy, dj, dw)
__device__ __forceinline__ void slot_delta(int q, int &dy, int &dj, int &dw) {
    switch (q) {
        case 0: dy = 0; dj = 1; dw = 0; return;
        case 1: dy = 0; dj = -1; dw = 0; return;
        case 2: dy = 0; dj = 0; dw = 1; return;
        case 3: dy = 0; dj = 0; dw = -1; return;
        case 4: dy = 1; dj = 0; dw = 0; return;
        case 5: dy = -1; dj = 0; dw = 0; return;
        case 6: dy = 0; dj = -1; dw = -1; return;
        case 7: dy = 0; dj = -1; dw = 1; return;
        case 8: dy = -1; dj = -1; dw = 0; return;
        case 9: dy = 1; dj = -1; dw = 0; return;
        case 10: dy = 0; dj = 1; dw = -1; return;
        case 11: dy = 0; dj = 1; dw = 1; return;
        case 12: dy = -1; dj = 1; dw = 0; return;
        default: dy = 1; dj = 1; dw = 0; return;
    }
}

__device__ __forceinline__ int soff(const TileGeom &t, int q) {
    int dy, dj, dw;
    slot_delta(q, dy, dj, dw);
    return dy * t.SYs + dj * t.SJ + dw;
}

// Which arcs of a node exist (grid border, chain ends, vertical inhibit off).
__device__ __forceinline__ unsigned arc_exists(const Geom &g, int y, int j, int W) {
    const bool up = j < g.K - 1, dn = j > 0;
    const bool l = W > 0, r = W < g.ng - 1, u = y > 0, d = y < g.h - 1;
    unsigned m = 0;
    m |= up ? 1u << 0 : 0;
    m |= dn ? 1u << 1 : 0;
    m |= r ? 1u << 2 : 0;
    m |= l ? 1u << 3 : 0;
    m |= d ? 1u << 4 : 0;
    m |= u ? 1u << 5 : 0;
    m |= (dn && l) ? 1u << 6 : 0;
    m |= (dn && r) ? 1u << 7 : 0;
    m |= (dn && u) ? 1u << 8 : 0;
    m |= (dn && d) ? 1u << 9 : 0;
    m |= (up && l) ? 1u << 10 : 0;
    m |= (up && r) ? 1u << 11 : 0;
    m |= (up && u) ? 1u << 12 : 0;
    m |= (up && d) ? 1u << 13 : 0;
    return m;
}

// Residual of slot q of the node at shared index pi (arc known to exist).
__device__ __forceinline__ int32_t smem_residual(const TileSmem &m, const TileGeom &t,
                                                 const Geom &g, int pi, int q) {
    switch (q) {
        case 0: return m.rc[pi];
        case 1: return kInfR;
        case 2: return m.rr[pi];
        case 3: return g.lam2 - m.rr[pi - 1];
        case 4: return m.rd[pi];
        case 5: return g.lam2 - m.rd[pi - t.SYs];
        case 6: return m.ri0[pi];
        case 7: return m.ri1[pi];
        case 8: return m.ri2[pi];
        case 9: return m.ri3[pi];
        case 10: return g.h2h - m.ri1[pi - 1 + t.SJ];
        case 11: return g.h2h - m.ri0[pi + 1 + t.SJ];
        case 12: return g.h2v - m.ri3[pi - t.SYs + t.SJ];
        default: return g.h2v - m.ri2[pi + t.SYs + t.SJ];
    }
}

// Fire-and-forget adds (PTX red): no result comes back, so a push does not
// wait for the memory system before the next one.
__device__ __forceinline__ void red_add_smem(int32_t *p, int32_t v) {
    asm volatile("red.shared.add.s32 [%0], %1;" ::"r"((unsigned)__cvta_generic_to_shared(p)),
                 "r"(v));
}
__device__ __forceinline__ void red_add_gmem(int32_t *p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v));
}

// Apply a push of d along slot q to the residual words in shared memory; when
// the word belongs to a halo node (slots whose residual is stored at the arc's
// head), the global copy is updated at once as well.  Only the data-arc
// residual can grow without a bound of its own (flow pushed back along the
// infinite reverse arc); it is checked for overflow when the tile is written
// back.  Every other word is a residual of an arc pair and stays within the
// pair's capacity.
__device__ __forceinline__ void smem_push_residual(const TileSmem &m, const TileGeom &t,
                                                   const State &s, int pi, int64_t gi,
                                                   const Geom &g, int q, int32_t d,
                                                   bool head_is_halo) {
    switch (q) {
        case 0: red_add_smem(&m.rc[pi], -d); return;
        case 1: red_add_smem(&m.rc[pi - t.SJ], d); return;   // chain never leaves the tile
        case 2: red_add_smem(&m.rr[pi], -d); return;
        case 3:
            if (head_is_halo) red_add_gmem(&s.rr[gi - 1], d);
            red_add_smem(&m.rr[pi - 1], d);
            return;
        case 4: red_add_smem(&m.rd[pi], -d); return;
        case 5:
            if (head_is_halo) red_add_gmem(&s.rd[gi - g.SY], d);
            red_add_smem(&m.rd[pi - t.SYs], d);
            return;
        case 6: red_add_smem(&m.ri0[pi], -d); return;
        case 7: red_add_smem(&m.ri1[pi], -d); return;
        case 8: red_add_smem(&m.ri2[pi], -d); return;
        case 9: red_add_smem(&m.ri3[pi], -d); return;
        case 10:
            if (head_is_halo) red_add_gmem(&s.ri1[gi - 1 + g.P], d);
            red_add_smem(&m.ri1[pi - 1 + t.SJ], d);
            return;
        case 11:
            if (head_is_halo) red_add_gmem(&s.ri0[gi + 1 + g.P], d);
            red_add_smem(&m.ri0[pi + 1 + t.SJ], d);
            return;
        case 12:
            if (head_is_halo) red_add_gmem(&s.ri3[gi - g.SY + g.P], d);
            red_add_smem(&m.ri3[pi - t.SYs + t.SJ], d);
            return;
        default:
            if (head_is_halo) red_add_gmem(&s.ri2[gi + g.SY + g.P], d);
            red_add_smem(&m.ri2[pi + t.SYs + t.SJ], d);
            return;
    }
}

struct TileOrigin {
    int tx, ty, W0, y0;
};

__device__ __forceinline__ TileOrigin tile_origin(const TileGeom &t, int tile) {
    TileOrigin o;
    o.tx = tile % t.tiles_w;
    o.ty = tile / t.tiles_w;
    o.W0 = o.tx * t.TW;
    o.y0 = o.ty * t.TH;
    return o;
}

// Staging with every global load issued before any shared-memory store: a
// thread's first two halo cells go through registers (HaloRegs), so the halo
// and the own nodes of a tile arrive in one round trip to L2 instead of one
// per loop.  Cells past the first 2 x blockDim (large depth ranges) are
// loaded afterwards by halo_rest.
struct HaloRegs {
    int32_t h[2], r1[2], r2[2];
    int pi[2], kind[2];
    bool ok[2];
};

// Halo cell n of the combined index space: the left and right columns
// (2 TH K cells), then the top and bottom rows (2 K TW cells).  kind 0..3 =
// left, right, top, bottom.
__device__ __forceinline__ void halo_cell(const Geom &g, const TileGeom &t, const TileOrigin &o,
                                          int n, int &pi, int64_t &gi, bool &in, int &kind) {
    const int ncol = 2 * t.TH * g.K;
    int yl, j, wl;
    if (n < ncol) {
        const int side = n / (t.TH * g.K), r = n - side * t.TH * g.K;
        yl = r / g.K;
        j = r - yl * g.K;
        wl = side ? t.TW : -1;
        kind = side;
    } else {
        n -= ncol;
        const int side = n / (g.K * t.TW), r = n - side * g.K * t.TW;
        j = r / t.TW;
        wl = r - j * t.TW;
        yl = side ? t.TH : -1;
        kind = 2 + side;
    }
    const int W = o.W0 + wl, y = o.y0 + yl;
    pi = pidx(t, yl, j, wl);
    in = W >= 0 && W < g.ng && y >= 0 && y < g.h;
    gi = ((int64_t)y * g.K + j) * g.P + W;
}

// Loads of a halo cell: the height, and the residual words stored at the head
// of an arc of the tile's own nodes (rr, ri1 left; ri0 right; rd, ri3 top; ri2
// bottom).  Positions outside the grid get height kInfH and zero residuals.
__device__ __forceinline__ void halo_load(const SolveArgs &a, const int32_t *hsrc, bool with_res,
                                          int64_t gi, bool in, int kind, int32_t &h, int32_t &r1,
                                          int32_t &r2) {
    const State &s = a.s;
    h = (in && hsrc) ? ld(&hsrc[gi]) : kInfH;   // hsrc NULL: heights unknown (infinite)
    r1 = r2 = 0;
    if (with_res && in) {
        if (kind == 0) {
            r1 = ld(&s.rr[gi]);
            r2 = ld(&s.ri1[gi]);
        } else if (kind == 1) {
            r1 = ld(&s.ri0[gi]);
        } else if (kind == 2) {
            r1 = ld(&s.rd[gi]);
            r2 = ld(&s.ri3[gi]);
        } else {
            r1 = ld(&s.ri2[gi]);
        }
    }
}

__device__ __forceinline__ void halo_store(const TileSmem &m, bool with_res, int pi, int kind,
                                           int32_t h, int32_t r1, int32_t r2) {
    m.ht[pi] = h;
    if (!with_res) return;
    if (kind == 0) {
        m.rr[pi] = r1;
        m.ri1[pi] = r2;
    } else if (kind == 1) {
        m.ri0[pi] = r1;
    } else if (kind == 2) {
        m.rd[pi] = r1;
        m.ri3[pi] = r2;
    } else {
        m.ri2[pi] = r1;
    }
}

__device__ __forceinline__ int halo_cells(const Geom &g, const TileGeom &t) {
    return 2 * t.TH * g.K + 2 * g.K * t.TW;
}

__device__ __forceinline__ void halo_issue(const SolveArgs &a, const TileOrigin &o, bool with_res,
                                           const int32_t *hsrc, HaloRegs &hr) {
    const int total = halo_cells(a.g, a.t);
#pragma unroll
    for (int u = 0; u < 2; u++) {
        const int n = threadIdx.x + u * blockDim.x;
        hr.ok[u] = n < total;
        hr.pi[u] = 0;
        hr.kind[u] = 0;
        hr.h[u] = kInfH;
        hr.r1[u] = hr.r2[u] = 0;
        if (!hr.ok[u]) continue;
        int64_t gi;
        bool in;
        halo_cell(a.g, a.t, o, n, hr.pi[u], gi, in, hr.kind[u]);
        halo_load(a, hsrc, with_res, gi, in, hr.kind[u], hr.h[u], hr.r1[u], hr.r2[u]);
    }
}

__device__ __forceinline__ void halo_commit(const TileSmem &m, bool with_res, const HaloRegs &hr) {
#pragma unroll
    for (int u = 0; u < 2; u++)
        if (hr.ok[u]) halo_store(m, with_res, hr.pi[u], hr.kind[u], hr.h[u], hr.r1[u], hr.r2[u]);
}

__device__ void halo_rest(const SolveArgs &a, const TileSmem &m, const TileOrigin &o,
                          bool with_res, const int32_t *hsrc) {
    const int total = halo_cells(a.g, a.t);
    for (int n = threadIdx.x + 2 * blockDim.x; n < total; n += blockDim.x) {
        int pi, kind;
        int64_t gi;
        bool in;
        halo_cell(a.g, a.t, o, n, pi, gi, in, kind);
        int32_t h, r1, r2;
        halo_load(a, hsrc, with_res, gi, in, kind, h, r1, r2);
        halo_store(m, with_res, pi, kind, h, r1, r2);
    }
}

// Per-block tables of the tile shape of the pair a block is working on,
// rebuilt only when the block moves to another pair (k_batch): for every own
// position n of a tile its shared index and coordinates, packed as
//   p (bits 0-12) | wl (13-17) | yl (18-20) | j (21-31)
// (shared index < 8192: a tile's 9 fields fit the 180 KB budget; wl < 32,
// yl < 8, j < 2048), and the per-slot push table of the sweep visits.  Visits
// then need no division to place a node.
__shared__ uint32_t s_info[kMaxTileNodes];

__device__ __forceinline__ uint32_t pack_info(int p, int wl, int yl, int j) {
    return (uint32_t)p | ((uint32_t)wl << 13) | ((uint32_t)yl << 18) | ((uint32_t)j << 21);
}
__device__ __forceinline__ int info_p(uint32_t v) { return (int)(v & 0x1fffu); }
__device__ __forceinline__ int info_wl(uint32_t v) { return (int)((v >> 13) & 31u); }
__device__ __forceinline__ int info_yl(uint32_t v) { return (int)((v >> 18) & 7u); }
__device__ __forceinline__ int info_j(uint32_t v) { return (int)(v >> 21); }

// Search direction of a relabel pass (see SolveArgs::dir).
__device__ __forceinline__ int eff_dir(const SolveArgs &a) {
    if (a.dir != 2) return a.dir;
    return ld(&a.s.hdr->rev) ? 0 : 1;
}

// ---------------------------------------------------------- relabel pass ---

// Local relaxation to the tile's fixed point.  Own nodes' residual-arc masks
// are in registers (mk), own heights and halo heights in shared memory.

template <int NPT>
__device__ bool relax_tile(const SolveArgs &a, const TileSmem &m, const int (&pi)[NPT],
                           const unsigned (&mk)[NPT], int first_inner = 4,
                           int max_outer = 1 << 30, const unsigned *done_ctr = nullptr,
                           unsigned items = 0, bool *cut = nullptr) {
    const TileGeom &t = a.t;
    int off[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; q++) off[q] = soff(t, q);
    // Asynchronous (chaotic) relaxation: each thread sweeps its nodes
    // kInner times between CTA barriers, reading neighbours' heights as other
    // warps update them.  Values only decrease and stay upper bounds, so any
    // interleaving converges to the same fixed point; an outer round in which
    // no height changed anywhere proves it has been reached.
    // Neighbour heights are read with plain loads, all 14 at once (a missing
    // arc reads the node's own height and is masked out), so they overlap:
    // a height read stale inside a round only delays convergence, and the
    // round that ends the loop changed nothing after fresh reads.
    constexpr int kInner = 2;
    int32_t *ht = m.ht;
    bool any_change = false;
    // Straggler cut (with done_ctr): after a round that changed heights, stop
    // when all but 1 + min(items / 8, half the grid) of the step's items are
    // done (the last items of a step much larger than the grid are not
    // stragglers: they started late).  The caller queues the tile again, and
    // the heights so far are upper bounds of the fixed point, so a later pass
    // resumes from them.  Thread 0 reads the done count at the start of a
    // round and publishes its decision before the round's barrier, in a slot
    // the next round does not overwrite.
    __shared__ int s_rstop[2];
    const unsigned margin = 1 + min(items / 8, gridDim.x / 2);
    for (int outer = 0;; outer++) {
        int changed = 0;
        unsigned seen = 0;
        if (done_ctr && threadIdx.x == 0) seen = *(volatile const unsigned *)done_ctr;
        // a first round of fewer sweeps settles tiles whose halo change does
        // not reach them without paying for a full round
        const int n_inner = outer == 0 ? first_inner : kInner;
        for (int inner = 0; inner < n_inner; inner++) {
#pragma unroll
            for (int k = 0; k < NPT; k++) {
                if (pi[k] < 0) continue;
                const int p = pi[k];
                const int32_t h = ht[p];
                if (h == 0) continue;
                const unsigned bits = mk[k];
                int32_t hv[kSlots];
#pragma unroll
                for (int q = 0; q < kSlots; q++) hv[q] = ht[p + (((bits >> q) & 1u) ? off[q] : 0)];
                int32_t hmin = kInfH;
#pragma unroll
                for (int q = 0; q < kSlots; q++)
                    if ((bits >> q) & 1u) hmin = min(hmin, hv[q]);
                if (hmin < kInfH && hmin + 1 < h) {
                    ht[p] = hmin + 1;
                    changed = 1;
                }
            }
        }
        if (done_ctr && threadIdx.x == 0) s_rstop[outer & 1] = seen + margin >= items;
        if (!__syncthreads_or(changed)) break;
        any_change = true;
        if (outer + 1 >= max_outer) break;
        if (done_ctr && s_rstop[outer & 1]) {
            *cut = true;
            break;
        }
    }
    return any_change;
}

// First relabel pass of a tile: residual-arc masks from the current state,
// heights reset (0 on nodes with sink capacity left, else infinity), local
// relaxation with an unknown (infinite) halo.  Returns the tile's active
// count (positive excess and a finite height).
template <int NPT>
__device__ long long relabel_init_tile(const SolveArgs &a, const TileSmem &m, int tile) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const State &s = a.s;
    const TileOrigin o = tile_origin(t, tile);
    const int dir = eff_dir(a);
    // halo heights are not known yet in this pass: staged as infinite
    HaloRegs hr;
    halo_issue(a, o, true, nullptr, hr);
    int pi[NPT], pq[NPT];
    unsigned mk[NPT];
    int64_t gi[NPT];
    int32_t v_rc[NPT], v_rr[NPT], v_rd[NPT], v_r0[NPT], v_r1[NPT], v_r2[NPT], v_r3[NPT], v_ex[NPT];
    // own nodes: every load first ...
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        pi[k] = pq[k] = -1;
        mk[k] = 0;
        gi[k] = 0;
        v_rc[k] = v_rr[k] = v_rd[k] = v_r0[k] = v_r1[k] = v_r2[k] = v_r3[k] = v_ex[k] = 0;
        if (n >= t.TN) continue;
        const uint32_t info = s_info[n];
        const int wl = info_wl(info), yl = info_yl(info), j = info_j(info);
        const int W = o.W0 + wl, y = o.y0 + yl;
        pq[k] = info_p(info);
        if (W >= g.ng || y >= g.h) continue;
        const int64_t i = ((int64_t)y * g.K + j) * g.P + W;
        pi[k] = pq[k];
        gi[k] = i;
        v_rc[k] = ld(&s.rc[i]);
        v_rr[k] = ld(&s.rr[i]);
        v_rd[k] = ld(&s.rd[i]);
        v_r0[k] = ld(&s.ri0[i]);
        v_r1[k] = ld(&s.ri1[i]);
        v_r2[k] = ld(&s.ri2[i]);
        v_r3[k] = ld(&s.ri3[i]);
        v_ex[k] = ld(&s.ex[i]);
    }
    // ... then the shared-memory stores
    halo_commit(m, true, hr);
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pq[k] < 0) continue;
        const int p = pq[k];
        if (pi[k] < 0) {
            m.ht[p] = kInfH;
            continue;
        }
        m.rc[p] = v_rc[k];
        m.rr[p] = v_rr[k];
        m.rd[p] = v_rd[k];
        m.ri0[p] = v_r0[k];
        m.ri1[p] = v_r1[k];
        m.ri2[p] = v_r2[k];
        m.ri3[p] = v_r3[k];
        const int32_t e = v_ex[k];
        if (dir == 0) {
            m.ht[p] = e < 0 ? 0 : kInfH;
            mk[k] = e > 0 ? 0x8000u : 0u;
        } else {
            m.ht[p] = e > 0 ? 0 : kInfH;
        }
    }
    halo_rest(a, m, o, true, nullptr);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const uint32_t info = s_info[threadIdx.x + k * blockDim.x];
        const unsigned ex = arc_exists(g, o.y0 + info_yl(info), info_j(info), o.W0 + info_wl(info));
#pragma unroll
        for (int q = 0; q < kSlots; q++) {
            if (!((ex >> q) & 1u)) continue;
            bool res;
            if (dir == 0) {
                res = smem_residual(m, t, g, pi[k], q) > 0;          // arc u -> head
            } else if (q == 0) {
                res = true;                                           // head j+1 -> u: infinite
            } else if (q == 1) {
                res = m.rc[pi[k] - t.SJ] > 0;                         // head j-1 -> u: data arc
            } else {
                const int32_t cap = q < 6 ? g.lam2 : (q == 8 || q == 9 || q == 12 || q == 13) ? g.h2v
                                                                                             : g.h2h;
                res = cap - smem_residual(m, t, g, pi[k], q) > 0;     // head -> u: pair reverse
            }
            if (res) mk[k] |= 1u << q;
        }
        __stcg(&a.amask[gi[k]], (uint16_t)mk[k]);
    }
    __syncthreads();
    // the first pass's relaxation is capped: the pass after it visits every
    // tile again, with the halo known, and relaxes each to its fixed point
    relax_tile<NPT>(a, m, pi, mk, 4, kInitOuter);
    int act = 0;
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const int32_t h = m.ht[pi[k]];
        __stcg(&a.hgt[gi[k]], h);
        act += (mk[k] & 0x8000u) && h < kInfH;
    }
    const long long tot = block_sum(act);
    if (threadIdx.x == 0) __stcg(&a.tile_cnt[tile], (int32_t)tot);
    return tot;
}

// Queue a tile for the next step, once: the caller that turns its flag from 0
// to 1 appends it to the list, and the tile's visit in that step clears the
// flag again.
__device__ __forceinline__ void enqueue(int32_t *flag, int32_t *list, int32_t *count, int tile) {
    if (atomicExch(&flag[tile], 1) == 0) __stcg(&list[atomicAdd(count, 1)], tile);
}

// Neighbour tile on side q (0: W-1, 1: W+1, 2: y-1, 3: y+1), or -1.
__device__ __forceinline__ int side_tile(const TileGeom &t, const TileOrigin &o, int tile, int q) {
    if (q == 0) return o.tx > 0 ? tile - 1 : -1;
    if (q == 1) return o.tx + 1 < t.tiles_w ? tile + 1 : -1;
    if (q == 2) return o.ty > 0 ? tile - t.tiles_w : -1;
    return o.ty + 1 < t.tiles_h ? tile + t.tiles_w : -1;
}

// Later relabel passes: masks from the first pass, heights from global
// memory (own and halo); relax, write back what changed, mark the neighbour
// tiles whose halo changed, and return the change of the tile's active count.
template <int NPT>
__device__ long long relabel_pass_tile(const SolveArgs &a, const TileSmem &m, int tile,
                                       int &changed, int32_t *dirty_next, int32_t *list_next,
                                       int32_t *count_next, const unsigned *done_ctr,
                                       unsigned items) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const TileOrigin o = tile_origin(t, tile);
    const long long before = ld(&a.tile_cnt[tile]);   // issued now, used at the end
    HaloRegs hr;
    halo_issue(a, o, false, a.hgt, hr);
    int pi[NPT], pq[NPT];
    unsigned mk[NPT];
    int64_t gi[NPT];
    int32_t h0[NPT];
    // own nodes: every load first, then the shared-memory stores
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        pi[k] = pq[k] = -1;
        mk[k] = 0;
        gi[k] = 0;
        h0[k] = kInfH;
        if (n >= t.TN) continue;
        const uint32_t info = s_info[n];
        const int wl = info_wl(info), yl = info_yl(info), j = info_j(info);
        const int W = o.W0 + wl, y = o.y0 + yl;
        pq[k] = info_p(info);
        if (W >= g.ng || y >= g.h) continue;
        const int64_t i = ((int64_t)y * g.K + j) * g.P + W;
        pi[k] = pq[k];
        gi[k] = i;
        mk[k] = ld(&a.amask[i]);
        h0[k] = ld(&a.hgt[i]);
    }
    halo_commit(m, false, hr);
#pragma unroll
    for (int k = 0; k < NPT; k++)
        if (pq[k] >= 0) m.ht[pq[k]] = h0[k];
    halo_rest(a, m, o, false, a.hgt);
    __shared__ int s_sides;
    if (threadIdx.x == 0) s_sides = 0;
    __syncthreads();
    // one sweep first: most tiles a halo change marks need no more
    bool cut = false;
    const bool ch = relax_tile<NPT>(a, m, pi, mk, 1, 1 << 30, done_ctr, items, &cut);
    int act = 0;
    unsigned sides = 0;
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const int32_t h = m.ht[pi[k]];
        if (h != h0[k]) {
            __stcg(&a.hgt[gi[k]], h);
            const uint32_t info = s_info[threadIdx.x + k * blockDim.x];
            const int wl = info_wl(info), yl = info_yl(info);
            sides |= (wl == 0 ? 1u : 0u) | (wl == t.TW - 1 ? 2u : 0u) | (yl == 0 ? 4u : 0u) |
                     (yl == t.TH - 1 ? 8u : 0u);
        }
        act += (mk[k] & 0x8000u) && h < kInfH;
    }
    if (sides) atomicOr(&s_sides, (int)sides);
    const long long tot = block_sum(act);   // also orders s_sides
    if (threadIdx.x < 4 && ((unsigned)s_sides >> threadIdx.x & 1u)) {
        const int nb = side_tile(t, o, tile, threadIdx.x);
        if (nb >= 0) enqueue(dirty_next, list_next, count_next, nb);
    }
    // a relaxation cut short goes on in the next pass
    if (cut && threadIdx.x == 4) enqueue(dirty_next, list_next, count_next, tile);
    if (ch) changed = 1;
    __syncthreads();
    if (threadIdx.x == 0) __stcg(&a.tile_cnt[tile], (int32_t)tot);
    return tot - before;
}

// ------------------------------------------------------------ sweep visit ---

// Per-slot push table of a tile shape, in shared memory: where a push along
// slot q changes the residual word (shared offset from the node, its kind and
// the pair capacity), where the head's excess lives (shared offset, global
// offset), and where the word lives in global memory when the head is a halo
// node.  A discharge then loops over a node's admissible slots only -- one or
// two on average -- instead of running the code of all 14.
//   .x  sword  shared offset of the residual word from the node (field * PN + off)
//   .y  sex    shared offset of the head's excess
//   .z  kind   0: word stored at the node (r = word, a push subtracts)
//              1: word stored at the head (r = cap - word, a push adds)
//              2: the infinite reverse data arc (a push adds to the head's rc)
//   .w  cap    pair capacity of kind 1
//   [1] .x dw, .y dy (head position in the tile), .z gfield (global array of
//       the word: 0 rc .. 6 ri3), .w grel (global offset of the word)
//   [2] .x gex (global offset of the head)
struct SlotTab {
    int4 a, b, c;
};

__device__ __forceinline__ SlotTab make_slot(const Geom &g, const TileGeom &t, int q) {
    int dy, dj, dw;
    slot_delta(q, dy, dj, dw);
    const int off = dy * t.SYs + dj * t.SJ + dw;
    // tile field order in shared memory: ht 0, ex 1, rc 2, rr 3, rd 4, ri0..ri3 5..8;
    // in global memory: rc 0, rr 1, rd 2, ri0..ri3 3..6, ex 7, ht 8
    int sfield, roff = 0, kind = 0, cap = 0, gfield = -1, grel = 0;
    switch (q) {
        case 0: sfield = 2; break;
        case 1: sfield = 2; roff = -t.SJ; kind = 2; break;
        case 2: sfield = 3; break;
        case 3: sfield = 3; roff = -1; kind = 1; cap = g.lam2; gfield = 1; grel = -1; break;
        case 4: sfield = 4; break;
        case 5: sfield = 4; roff = -t.SYs; kind = 1; cap = g.lam2; gfield = 2; grel = -(int)g.SY; break;
        case 6: sfield = 5; break;
        case 7: sfield = 6; break;
        case 8: sfield = 7; break;
        case 9: sfield = 8; break;
        case 10: sfield = 6; roff = -1 + t.SJ; kind = 1; cap = g.h2h; gfield = 4; grel = -1 + g.P; break;
        case 11: sfield = 5; roff = 1 + t.SJ; kind = 1; cap = g.h2h; gfield = 3; grel = 1 + g.P; break;
        case 12:
            sfield = 8; roff = -t.SYs + t.SJ; kind = 1; cap = g.h2v; gfield = 6;
            grel = -(int)g.SY + g.P;
            break;
        default:
            sfield = 7; roff = t.SYs + t.SJ; kind = 1; cap = g.h2v; gfield = 5;
            grel = (int)g.SY + g.P;
            break;
    }
    SlotTab e;
    e.a = make_int4(sfield * t.PN + roff, t.PN + off, kind, cap);
    e.b = make_int4(dw, dy, gfield, grel);
    e.c = make_int4((int)(dy * g.SY + (int64_t)dj * g.P + dw), 0, 0, 0);
    return e;
}

__shared__ SlotTab s_slot[kSlots];

// Fill the block's tables (s_info, s_slot) for the tile shape of pair a.
__device__ void build_tables(const SolveArgs &a) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    for (int n = threadIdx.x; n < t.TN; n += blockDim.x) {
        int wl, yl, j;
        if (t.R) {
            // lanes: TW sites x R rows of one layer; the warp group g = n / 32
            // is placed at group (g * spread) mod M, M = TN / 32, numbered
            // layer first, then row group
            wl = n % t.TW;
            const int u = (n / t.TW) % t.R;
            const int M = t.TN / 32;
            const int gp = (int)(((long long)(n / 32) * t.spread) % M);
            j = gp % g.K;
            yl = (gp / g.K) * t.R + u;
        } else {
            wl = n % t.TW;
            const int r = n / t.TW;
            j = r % g.K;
            yl = r / g.K;
        }
        s_info[n] = pack_info(pidx(t, yl, j, wl), wl, yl, j);
    }
    if (threadIdx.x < kSlots) s_slot[threadIdx.x] = make_slot(g, t, threadIdx.x);
}



// Up to local_iters push/relabel iterations of one tile in shared memory.
template <int NPT, int BT>
__device__ void sweep_tile(const SolveArgs &a, const TileSmem &m, int tile, int round, int iters,
                           int &overflow, int32_t *list_next, int32_t *count_next,
                           const unsigned *done_ctr, unsigned items,
                           uint32_t (*s_wlist)[8 * 32]) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const State &s = a.s;
    const TileOrigin o = tile_origin(t, tile);
    int32_t *act_next = a.tile_act + ((round + 1) & 1) * t.T;
    const int64_t tile_g0 = (int64_t)o.y0 * g.SY + o.W0;
    __shared__ unsigned s_touch;
    __shared__ int s_stop;
    if (threadIdx.x == 0) {
        s_touch = 0;   // read only after the staging barrier below
        s_stop = 0;
    }
    HaloRegs hr;
    halo_issue(a, o, true, s.ht, hr);
    // own node k of this thread: its packed position (s_info) and whether it
    // lies inside the grid (bit k of vmask); positions past the tile's nodes
    // are not in vmask either
    uint32_t inf[NPT];
    unsigned vmask = 0, tmask = 0;
    int32_t o_ex[NPT], o_rc[NPT], o_rr[NPT], o_rd[NPT], o_r0[NPT], o_r1[NPT], o_r2[NPT],
        o_r3[NPT], o_ht[NPT];
    // own nodes: every load first (the originals stay in registers for the
    // write-back as deltas) ...
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        inf[k] = 0;
        o_ex[k] = o_rc[k] = o_rr[k] = o_rd[k] = o_r0[k] = o_r1[k] = o_r2[k] = o_r3[k] = 0;
        o_ht[k] = kInfH;
        if (n >= t.TN) continue;
        const uint32_t info = s_info[n];
        inf[k] = info;
        tmask |= 1u << k;
        const int W = o.W0 + info_wl(info), y = o.y0 + info_yl(info);
        if (W >= g.ng || y >= g.h) continue;
        vmask |= 1u << k;
        const int64_t i = tile_g0 + (int64_t)info_yl(info) * g.SY +
                          (int64_t)info_j(info) * g.P + info_wl(info);
        o_ex[k] = ld(&s.ex[i]);
        o_ht[k] = ld(&s.ht[i]);
        o_rc[k] = ld(&s.rc[i]);
        o_rr[k] = ld(&s.rr[i]);
        o_rd[k] = ld(&s.rd[i]);
        o_r0[k] = ld(&s.ri0[i]);
        o_r1[k] = ld(&s.ri1[i]);
        o_r2[k] = ld(&s.ri2[i]);
        o_r3[k] = ld(&s.ri3[i]);
    }
    // ... then the shared-memory stores
    halo_commit(m, true, hr);
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (!((tmask >> k) & 1u)) continue;
        const int p = info_p(inf[k]);
        m.ex[p] = o_ex[k];
        m.ht[p] = o_ht[k];
        if (!((vmask >> k) & 1u)) continue;
        m.rc[p] = o_rc[k];
        m.rr[p] = o_rr[k];
        m.rd[p] = o_rd[k];
        m.ri0[p] = o_r0[k];
        m.ri1[p] = o_r1[k];
        m.ri2[p] = o_r2[k];
        m.ri3[p] = o_r3[k];
    }
    halo_rest(a, m, o, true, s.ht);
    __syncthreads();
    int off[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; q++) off[q] = soff(t, q);
    int32_t *const sbase = m.ht;                 // field f of the tile at sbase + f * PN
    const int64_t gstride = s.rr - s.rc;         // global fields are equally spaced
    // Local iterations, one warp at a time and with no block barrier: each
    // warp compacts its own active nodes (positive excess, finite height; the
    // nodes its lanes own) into a warp list of packed positions with ballots,
    // discharges the list 32 nodes at a time, and goes on to its next
    // iteration.  Discharges of different warps run concurrently on shared
    // memory; the lock-free argument that holds between tiles holds between
    // warps (only a node's own warp lowers its excess, and residuals are
    // consumed only by an arc's tail).  Every load of a discharge depends only
    // on the list entry, so they are in flight together.
    unsigned nb_touch = 0;   // bit 0: left, 1: right, 2: up, 3: down neighbour tile received flow
    const int lane = threadIdx.x & 31;
    uint32_t *wl_list = s_wlist[threadIdx.x >> 5];
    volatile int32_t *vex = m.ex;
    volatile int32_t *vht = m.ht;
    // Straggler cut: a step ends when its last item does, so a visit still
    // running when nearly all of its step's items are done (all but 1 +
    // min(items / 8, half the grid)) stops after half its local iterations.
    // Its tile keeps its work and is queued for the next round.  Thread 0
    // reads the step's done count once per iteration and uses it one
    // iteration later (the load's latency hides behind the iteration).  No
    // cut without done_ctr (fixed-sweep mode: a round is a full round).
    unsigned seen = 0;
    const unsigned margin = 1 + min(items / 8, gridDim.x / 2);
    for (int it = 0; it < iters; it++) {
        if (done_ctr && threadIdx.x == 0) {
            if (it >= 2 && seen + margin >= items) s_stop = 1;
            seen = *(volatile const unsigned *)done_ctr;
        }
        if (it >= iters / 2 && __shfl_sync(0xffffffffu, *(volatile int *)&s_stop, 0)) break;
        int32_t ce[NPT], ch[NPT];
#pragma unroll
        for (int k = 0; k < NPT; k++) {
            const int p = info_p(inf[k]);
            ce[k] = vex[p];
            ch[k] = vht[p];
        }
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < NPT; k++) {
            const bool act = ((vmask >> k) & 1u) && ce[k] > 0 && ch[k] < kInfH;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (act) wl_list[cnt + __popc(bal & ((1u << lane) - 1u))] = inf[k];
            cnt += __popc(bal);
        }
        __syncwarp();
        if (cnt == 0) continue;
        for (int li = lane; li < cnt; li += 32) {
            const uint32_t info = wl_list[li];
            const int p = info_p(info);
            const int wl = info_wl(info), yl = info_yl(info), j = info_j(info);
            const int64_t gin = tile_g0 + (int64_t)yl * g.SY + (int64_t)j * g.P + wl;
            const unsigned exb = arc_exists(g, o.y0 + yl, j, o.W0 + wl);
            // all loads issued before any is used (the existing arcs' heights
            // are read whatever their residual), so they overlap
            const int32_t e = vex[p];
            const int32_t hu = vht[p];
            int32_t rr[kSlots], hv[kSlots];
#pragma unroll
            for (int q = 0; q < kSlots; q++) {
                const bool ex = (exb >> q) & 1u;
                rr[q] = ex ? smem_residual(m, t, g, p, q) : 0;
                hv[q] = vht[p + (ex ? off[q] : 0)];
            }
            if (e <= 0 || hu >= kInfH) continue;
            // residual and admissible slots as bit masks (registers only)
            unsigned resid = 0, adm = 0;
#pragma unroll
            for (int q = 0; q < kSlots; q++) {
                const bool rp = rr[q] > 0;
                resid |= (unsigned)rp << q;
                adm |= (unsigned)(rp && hv[q] < hu) << q;
            }
            int32_t left = e;
            // push along the admissible slots, in slot order, until the
            // excess is gone; a slot's residual is the one loaded above (it
            // can only have grown since: pushing it is always valid)
            for (unsigned bits = adm; bits && left > 0; bits &= bits - 1u) {
                const int q = __ffs(bits) - 1;
                int32_t r = 0;
#pragma unroll
                for (int qq = 0; qq < kSlots; qq++) r = qq == q ? rr[qq] : r;
                const int32_t d = min(left, r);
                const SlotTab st = s_slot[q];
                int32_t *wp = sbase + p + st.a.x;
                red_add_smem(wp, st.a.z == 0 ? -d : d);
                const int wl2 = wl + st.b.x, yl2 = yl + st.b.y;
                if (wl2 < 0 || wl2 >= t.TW || yl2 < 0 || yl2 >= t.TH) {
                    // the head is a halo node: its excess, and a word stored
                    // at it, change in global memory at once
                    if (st.a.z == 1) red_add_gmem(s.rc + st.b.z * gstride + gin + st.b.w, d);
                    red_add_gmem(s.ex + gin + st.c.x, d);
                    nb_touch |= wl2 < 0 ? 1u : wl2 >= t.TW ? 2u : yl2 < 0 ? 4u : 8u;
                } else {
                    red_add_smem(sbase + p + st.a.y, d);
                }
                left -= d;
            }
            if (left != e) red_add_smem(&m.ex[p], left - e);
            if (left > 0) {
                // every admissible slot is saturated: relabel over the others
                const unsigned rest = resid & ~adm;
                int32_t hmin = kInfH;
#pragma unroll
                for (int q = 0; q < kSlots; q++)
                    if ((rest >> q) & 1u) hmin = min(hmin, hv[q]);
                vht[p] = hmin >= kInfH - 1 ? kInfH : hmin + 1;
            }
        }
        __syncwarp();
    }
    __syncthreads();
    // write back own nodes as deltas (other tiles may have updated the same
    // words through global atomics meanwhile); note whether work is left
    int still = 0;
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (!((vmask >> k) & 1u)) continue;
        const uint32_t info = inf[k];
        const int p = info_p(info);
        const int64_t i = tile_g0 + (int64_t)info_yl(info) * g.SY +
                          (int64_t)info_j(info) * g.P + info_wl(info);
        int32_t v;
        if ((v = m.ex[p] - o_ex[k])) atomicAdd(&s.ex[i], v);
        // the data-arc residual is the one word that can grow without a bound
        // of its own (flow pushed back down the infinite reverse arc); only
        // this tile changes it (the chain stays inside the tile)
        overflow |= m.rc[p] > kCapLimit || m.rc[p] < 0;
        if ((v = m.rc[p] - o_rc[k])) atomicAdd(&s.rc[i], v);
        if ((v = m.rr[p] - o_rr[k])) atomicAdd(&s.rr[i], v);
        if ((v = m.rd[p] - o_rd[k])) atomicAdd(&s.rd[i], v);
        if ((v = m.ri0[p] - o_r0[k])) atomicAdd(&s.ri0[i], v);
        if ((v = m.ri1[p] - o_r1[k])) atomicAdd(&s.ri1[i], v);
        if ((v = m.ri2[p] - o_r2[k])) atomicAdd(&s.ri2[i], v);
        if ((v = m.ri3[p] - o_r3[k])) atomicAdd(&s.ri3[i], v);
        if (m.ht[p] != o_ht[k]) __stcg(&s.ht[i], m.ht[p]);
        still |= m.ex[p] > 0 && m.ht[p] < kInfH;
    }
    // one barrier for the tile's flags: bits 0-3 neighbour tiles that received
    // flow, bit 4 work left in this tile
    const unsigned wbits = __reduce_or_sync(0xffffffffu, nb_touch | (still ? 16u : 0u));
    if ((threadIdx.x & 31) == 0 && wbits) atomicOr(&s_touch, wbits);
    __syncthreads();
    const unsigned touch = s_touch;
    const bool still_any = (touch & 16u) != 0;
    if (threadIdx.x < 4 && (touch >> threadIdx.x & 1u)) {
        const int nb = side_tile(t, o, tile, threadIdx.x);
        if (nb >= 0) enqueue(act_next, list_next, count_next, nb);
    }
    if (threadIdx.x == 4 && still_any) enqueue(act_next, list_next, count_next, tile);
    __syncthreads();
}

// ------------------------------------------------------- the solve loop ---
//
// One cooperative launch solves n independent pairs.  Each pair runs its own
// sequence of steps; in a step each of its tiles with work does the pair's
// current phase:
//
//   INIT   first relabel pass (masks, heights reset, in-tile distances)
//   PASS   later relabel pass (all tiles once, then tiles whose halo changed)
//   SWEEP  one sweep round over the tiles with work
//   LABELS label extraction (extraction launches)
//   DONE   nothing
//
// A step's work items are all T tiles of the pair (INIT, the first PASS, the
// first SWEEP round -- those with active nodes -- and LABELS) or the tiles
// queued for it by the visits of the step before.  Blocks claim items one at
// a time from a per-pair claim word (step | items | next item), taking them
// from any pair that has some; the block that completes a step's last item
// advances that pair's state machine and publishes its next step.  There is
// no grid barrier: a pair in a latency-bound tail steps as fast as its own
// visits allow while other blocks work on other pairs.
// Per pair the schedule is the one of a single solve: a relabel (capped at
// relabel_passes passes unless it decides termination), then sweep rounds --
// sweeps_per_relabel of them, or in the tail (few active nodes) until the
// tiles with work stop decreasing and the sweep rounds have cost as much as the
// relabel did, both counted in tile visits one CTA makes in sequence.

constexpr int kMaxPairs = 64;
enum { PH_INIT = 0, PH_PASS = 1, PH_SWEEP = 2, PH_LABELS = 3, PH_DONE = 4 };

struct PairState {
    int phase, pass, full, conv, tail, status, cap;
    int exact_end;     // ended on a relabel run to its fixed point that found nothing active
    int ht_labels;     // extraction reads the solve's exact heights (no relabel of its own)
    long long round, nrounds, rounds_total, relabels, passes, outer;
    long long active, prev1, prev2, relabel_visits, relabel_depth, last_relabel_depth, sweep_depth;
    long long visits_sweep_total, visits_relabel_total;
    long long ns_sweep, ns_relabel;    // device time of the steps in each phase
    unsigned long long t_step;         // start of the current step (global timer)
};

// Per-pair control words of a launch.  claim packs the current step's queue
// slot (step mod 3), its number of items and the next item (24 bits each):
// one atomic add both claims an item and tells where its step's queue is.
struct PairCtl {
    unsigned long long claim;
    unsigned int done;      // items of the current step completed
    unsigned int step;      // current step
    long long red[3][4];    // per-step sums (slot = step mod 3)
    int32_t qcount[3];      // queued tiles per step slot
    int32_t pad;
    PairState st;           // written only by the block that advances the pair
};

constexpr unsigned kItemMask = 0xffffffu;
// An idle block gives up after this long unless the options set a limit.
constexpr unsigned long long kDefaultIdleLimitNs = 60ull * 1000 * 1000 * 1000;

static_assert(sizeof(PairState) % 8 == 0, "PairState is copied in 8-byte words");

// Copy of a pair's state as other SMs wrote it (L2-coherent loads).
__device__ __forceinline__ void load_state(PairState *dst, const PairState *src) {
    const long long *s = (const long long *)src;
    long long *d = (long long *)dst;
    for (int i = 0; i < (int)(sizeof(PairState) / 8); i++) d[i] = __ldcg(s + i);
}

__device__ __forceinline__ unsigned long long pack_claim(unsigned step, unsigned items,
                                                         unsigned next) {
    // bits 48-63: the step's queue slot (step mod 3), so a block that claims
    // an item knows where the step's queue is from the claim alone
    return ((unsigned long long)(step % 3u) << 48) |
           ((unsigned long long)(items & kItemMask) << 24) | (next & kItemMask);
}

struct BatchArgs {
    int n;            // pairs
    int extract;      // 0: max-flow solve, 1: label extraction
    unsigned long long idle_limit_ns;   // a block idle this long aborts the launch
    Ctrl *bar;        // abort flag and the count of finished pairs (Ctrl::active)
    PairCtl *ctl;     // [n]
    SolveArgs pair[kMaxPairs];
};

static_assert(sizeof(BatchArgs) <= 32000, "the batch arguments travel as kernel parameters");

__device__ void start_relabel(PairState &st, const SolveArgs &a) {
    if (a.mode == GS_MODE_EXACT && st.outer >= a.max_iters) {
        st.phase = PH_DONE;
        st.status = GS_ERR_TIMEOUT;
        return;
    }
    st.outer++;
    st.phase = PH_INIT;
    st.relabel_visits = 0;
    st.relabel_depth = 0;
}

// Critical-path cost of a step that visited `visits` tiles of a pair: the
// number of tile visits one CTA makes in sequence, at least one.
__device__ __forceinline__ long long step_depth(long long visits) {
    return max(1ll, (visits + gridDim.x - 1) / gridDim.x);
}

// Advance one pair at the end of a step; v = the step's sums {a, b, c, overflow}.
__device__ void advance(PairState &st, const SolveArgs &a, const long long v[4], int extract) {
    if (v[3] && st.status == GS_OK) {
        st.status = GS_ERR_OVERFLOW;
        st.phase = PH_DONE;
        return;
    }
    switch (st.phase) {
        case PH_INIT:
            st.active = v[0];
            st.relabel_visits = v[2];
            st.relabel_depth = step_depth(v[2]);
            st.passes++;
            st.pass = 1;
            st.phase = PH_PASS;
            break;
        case PH_PASS: {
            st.active += v[0];
            st.relabel_visits += v[2];
            st.relabel_depth += step_depth(v[2]);
            st.passes++;
            bool end = false;
            st.conv = 0;
            if (v[1] == 0) {
                st.conv = 1;
                end = true;
            } else if (!extract && !st.full && st.pass >= st.cap) {
                end = true;
            } else {
                st.pass++;
            }
            if (!end) break;
            if (extract) {
                st.phase = PH_LABELS;
                break;
            }
            st.relabels++;
            st.last_relabel_depth = st.relabel_depth;
            // a relabel run to its fixed point because the capped one reached no
            // active node, and that found some: later relabels reach as far
            if (st.full && st.active > 0) st.cap = max(st.cap, st.pass);
            st.visits_relabel_total += st.relabel_visits;
            if (st.active == 0) {
                if (st.conv) {
                    st.phase = PH_DONE;
                    st.exact_end = 1;
                } else {
                    st.full = 1;     // nothing active within reach: decide with an exact relabel
                    start_relabel(st, a);
                }
                break;
            }
            st.full = 0;
            st.tail = st.active * 64 <= (long long)a.g.N;
            st.nrounds = st.tail ? 64ll * a.sweeps_per_relabel : a.sweeps_per_relabel;
            if (a.mode == GS_MODE_FIXED_SWEEPS) {
                st.nrounds = min(st.nrounds, a.fixed_sweeps - st.rounds_total);
                if (st.nrounds <= 0) {
                    st.phase = PH_DONE;
                    break;
                }
            }
            st.round = 0;
            st.sweep_depth = 0;
            st.prev1 = st.prev2 = 1ll << 40;
            st.phase = PH_SWEEP;
            break;
        }
        case PH_SWEEP: {
            const long long worked = v[0];
            st.rounds_total++;
            st.round++;
            st.sweep_depth += step_depth(worked);
            st.visits_sweep_total += worked;
            const bool stalled = st.tail && st.round >= 3 && worked * 10 > st.prev2 * 9 &&
                                 st.sweep_depth > st.last_relabel_depth;
            st.prev2 = st.prev1;
            st.prev1 = worked;
            if (worked == 0 || stalled || st.round >= st.nrounds) {
                if (a.mode == GS_MODE_FIXED_SWEEPS && st.rounds_total >= a.fixed_sweeps)
                    st.phase = PH_DONE;
                else
                    start_relabel(st, a);
            }
            break;
        }
        case PH_LABELS:
            st.active = v[0];      // sink capacity left
            if (v[1]) st.status = GS_ERR_LABELS;
            st.phase = PH_DONE;
            break;
        default:
            break;
    }
}

// Labels of one tile's sites and the tile's remaining sink capacity.
__device__ long long labels_tile(const SolveArgs &a, int tile, const int32_t *hsrc, int &bad) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const TileOrigin o = tile_origin(t, tile);
    unsigned long long deficit = 0;
    int b = 0;
    const int dir = eff_dir(a);
    const bool rev = ld(&a.s.hdr->rev) != 0;
    for (int sidx = threadIdx.x; sidx < t.TW * t.TH; sidx += blockDim.x) {
        const int wl = sidx % t.TW, yl = sidx / t.TW;
        const int W = o.W0 + wl, y = o.y0 + yl;
        if (W >= g.ng || y >= g.h) continue;
        int64_t i = (int64_t)y * g.SY + W;
        int lab = 0, prev = 1;
        for (int j = 0; j < g.K; j++, i += g.P) {
            const int32_t h = ld(&hsrc[i]);
            const int in = dir == 1 ? (h < kInfH) : (h >= kInfH);
            b |= in && !prev;
            lab += in;
            prev = in;
            const int32_t e = ld(&a.s.ex[i]);
            if (e < 0) deficit += (unsigned long long)(-(int64_t)e);
        }
        a.labels[(int64_t)y * g.ng + W] = rev ? g.D - 1 - lab : lab;
    }
    bad = __syncthreads_or(b);
    return block_sum((long long)deficit);
}

// Phases whose items are the tiles queued by the step before.
__device__ __forceinline__ bool queued(const PairState &st) {
    return (st.phase == PH_PASS && st.pass > 1) || (st.phase == PH_SWEEP && st.round > 0);
}

// Items of a pair's step from its state and the queue the step before filled.
__device__ __forceinline__ unsigned step_items(const PairState &st, const SolveArgs &a,
                                               const PairCtl *c, unsigned step) {
    if (st.phase == PH_DONE) return 0;
    return queued(st) ? (unsigned)*(volatile const int32_t *)&c->qcount[step % 3] : (unsigned)a.t.T;
}

// Statistics and results of a finished pair.
__device__ void pair_results(const BatchArgs &B, const PairState &st, const SolveArgs &a,
                             int status) {
    if (!B.extract) {
        Ctrl *c = a.ctrl;
        c->stats[0] = st.relabels;
        c->stats[1] = st.rounds_total;
        c->stats[2] = st.passes;
        c->stats[4] = st.active;
        c->stats[5] = st.ns_sweep;
        c->stats[6] = st.ns_relabel;
        c->stats[7] = 1;
        c->visits_sweep = st.visits_sweep_total;
        c->visits_relabel = st.visits_relabel_total;
        c->converged = st.phase == PH_DONE && status == GS_OK;
        // the heights are then the exact distances to the remaining sink
        // capacity: an extraction that needs just those reuses them
        if (st.exact_end && status == GS_OK) a.s.hdr->exact_heights = 1;
    } else {
        a.ctrl->stats[3] = st.passes;
        *a.flow = (int64_t)a.s.hdr->init_deficit - st.active;
    }
    if (status != GS_OK) atomicCAS(a.status, GS_OK, status);
}

// End of a pair's step (one thread, after every item completed): advance the
// state machine -- through any steps that have no items -- and publish the
// next step's claim word, or count the pair finished.
__device__ void end_step(const BatchArgs &B, int p, int slot) {
    PairCtl *c = B.ctl + p;
    const SolveArgs &a = B.pair[p];
    // the step's sums, its number, the pair's state and the queue the step
    // filled for the next one, loaded together (the caller's acquire on the
    // done count orders them after every item's writes)
    long long v0[4];
    for (int k = 0; k < 4; k++) v0[k] = *(volatile long long *)&c->red[slot][k];
    const int32_t q0 = *(volatile int32_t *)&c->qcount[(slot + 1) % 3];
    unsigned step = *(volatile unsigned *)&c->step;
    PairState st;
    load_state(&st, &c->st);
    bool first = true;
    unsigned items = 0;
    const unsigned long long t_now = now_ns();
    if (st.phase == PH_SWEEP) st.ns_sweep += (long long)(t_now - st.t_step);
    else st.ns_relabel += (long long)(t_now - st.t_step);
    st.t_step = t_now;
    for (;;) {
        long long v[4];
        const bool pre = first && step % 3 == (unsigned)slot;   // the prefetched words apply
        if (pre)
            for (int k = 0; k < 4; k++) v[k] = v0[k];
        else
            for (int k = 0; k < 4; k++) v[k] = *(volatile long long *)&c->red[step % 3][k];
        first = false;
        advance(st, a, v, B.extract);
        const unsigned next = step + 1;
        for (int k = 0; k < 4; k++) c->red[next % 3][k] = 0;
        c->qcount[(next + 1) % 3] = 0;
        items = st.phase == PH_DONE ? 0u
                : (pre && queued(st)) ? (unsigned)q0
                                      : step_items(st, a, c, next);
        step = next;
        if (st.phase == PH_DONE || items > 0) break;
    }
    c->st = st;
    c->done = 0;
    c->step = step;
    if (st.phase == PH_DONE) pair_results(B, st, a, st.status);
    atom_exch_release(&c->claim, pack_claim(step, items, 0));
    if (st.phase == PH_DONE) atomicAdd(&B.bar->active, 1);
}

template <int NPT, int BT>
__global__ void __launch_bounds__(BT, BT == 256 ? 2 : 1) k_batch(const __grid_constant__ BatchArgs B) {
    extern __shared__ int32_t smem[];
    __shared__ uint32_t s_wlist[BT / 32][8 * 32];   // the sweep's per-warp active lists
    // pair, item, queue slot of the step, exit flag, items of the step, the
    // queued tile at the item (speculative), the item's tile count (speculative)
    __shared__ int s_claim[7];
    __shared__ PairState s_st;
    int tables_for = -1;           // pair whose tile-shape tables the block holds
    // block 0 starts every pair and publishes its first step
    if (blockIdx.x == 0) {
        for (int p = threadIdx.x; p < B.n; p += blockDim.x) {
            PairCtl *c = B.ctl + p;
            PairState st;
            memset(&st, 0, sizeof(st));
            st.status = GS_OK;
            st.cap = B.pair[p].relabel_passes;
            st.t_step = now_ns();
            const SolveArgs &a = B.pair[p];
            if (!B.extract) {
                a.s.hdr->exact_heights = 0;
                start_relabel(st, a);
            } else if (a.dir == 2 && ld(&a.s.hdr->rev) && ld(&a.s.hdr->exact_heights)) {
                // the label-reversed problem's labels come from distances to the
                // sink capacity, which the finished solve left exact in ht
                st.phase = PH_LABELS;
                st.ht_labels = 1;
            } else {
                start_relabel(st, a);
            }
            c->st = st;
            c->step = 0;
            c->done = 0;
            const unsigned items = step_items(st, B.pair[p], c, 0);
            if (st.phase == PH_DONE) pair_results(B, st, B.pair[p], st.status);
            __threadfence();
            atomicExch(&c->claim, pack_claim(0, items, 0));
            if (st.phase == PH_DONE) atomicAdd(&B.bar->active, 1);
        }
    }
    for (;;) {
        // claim an item of any pair (thread 0); idle polling backs off to 256 ns
        if (threadIdx.x == 0) {
            const unsigned long long t0 = now_ns();
            int got = 0;
            for (int spin = 0; !got; spin++) {
                if (aborted(B.bar) || *(volatile int32_t *)&B.bar->active >= B.n) {
                    s_claim[3] = 1;
                    break;
                }
                for (int k = 0; k < B.n && !got; k++) {
                    const int p = (int)((blockIdx.x + k) % B.n);
                    PairCtl *c = B.ctl + p;
                    const unsigned long long w0 = *(volatile unsigned long long *)&c->claim;
                    if ((w0 & kItemMask) >= ((w0 >> 24) & kItemMask)) continue;
                    const unsigned long long w = atom_add_acquire(&c->claim, 1ull);
                    const unsigned items = (unsigned)((w >> 24) & kItemMask);
                    const unsigned idx = (unsigned)(w & kItemMask);
                    if (idx >= items) continue;
                    // everything the item needs, loaded together: the pair's
                    // state, and both ways the item may name its tile (the
                    // queued tile at this slot, or tile idx with its count)
                    const int sl = (int)((w >> 48) & 3u);
                    const SolveArgs &ap = B.pair[p];
                    const int32_t qt = ld(&ap.tile_list[sl * ap.t.T + idx]);
                    const int32_t tc = ld(&ap.tile_cnt[idx]);
                    load_state(&s_st, &c->st);
                    s_claim[0] = p;
                    s_claim[1] = (int)idx;
                    s_claim[2] = sl;
                    s_claim[3] = 0;
                    s_claim[4] = (int)items;
                    s_claim[5] = qt;
                    s_claim[6] = tc;
                    got = 1;
                }
                if (!got) {
                    if (now_ns() - t0 > B.idle_limit_ns) {
                        atomicExch(&B.bar->abort, 1);
                        s_claim[3] = 1;
                        break;
                    }
                    __nanosleep(32u << min(spin, 3));
                }
            }
        }
        __syncthreads();
        if (s_claim[3]) break;
        const int pr = s_claim[0];
        const int slot = s_claim[2], next = (slot + 1) % 3;
        PairCtl *c = B.ctl + pr;
        const SolveArgs &a = B.pair[pr];
        if (pr != tables_for) {      // uniform: every thread read the same claim
            build_tables(a);
            tables_for = pr;
            __syncthreads();
        }
        const int phase = s_st.phase;
        const int T = a.t.T;
        const TileSmem m = tile_smem(smem, a.t.PN);
        int32_t *list_next = a.tile_list + next * T;
        int32_t *count_next = &c->qcount[next];
        const int tile = queued(s_st) ? s_claim[5]
                         : (phase == PH_SWEEP && s_claim[6] <= 0) ? -1   // nothing to sweep
                                                                   : s_claim[1];
        long long va = 0, vb = 0, vc = 0;
        int ovf = 0;
        if (tile >= 0) {
            if (phase == PH_INIT) {
                // a pair whose tiles need 4 nodes per thread runs the
                // 4-node code also when the launch is sized for 8
                va = (NPT == 8 && a.npt == 4) ? relabel_init_tile<4>(a, m, tile)
                                              : relabel_init_tile<NPT>(a, m, tile);
                vc = 1;
                if (threadIdx.x == 0) {
                    __stcg(&a.tile_dirty[tile], 0);
                    __stcg(&a.tile_dirty[T + tile], 0);
                    __stcg(&a.tile_act[tile], 0);
                    __stcg(&a.tile_act[T + tile], 0);
                }
            } else if (phase == PH_PASS) {
                const int pass = s_st.pass;
                int32_t *dcur = a.tile_dirty + (pass & 1) * T;
                int32_t *dnext = a.tile_dirty + ((pass + 1) & 1) * T;
                if (pass > 1 && threadIdx.x == 0) __stcg(&dcur[tile], 0);
                int ch = 0;
                va = (NPT == 8 && a.npt == 4)
                         ? relabel_pass_tile<4>(a, m, tile, ch, dnext, list_next, count_next,
                                                &c->done, (unsigned)s_claim[4])
                         : relabel_pass_tile<NPT>(a, m, tile, ch, dnext, list_next, count_next,
                                                  &c->done, (unsigned)s_claim[4]);
                vb = ch;
                vc = 1;
            } else if (phase == PH_SWEEP) {
                const int cur = (int)(s_st.round & 1);
                if (threadIdx.x == 0) __stcg(&a.tile_act[cur * T + tile], 0);
                const int iters = s_st.tail ? a.tail_iters : a.local_iters;
                const unsigned *done_ctr = a.mode == GS_MODE_FIXED_SWEEPS ? nullptr : &c->done;
                if (NPT == 8 && a.npt == 4)
                    sweep_tile<4, BT>(a, m, tile, cur, iters, ovf, list_next, count_next, done_ctr,
                                      (unsigned)s_claim[4], s_wlist);
                else
                    sweep_tile<NPT, BT>(a, m, tile, cur, iters, ovf, list_next, count_next,
                                        done_ctr, (unsigned)s_claim[4], s_wlist);
                ovf = __syncthreads_or(ovf);
                va = 1;
            } else {   // PH_LABELS
                int bad = 0;
                va = labels_tile(a, tile, s_st.ht_labels ? a.s.ht : a.hgt, bad);
                vb = bad;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            long long *rp = c->red[slot];
            if (va) atomicAdd((unsigned long long *)&rp[0], (unsigned long long)va);
            if (vb) atomicAdd((unsigned long long *)&rp[1], (unsigned long long)vb);
            if (vc) atomicAdd((unsigned long long *)&rp[2], (unsigned long long)vc);
            if (ovf) atomicAdd((unsigned long long *)&rp[3], 1ull);
            // the step's item count, as claimed (the step cannot end before
            // this item does); the count is a release (the item's writes
            // before it) and an acquire (every item's writes after it)
            const unsigned total = (unsigned)s_claim[4];
            if (atom_add_acq_rel(&c->done, 1u) + 1u == total) end_step(B, pr, slot);
        }
        __syncthreads();
    }
    // pairs still running when the launch gave up
    if (blockIdx.x == 0 && aborted(B.bar)) {
        __syncthreads();
        for (int p = threadIdx.x; p < B.n; p += blockDim.x) {
            PairState st;
            load_state(&st, &B.ctl[p].st);
            if (st.phase != PH_DONE) pair_results(B, st, B.pair[p], GS_ERR_TIMEOUT);
        }
    }
}

// ------------------------------------------------------------ host side ---

// Tile shape: whole chains (all K layers), TW sites x TH rows.  The shared
// memory holds 9 int32 fields over the tile and a one-site halo; at most 8
// nodes per thread (4 preferred).  Wider tiles first (coalesced rows of 32
// sites), then the tallest that fits up to TH = 4.
static bool pick_tile(const Geom &g, TileGeom &t, int &npt, size_t &smem, int want_w = 0,
                      int want_h = 0, int bt = kTileThreads) {
    // dynamic shared memory of a tile; with the kernel's ~34 KB of static
    // shared arrays it must stay under the 227 KB a block may opt in to.  With
    // 256-thread blocks the library's own choice first tries to keep two tiles
    // within an SM (long chains fall back to one block per SM).
    const size_t budgets[2] = {(bt == 256 && !want_w) ? size_t(80 * 1024) : size_t(180 * 1024),
                               size_t(180 * 1024)};
    // more sites first, squarer first among equals: a breadth-first path then
    // crosses fewer tile borders (measured: 8x8 beats 16x4 at 31 depth layers,
    // 8x4 beats 16x2 at 47)
    static const int cand[][2] = {{16, 8}, {8, 8}, {16, 4}, {32, 4}, {8, 4}, {32, 2},
                                  {16, 2}, {4, 8}, {8, 2},  {4, 4},  {16, 1}, {8, 1},
                                  {4, 2},  {4, 1}};
    if (want_w || want_h) {
        if (!(want_w == 4 || want_w == 8 || want_w == 16 || want_w == 32) || want_h < 1 ||
            want_h > 8)
            return false;
    }
    for (int pass = 0; pass < 4; pass++) {
        const size_t budget = budgets[pass / 2];
        const int max_nodes = (pass % 2 == 0 ? 4 : 8) * bt;
        for (int ci = 0; ci < (want_w ? 1 : (int)(sizeof(cand) / sizeof(cand[0]))); ci++) {
            const int TW = want_w ? want_w : cand[ci][0], TH = want_w ? want_h : cand[ci][1];
            const int TN = TH * g.K * TW;
            // Bank-conflict-free placement: a warp takes the same TW sites in
            // R = 32 / TW consecutive rows of sites (same layer), and the row
            // stride is padded to TW (mod 32), so its 32 lanes touch 32
            // different banks in every access of a visit (two rows of 16
            // sites one layer apart, 18 words apart, shared two banks).
            // Needs TH a multiple of R.
            const int R = (TW <= 32 && TH % (32 / TW) == 0) ? 32 / TW : 0;
            int SYs = g.K * (TW + 2);
            if (R) SYs += ((TW - SYs) % 32 + 32) % 32;
            const int PN = (TH + 2) * SYs;
            const size_t bytes = 9 * (size_t)PN * sizeof(int32_t);
            // the packed node info holds shared indices below 8192 and depth
            // layers below 2048
            if (TN > max_nodes || TN > kMaxTileNodes || bytes > budget || PN >= 8192 ||
                g.K >= 2048)
                continue;
            t.TW = TW;
            t.TH = TH;
            t.PW = TW + 2;
            t.SJ = t.PW;
            t.SYs = SYs;
            t.PN = PN;
            t.TN = TN;
            t.R = R;
            // a multiplier near 0.618 M coprime with M: the groups a thread
            // holds (32 x 16 nodes apart) map to spread-out parts of the tile,
            // so a cluster of active nodes falls on many warps, not on one
            t.spread = 1;
            if (R) {
                const int M = TN / 32;
                for (int a = (int)(0.618 * M); a < 2 * M + 2; a++) {
                    int x = a, y = M;
                    while (y) {
                        const int r = x % y;
                        x = y;
                        y = r;
                    }
                    if (a >= 1 && x == 1) {
                        t.spread = a % M == 0 ? 1 : a;
                        break;
                    }
                }
            }
            t.tiles_w = (g.ng + TW - 1) / TW;
            t.tiles_h = (g.h + TH - 1) / TH;
            t.T = t.tiles_w * t.tiles_h;
            npt = pass % 2 == 0 ? 4 : 8;
            smem = bytes;
            return true;
        }
    }
    return false;
}

// Per-tile flags are sized for the most tiles any allowed shape gives (4 x 1
// sites), so one workspace serves every tile shape.
static int64_t max_tiles(const Geom &g) { return (int64_t)((g.ng + 3) / 4) * g.h; }

size_t tiled_work_extra(const Geom &g) {
    return round_up(g.N * sizeof(uint16_t), 256) + round_up(8 * max_tiles(g) * sizeof(int32_t), 256);
}

// Per-pair arguments from the pair's geometry, state and workspace.
static int setup_args(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                      SolveArgs &a, int &npt, size_t &smem, int bt) {
    memset(&a, 0, sizeof(a));
    a.g = g;
    a.s = s;
    if (!pick_tile(g, a.t, npt, smem, o->tile_w, o->tile_h, bt)) return GS_ERR_INVAL;
    a.npt = npt;
    // a step's item count travels in 24 bits of the claim word
    if (a.t.T > (int)(kItemMask - 4096)) return GS_ERR_INVAL;
    char *extra = (char *)w.mark + round_up(g.N * sizeof(int32_t), 256);
    a.amask = (uint16_t *)extra;
    a.tile_act = (int32_t *)(extra + round_up(g.N * sizeof(uint16_t), 256));
    a.tile_dirty = a.tile_act + 2 * a.t.T;
    a.tile_cnt = a.tile_act + 4 * a.t.T;
    a.tile_list = a.tile_act + 5 * a.t.T;
    a.ctrl = w.ctrl;
    return GS_OK;
}

static void solve_fields(SolveArgs &a, const gs_solve_opts *o) {
    a.hgt = a.s.ht;
    a.dir = 0;
    a.mode = o->mode;
    a.sweeps_per_relabel = o->sweeps_per_relabel;
    a.local_iters = o->local_iters > 0 ? o->local_iters : 8;
    a.relabel_passes = o->relabel_passes > 0 ? o->relabel_passes : 8;
    a.tail_iters = o->tail_iters > 0 ? o->tail_iters : 4 * a.local_iters;
    a.fixed_sweeps = o->fixed_sweeps;
    a.max_iters = o->max_iters;
}

// Cooperative launch of the batch kernel with the whole grid resident.  The
// launch goes through cudaLaunchKernelEx with the cooperative attribute, so a
// caller may capture it in a CUDA graph.
static int launch_batch(const BatchArgs &B, int npt, size_t smem, int total_tiles, int bt,
                        cudaStream_t st) {
    void (*kern)(const BatchArgs) = bt == 256 ? (npt == 4 ? k_batch<4, 256> : k_batch<8, 256>)
                                              : (npt == 4 ? k_batch<4, 512> : k_batch<8, 512>);
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    int sms = 0, coop = 0;
    GS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return GS_ERR_CUDA;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, bt, smem));
    if (per_sm < 1) return GS_ERR_INVAL;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(per_sm * sms, total_tiles));
    cfg.blockDim = dim3(bt);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GS_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, B));
    count_launches(1);
    return GS_OK;
}

// Control words of a batch launch: the abort flag and finished-pair count,
// then one PairCtl per pair.
constexpr size_t kBatchCtrlBytes = 256 + kMaxPairs * sizeof(PairCtl);
static_assert(256 + kBatchCtrlBytes <= kWorkCtrlBytes, "a pair's workspace holds a batch's control");

// Idle limit of a launch from one pair's options (0: the default); a batch
// takes the smallest.
static unsigned long long idle_limit_ns(const gs_solve_opts *o) {
    return o->idle_limit_us > 0 ? 1000ull * (unsigned long long)o->idle_limit_us
                                : kDefaultIdleLimitNs;
}

static int run_batch(BatchArgs &B, int npt, size_t smem, int bt, void *ctrl_mem,
                     cudaStream_t st) {
    B.bar = (Ctrl *)ctrl_mem;
    B.ctl = (PairCtl *)((char *)ctrl_mem + 256);
    int total = 0;
    for (int p = 0; p < B.n; p++) total += B.pair[p].t.T;
    GS_CUDA_TRY(cudaMemsetAsync(ctrl_mem, 0, 256 + (size_t)B.n * sizeof(PairCtl), st));
    return launch_batch(B, npt, smem, total, bt, st);
}

size_t batch_ctrl_bytes() { return kBatchCtrlBytes; }

// Threads per block a pair's options ask for.
static int cta_threads(const gs_solve_opts *o) { return o->cta_threads == 256 ? 256 : 512; }

int tiled_solve(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                int32_t *status, cudaStream_t st) {
    static BatchArgs B;   // host staging of the kernel argument (copied at launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    memset(&B, 0, sizeof(B));
    B.n = 1;
    B.extract = 0;
    B.idle_limit_ns = idle_limit_ns(o);
    int npt;
    size_t smem;
    const int bt = cta_threads(o);
    int rc = setup_args(g, s, w, o, B.pair[0], npt, smem, bt);
    if (rc) return rc;
    solve_fields(B.pair[0], o);
    B.pair[0].status = status;
    GS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), st));
    return run_batch(B, npt, smem, bt, (char *)w.ctrl + 256, st);
}

int tiled_extract(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                  int32_t *labels, int64_t *flow, int32_t *status, cudaStream_t st) {
    static BatchArgs B;
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    memset(&B, 0, sizeof(B));
    B.n = 1;
    B.extract = 1;
    B.idle_limit_ns = idle_limit_ns(o);
    int npt;
    size_t smem;
    const int bt = cta_threads(o);
    int rc = setup_args(g, s, w, o, B.pair[0], npt, smem, bt);
    if (rc) return rc;
    SolveArgs &a = B.pair[0];
    a.hgt = w.mark;
    a.dir = o->mode == GS_MODE_EXACT ? 2 : 0;
    a.mode = GS_MODE_EXACT;
    a.max_iters = 1;
    a.labels = labels;
    a.flow = flow;
    a.status = status;
    return run_batch(B, npt, smem, bt, (char *)w.ctrl + 256, st);
}

}  // namespace gs

extern "C" int gs_tile_info(const gs_params *p, const gs_solve_opts *o, int32_t *out) {
    gs::Geom g;
    if (gs::make_geom(p, &g) != GS_OK || !o || !out) return GS_ERR_INVAL;
    gs::TileGeom t;
    int npt;
    size_t smem;
    if (!gs::pick_tile(g, t, npt, smem, o->tile_w, o->tile_h, gs::cta_threads(o)))
        return GS_ERR_INVAL;
    out[0] = t.TW;
    out[1] = t.TH;
    out[2] = t.T;
    out[3] = (int32_t)smem;
    return GS_OK;
}

// ------------------------------------------------------------ batched ABI ---

extern "C" size_t gs_batch_workspace_bytes(int32_t n) {
    if (n < 1 || n > gs::kMaxPairs) return 0;
    return gs::kBatchCtrlBytes;
}

extern "C" int gs_solve_batched(const gs_pair_desc *descs, int32_t n, void *batch_ws, void *stream) {
    using namespace gs;
    if (!descs || n < 1 || n > kMaxPairs || !batch_ws || ((uintptr_t)batch_ws & 255))
        return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    static BatchArgs B, E;   // host staging of the kernel arguments (copied at launch)
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    memset(&B, 0, sizeof(B));
    memset(&E, 0, sizeof(E));
    B.n = E.n = n;
    B.extract = 0;
    E.extract = 1;
    B.idle_limit_ns = kDefaultIdleLimitNs;
    int npt_max = 4;
    size_t smem_max = 0;
    // one block size for the launch: 256 threads only when every pair asks
    int bt = 256;
    for (int i = 0; i < n; i++)
        if (cta_threads(&descs[i].o) != 256) bt = 512;
    for (int i = 0; i < n; i++) {
        const gs_pair_desc &d = descs[i];
        Geom g;
        if (make_geom(&d.p, &g) != GS_OK || !d.L || !d.R || !d.cost || !d.graph || !d.workspace ||
            !d.labels || !d.flow || !d.status)
            return GS_ERR_INVAL;
        if (gs_check_solve_opts(&d.o) != GS_OK || d.o.engine != GS_ENGINE_TILED ||
            ((uintptr_t)d.graph & 255) || ((uintptr_t)d.workspace & 255))
            return GS_ERR_INVAL;
        B.idle_limit_ns = std::min(B.idle_limit_ns, idle_limit_ns(&d.o));
        const State s = state_view(d.graph, g);
        const Work w = work_view(d.workspace, g);
        int npt;
        size_t smem;
        if (setup_args(g, s, w, &d.o, B.pair[i], npt, smem, bt) != GS_OK) return GS_ERR_INVAL;
        solve_fields(B.pair[i], &d.o);
        B.pair[i].status = d.status;
        E.pair[i] = B.pair[i];
        SolveArgs &x = E.pair[i];
        x.hgt = w.mark;
        x.dir = d.o.mode == GS_MODE_EXACT ? 2 : 0;
        x.mode = GS_MODE_EXACT;
        x.max_iters = 1;
        x.labels = d.labels;
        x.flow = d.flow;
        npt_max = std::max(npt_max, npt);
        smem_max = std::max(smem_max, smem);
    }
    // per pair: data term and graph (small launches), then one launch for all
    // solves and one for all label extractions
    for (int i = 0; i < n; i++) {
        const gs_pair_desc &d = descs[i];
        int rc = gs_stereo_cost_volume(d.L, d.R, d.p.w, &d.p, d.cost, stream);
        if (rc) return rc;
        rc = gs_build_graph(d.cost, &d.p, d.graph, d.status, stream);
        if (rc) return rc;
        GS_CUDA_TRY(cudaMemsetAsync(B.pair[i].ctrl, 0, sizeof(Ctrl), st));
    }
    E.idle_limit_ns = B.idle_limit_ns;
    int rc = run_batch(B, npt_max, smem_max, bt, batch_ws, st);
    if (rc) return rc;
    return run_batch(E, npt_max, smem_max, bt, batch_ws, st);
}
