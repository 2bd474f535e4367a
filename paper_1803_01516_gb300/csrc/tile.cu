// Persistent, tiled push-relabel with global relabelling (§4.4) for the chain
// graph of §3 / Fig. 4.
//
// One cooperative launch runs the whole solve.  The node grid is cut into
// tiles of TW sites x TH rows x all K chain layers (whole chains, so the data
// arcs and their infinite reverse arcs never leave a tile).  A CTA stages a
// tile plus a one-site halo in shared memory and works on it locally; tiles
// exchange flow only through atomics on global memory, and CTAs meet at grid
// barriers between phases:
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
#include <cooperative_groups.h>

#include "arcs.cuh"

namespace gs {

constexpr int kTileThreads = 512;
constexpr int kMaxTileNodes = 4096;           // own nodes per tile (8 per thread at most)
constexpr long long kSpinLimit = 1ll << 24;   // grid-barrier wait bound (~1-2 s)

struct TileGeom {
    int TW, TH;        // sites per tile along W and y
    int PW;            // padded row length TW + 2
    int SJ;            // shared-memory stride of one chain layer (= PW)
    int SYs;           // shared-memory stride of one row (= K * PW)
    int PN;            // padded nodes per tile (TH + 2) * K * PW
    int TN;            // own nodes per tile TH * K * TW
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
    void *log;           // diagnostics: per-relabel counters (label-mark buffer)
    int32_t *hgt;        // distances the relabel passes compute (state heights, or marks)
    int dir;             // 0: distance to sink capacity over out-arcs (heights);
                         // 1: distance from positive excess over in-arcs (reachability)
    Ctrl *ctrl;
    int mode, sweeps_per_relabel, local_iters, relabel_passes, tail_iters;
    long long fixed_sweeps, max_iters;
};

// ------------------------------------------------------------ grid sync ---

// Grid-wide barrier that also sums two values over the blocks (thread 0's
// arguments count).  Waits are bounded: after kSpinLimit polls the block sets
// ctrl->abort and leaves.
struct Sum2 {
    long long a, b;
};

__device__ Sum2 grid_sync_sum2(Ctrl *ctrl, long long va, long long vb) {
    __shared__ long long s_res[2];
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &ctrl->bar_gen;
        const unsigned int gen = *vgen;
        const int slot = gen & 1;
        if (va) atomicAdd((unsigned long long *)&ctrl->bar_red[slot][0], (unsigned long long)va);
        if (vb) atomicAdd((unsigned long long *)&ctrl->bar_red[slot][1], (unsigned long long)vb);
        __threadfence();
        const unsigned int arrived = atomicAdd(&ctrl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            ctrl->bar_count = 0;
            ctrl->bar_red[slot ^ 1][0] = 0;
            ctrl->bar_red[slot ^ 1][1] = 0;
            __threadfence();
            atomicAdd(&ctrl->bar_gen, 1u);
        } else {
            long long spins = 0;
            while (*vgen == gen) {
                if (++spins > kSpinLimit) {
                    atomicExch(&ctrl->abort, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_res[0] = *(volatile long long *)&ctrl->bar_red[slot][0];
        s_res[1] = *(volatile long long *)&ctrl->bar_red[slot][1];
    }
    __syncthreads();
    return Sum2{s_res[0], s_res[1]};
}

__device__ __forceinline__ long long grid_sync_sum(Ctrl *ctrl, long long v) {
    return grid_sync_sum2(ctrl, v, 0).a;
}

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

// Apply a push of d along slot q to the residual words in shared memory; when
// the word belongs to a halo node (slots whose residual is stored at the arc's
// head), the global copy is updated at once as well.  Only the data-arc
// residual can grow without a bound of its own (flow pushed back along the
// infinite reverse arc); its new value is returned for the overflow check.
// Every other word is a residual of an arc pair and stays within the pair's
// capacity, so those updates need no returned value.
__device__ __forceinline__ int32_t smem_push_residual(const TileSmem &m, const TileGeom &t,
                                                      const State &s, int pi, int64_t gi,
                                                      const Geom &g, int q, int32_t d,
                                                      bool head_is_halo) {
    switch (q) {
        case 0: atomicSub(&m.rc[pi], d); return 0;
        case 1: return atomicAdd(&m.rc[pi - t.SJ], d) + d;   // chain never leaves the tile
        case 2: atomicSub(&m.rr[pi], d); return 0;
        case 3:
            if (head_is_halo) atomicAdd(&s.rr[gi - 1], d);
            atomicAdd(&m.rr[pi - 1], d);
            return 0;
        case 4: atomicSub(&m.rd[pi], d); return 0;
        case 5:
            if (head_is_halo) atomicAdd(&s.rd[gi - g.SY], d);
            atomicAdd(&m.rd[pi - t.SYs], d);
            return 0;
        case 6: atomicSub(&m.ri0[pi], d); return 0;
        case 7: atomicSub(&m.ri1[pi], d); return 0;
        case 8: atomicSub(&m.ri2[pi], d); return 0;
        case 9: atomicSub(&m.ri3[pi], d); return 0;
        case 10:
            if (head_is_halo) atomicAdd(&s.ri1[gi - 1 + g.P], d);
            atomicAdd(&m.ri1[pi - 1 + t.SJ], d);
            return 0;
        case 11:
            if (head_is_halo) atomicAdd(&s.ri0[gi + 1 + g.P], d);
            atomicAdd(&m.ri0[pi + 1 + t.SJ], d);
            return 0;
        case 12:
            if (head_is_halo) atomicAdd(&s.ri3[gi - g.SY + g.P], d);
            atomicAdd(&m.ri3[pi - t.SYs + t.SJ], d);
            return 0;
        default:
            if (head_is_halo) atomicAdd(&s.ri2[gi + g.SY + g.P], d);
            atomicAdd(&m.ri2[pi + t.SYs + t.SJ], d);
            return 0;
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

// Load the halo (one site around the tile, all layers) for the fields the
// arcs of the tile's own nodes read: heights everywhere, and the residual
// words stored at the head of an arc (rr, ri1 at W0-1; ri0 at W0+TW; rd, ri3
// at y0-1; ri2 at y0+TH).  Positions outside the grid get height kInfH and
// zero residuals.
__device__ void load_halo(const SolveArgs &a, const TileSmem &m, const TileOrigin &o,
                          bool with_residuals, const int32_t *hsrc) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const State &s = a.s;
    // left / right columns: TH * K each
    for (int n = threadIdx.x; n < 2 * t.TH * g.K; n += blockDim.x) {
        const int side = n / (t.TH * g.K);
        const int r = n - side * t.TH * g.K;
        const int yl = r / g.K, j = r - yl * g.K;
        const int wl = side ? t.TW : -1;
        const int W = o.W0 + wl, y = o.y0 + yl;
        const int pi = pidx(t, yl, j, wl);
        const bool in = W >= 0 && W < g.ng && y < g.h;
        const int64_t gi = ((int64_t)y * g.K + j) * g.P + W;
        m.ht[pi] = in ? ld(&hsrc[gi]) : kInfH;
        if (with_residuals) {
            if (side == 0) {
                m.rr[pi] = in ? ld(&s.rr[gi]) : 0;
                m.ri1[pi] = in ? ld(&s.ri1[gi]) : 0;
            } else {
                m.ri0[pi] = in ? ld(&s.ri0[gi]) : 0;
            }
        }
    }
    // top / bottom rows: K * TW each
    for (int n = threadIdx.x; n < 2 * g.K * t.TW; n += blockDim.x) {
        const int side = n / (g.K * t.TW);
        const int r = n - side * g.K * t.TW;
        const int j = r / t.TW, wl = r - j * t.TW;
        const int yl = side ? t.TH : -1;
        const int W = o.W0 + wl, y = o.y0 + yl;
        const int pi = pidx(t, yl, j, wl);
        const bool in = y >= 0 && y < g.h && W < g.ng;
        const int64_t gi = ((int64_t)y * g.K + j) * g.P + W;
        m.ht[pi] = in ? ld(&hsrc[gi]) : kInfH;
        if (with_residuals) {
            if (side == 0) {
                m.rd[pi] = in ? ld(&s.rd[gi]) : 0;
                m.ri3[pi] = in ? ld(&s.ri3[gi]) : 0;
            } else {
                m.ri2[pi] = in ? ld(&s.ri2[gi]) : 0;
            }
        }
    }
}

// ---------------------------------------------------------- relabel pass ---

// Local relaxation to the tile's fixed point.  Own nodes' residual-arc masks
// are in registers (mk), own heights and halo heights in shared memory.  A
// row of the tile (one depth layer of one site row) is revisited only while a
// row it has arcs into (same, next and previous layer and site row) changed in
// the previous iteration; three rotating bitmaps carry the changed rows.
constexpr int kMaxRows = 1024;

template <int NPT>
__device__ bool relax_tile(const SolveArgs &a, const TileSmem &m, const int (&pi)[NPT],
                           const unsigned (&mk)[NPT]) {
    const TileGeom &t = a.t;
    const int K = a.g.K;
    const int R = t.TH * K;
    const int RW = (R + 31) >> 5;
    __shared__ unsigned dirty[3][kMaxRows / 32];
    int off[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; q++) off[q] = soff(t, q);
    for (int w = threadIdx.x; w < 3 * (kMaxRows / 32); w += blockDim.x) (&dirty[0][0])[w] = 0;
    __syncthreads();
    int row[NPT];
#pragma unroll
    for (int k = 0; k < NPT; k++) row[k] = (threadIdx.x + k * blockDim.x) / t.TW;
    bool any_change = false;
    for (int iter = 0;; iter++) {
        const unsigned *cur = dirty[iter % 3];
        unsigned *nxt = dirty[(iter + 1) % 3];
        unsigned *clr = dirty[(iter + 2) % 3];
        for (int w = threadIdx.x; w < RW; w += blockDim.x) clr[w] = 0;
        int changed = 0;
#pragma unroll
        for (int k = 0; k < NPT; k++) {
            if (pi[k] < 0) continue;
            const int r = row[k];
            if (iter > 0) {
                bool dep = false;
#pragma unroll
                for (int dy = -1; dy <= 1; dy++)
#pragma unroll
                    for (int dj = -1; dj <= 1; dj++) {
                        const int rr = r + dy * K + dj;
                        if (rr >= 0 && rr < R) dep |= (cur[rr >> 5] >> (rr & 31)) & 1u;
                    }
                if (!dep) continue;
            }
            const int32_t h = m.ht[pi[k]];
            if (h == 0) continue;
            int32_t hmin = kInfH;
            const unsigned bits = mk[k] & 0x3fffu;
#pragma unroll
            for (int q = 0; q < kSlots; q++)
                if (bits & (1u << q)) hmin = min(hmin, m.ht[pi[k] + off[q]]);
            if (hmin < kInfH && hmin + 1 < h) {
                m.ht[pi[k]] = hmin + 1;
                atomicOr(&nxt[r >> 5], 1u << (r & 31));
                changed = 1;
            }
        }
        if (!__syncthreads_or(changed)) break;
        any_change = true;
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
    load_halo(a, m, o, true, a.hgt);
    int pi[NPT];
    unsigned mk[NPT];
    int64_t gi[NPT];
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        pi[k] = -1;
        mk[k] = 0;
        gi[k] = 0;
        if (n >= t.TN) continue;
        const int wl = n % t.TW, r = n / t.TW, j = r % g.K, yl = r / g.K;
        const int W = o.W0 + wl, y = o.y0 + yl;
        const int p = pidx(t, yl, j, wl);
        if (W >= g.ng || y >= g.h) {
            m.ht[p] = kInfH;
            continue;
        }
        const int64_t i = ((int64_t)y * g.K + j) * g.P + W;
        pi[k] = p;
        gi[k] = i;
        m.rc[p] = ld(&s.rc[i]);
        m.rr[p] = ld(&s.rr[i]);
        m.rd[p] = ld(&s.rd[i]);
        m.ri0[p] = ld(&s.ri0[i]);
        m.ri1[p] = ld(&s.ri1[i]);
        m.ri2[p] = ld(&s.ri2[i]);
        m.ri3[p] = ld(&s.ri3[i]);
        const int32_t e = ld(&s.ex[i]);
        if (a.dir == 0) {
            m.ht[p] = e < 0 ? 0 : kInfH;
            mk[k] = e > 0 ? 0x8000u : 0u;
        } else {
            m.ht[p] = e > 0 ? 0 : kInfH;
        }
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const int n = threadIdx.x + k * blockDim.x;
        const int wl = n % t.TW, r = n / t.TW, j = r % g.K, yl = r / g.K;
        const unsigned ex = arc_exists(g, o.y0 + yl, j, o.W0 + wl);
#pragma unroll
        for (int q = 0; q < kSlots; q++) {
            if (!((ex >> q) & 1u)) continue;
            bool res;
            if (a.dir == 0) {
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
    // halo heights are not known yet in this pass: treat as infinite
    for (int n = threadIdx.x; n < 2 * t.TH * g.K; n += blockDim.x) {
        const int side = n / (t.TH * g.K), r = n - side * t.TH * g.K;
        const int yl = r / g.K, j = r - yl * g.K;
        m.ht[pidx(t, yl, j, side ? t.TW : -1)] = kInfH;
    }
    for (int n = threadIdx.x; n < 2 * g.K * t.TW; n += blockDim.x) {
        const int side = n / (g.K * t.TW), r = n - side * g.K * t.TW;
        const int j = r / t.TW, wl = r - j * t.TW;
        m.ht[pidx(t, side ? t.TH : -1, j, wl)] = kInfH;
    }
    __syncthreads();
    relax_tile<NPT>(a, m, pi, mk);
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

// Later relabel passes: masks from the first pass, heights from global
// memory (own and halo); relax, write back what changed, mark the neighbour
// tiles whose halo changed, and return the change of the tile's active count.
template <int NPT>
__device__ long long relabel_pass_tile(const SolveArgs &a, const TileSmem &m, int tile,
                                       int &changed, int32_t *dirty_next) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const State &s = a.s;
    const TileOrigin o = tile_origin(t, tile);
    load_halo(a, m, o, false, a.hgt);
    int pi[NPT];
    unsigned mk[NPT];
    int64_t gi[NPT];
    int32_t h0[NPT];
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        pi[k] = -1;
        mk[k] = 0;
        gi[k] = 0;
        h0[k] = kInfH;
        if (n >= t.TN) continue;
        const int wl = n % t.TW, r = n / t.TW, j = r % g.K, yl = r / g.K;
        const int W = o.W0 + wl, y = o.y0 + yl;
        const int p = pidx(t, yl, j, wl);
        if (W >= g.ng || y >= g.h) {
            m.ht[p] = kInfH;
            continue;
        }
        const int64_t i = ((int64_t)y * g.K + j) * g.P + W;
        pi[k] = p;
        gi[k] = i;
        mk[k] = ld(&a.amask[i]);
        h0[k] = ld(&a.hgt[i]);
        m.ht[p] = h0[k];
    }
    __shared__ int s_sides;
    if (threadIdx.x == 0) s_sides = 0;
    __syncthreads();
    const bool ch = relax_tile<NPT>(a, m, pi, mk);
    int act = 0;
    unsigned sides = 0;
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const int32_t h = m.ht[pi[k]];
        if (h != h0[k]) {
            __stcg(&a.hgt[gi[k]], h);
            const int n = threadIdx.x + k * blockDim.x;
            const int wl = n % t.TW, yl = (n / t.TW) / g.K;
            sides |= (wl == 0 ? 1u : 0u) | (wl == t.TW - 1 ? 2u : 0u) | (yl == 0 ? 4u : 0u) |
                     (yl == t.TH - 1 ? 8u : 0u);
        }
        act += (mk[k] & 0x8000u) && h < kInfH;
    }
    if (sides) atomicOr(&s_sides, (int)sides);
    const long long tot = block_sum(act);   // also orders s_sides
    if (threadIdx.x == 0) {
        const unsigned sd = (unsigned)s_sides;
        if ((sd & 1u) && o.tx > 0) __stcg(&dirty_next[tile - 1], 1);
        if ((sd & 2u) && o.tx + 1 < t.tiles_w) __stcg(&dirty_next[tile + 1], 1);
        if ((sd & 4u) && o.ty > 0) __stcg(&dirty_next[tile - t.tiles_w], 1);
        if ((sd & 8u) && o.ty + 1 < t.tiles_h) __stcg(&dirty_next[tile + t.tiles_w], 1);
    }
    if (ch) changed = 1;
    const long long before = ld(&a.tile_cnt[tile]);
    __syncthreads();
    if (threadIdx.x == 0) __stcg(&a.tile_cnt[tile], (int32_t)tot);
    return tot - before;
}

// ------------------------------------------------------------ sweep visit ---

// Up to local_iters push/relabel iterations of one tile in shared memory.
template <int NPT>
__device__ void sweep_tile(const SolveArgs &a, const TileSmem &m, int tile, int round, int iters,
                           int &overflow) {
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const State &s = a.s;
    const TileOrigin o = tile_origin(t, tile);
    int32_t *act_next = a.tile_act + ((round + 1) & 1) * t.T;
    // per own node: shared index, coordinates in the tile and existing arcs,
    // so the discharge loop needs no divisions
    __shared__ uint32_t s_info[kMaxTileNodes];
    __shared__ uint16_t s_exb[kMaxTileNodes];
    load_halo(a, m, o, true, s.ht);
    int pi[NPT];
    int64_t gi[NPT];
    unsigned ex_bits[NPT];
    int32_t o_ex[NPT], o_rc[NPT], o_rr[NPT], o_rd[NPT], o_r0[NPT], o_r1[NPT], o_r2[NPT],
        o_r3[NPT], o_ht[NPT];
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        const int n = threadIdx.x + k * blockDim.x;
        pi[k] = -1;
        gi[k] = 0;
        ex_bits[k] = 0;
        if (n >= t.TN) continue;
        const int wl = n % t.TW, r = n / t.TW, j = r % g.K, yl = r / g.K;
        const int W = o.W0 + wl, y = o.y0 + yl;
        const int p = pidx(t, yl, j, wl);
        if (W >= g.ng || y >= g.h) {
            m.ht[p] = kInfH;
            m.ex[p] = 0;
            continue;
        }
        const int64_t i = ((int64_t)y * g.K + j) * g.P + W;
        pi[k] = p;
        gi[k] = i;
        ex_bits[k] = arc_exists(g, y, j, W);
        s_info[n] = (uint32_t)p | ((uint32_t)wl << 16) | ((uint32_t)yl << 21) | ((uint32_t)j << 25);
        s_exb[n] = (uint16_t)ex_bits[k];
        m.ex[p] = o_ex[k] = ld(&s.ex[i]);
        m.ht[p] = o_ht[k] = ld(&s.ht[i]);
        m.rc[p] = o_rc[k] = ld(&s.rc[i]);
        m.rr[p] = o_rr[k] = ld(&s.rr[i]);
        m.rd[p] = o_rd[k] = ld(&s.rd[i]);
        m.ri0[p] = o_r0[k] = ld(&s.ri0[i]);
        m.ri1[p] = o_r1[k] = ld(&s.ri1[i]);
        m.ri2[p] = o_r2[k] = ld(&s.ri2[i]);
        m.ri3[p] = o_r3[k] = ld(&s.ri3[i]);
    }
    __syncthreads();
    int off[kSlots];
    int64_t goff[kSlots];
#pragma unroll
    for (int q = 0; q < kSlots; q++) {
        off[q] = soff(t, q);
        int dy, dj, dw;
        slot_delta(q, dy, dj, dw);
        goff[q] = dy * g.SY + (int64_t)dj * g.P + dw;
    }
    // Each local iteration first compacts the tile's active nodes (positive
    // excess, finite height) into a list, then discharges the list densely, so
    // warps do not idle on inactive lanes.
    __shared__ int s_nact[2];
    __shared__ uint16_t s_list[kMaxTileNodes];
    const int64_t tile_g0 = (int64_t)o.y0 * g.SY + o.W0;
    if (threadIdx.x == 0) s_nact[0] = s_nact[1] = 0;
    __syncthreads();
    unsigned nb_touch = 0;   // bit 0: left, 1: right, 2: up, 3: down neighbour tile received flow
    const int lane = threadIdx.x & 31;
    for (int it = 0; it < iters; it++) {
        int *cnt = &s_nact[it & 1];
#pragma unroll
        for (int k = 0; k < NPT; k++) {
            const bool act = pi[k] >= 0 && m.ex[pi[k]] > 0 && m.ht[pi[k]] < kInfH;
            const unsigned bal = __ballot_sync(0xffffffffu, act);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(cnt, __popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (act) s_list[base + __popc(bal & ((1u << lane) - 1u))] =
                    (uint16_t)(threadIdx.x + k * blockDim.x);
            }
        }
        __syncthreads();
        const int nact = *cnt;
        if (threadIdx.x == 0) s_nact[(it + 1) & 1] = 0;
        if (nact == 0) break;
        for (int li = threadIdx.x; li < nact; li += blockDim.x) {
            const int n = s_list[li];
            const uint32_t info = s_info[n];
            const int p = (int)(info & 0xffffu);
            const int wl = (int)((info >> 16) & 31u), yl = (int)((info >> 21) & 15u);
            const int j = (int)(info >> 25);
            const int64_t gin = tile_g0 + (int64_t)yl * g.SY + (int64_t)j * g.P + wl;
            const unsigned exb = s_exb[n];
            const int32_t e = m.ex[p];
            const int32_t hu = m.ht[p];
            if (e <= 0 || hu >= kInfH) continue;
            int32_t rr[kSlots], hv[kSlots];
#pragma unroll
            for (int q = 0; q < kSlots; q++) {
                rr[q] = ((exb >> q) & 1u) ? smem_residual(m, t, g, p, q) : 0;
                hv[q] = rr[q] > 0 ? m.ht[p + off[q]] : kInfH;
            }
            int32_t left = e;
#pragma unroll
            for (int q = 0; q < kSlots; q++) {
                if (left > 0 && rr[q] > 0 && hv[q] < hu) {
                    const int32_t d = min(left, rr[q]);
                    int dy, dj, dw;
                    slot_delta(q, dy, dj, dw);
                    const int wl2 = wl + dw, yl2 = yl + dy;
                    const bool halo = wl2 < 0 || wl2 >= t.TW || yl2 < 0 || yl2 >= t.TH;
                    const int32_t grown = smem_push_residual(m, t, s, p, gin, g, q, d, halo);
                    overflow |= grown > kCapLimit;
                    // an excess never exceeds the total source capacity (<= 2^30,
                    // checked when the graph is built): no overflow check needed
                    if (halo) {
                        atomicAdd(&s.ex[gin + goff[q]], d);
                        nb_touch |= wl2 < 0 ? 1u : wl2 >= t.TW ? 2u : yl2 < 0 ? 4u : 8u;
                    } else {
                        atomicAdd(&m.ex[p + off[q]], d);
                    }
                    rr[q] -= d;
                    left -= d;
                }
            }
            if (left != e) atomicSub(&m.ex[p], e - left);
            if (left > 0) {
                int32_t hmin = kInfH;
#pragma unroll
                for (int q = 0; q < kSlots; q++)
                    if (rr[q] > 0) hmin = min(hmin, hv[q]);
                m.ht[p] = hmin >= kInfH - 1 ? kInfH : hmin + 1;
            }
        }
        __syncthreads();
    }
    __syncthreads();
    // write back own nodes as deltas (other tiles may have updated the same
    // words through global atomics meanwhile); note whether work is left
    int still = 0;
#pragma unroll
    for (int k = 0; k < NPT; k++) {
        if (pi[k] < 0) continue;
        const int p = pi[k];
        const int64_t i = gi[k];
        int32_t v;
        if ((v = m.ex[p] - o_ex[k])) atomicAdd(&s.ex[i], v);
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
    const int still_any = __syncthreads_or(still);
    const unsigned touch = (unsigned)__syncthreads_or((int)(nb_touch & 1u)) |
                           ((unsigned)__syncthreads_or((int)(nb_touch & 2u)) << 1) |
                           ((unsigned)__syncthreads_or((int)(nb_touch & 4u)) << 2) |
                           ((unsigned)__syncthreads_or((int)(nb_touch & 8u)) << 3);
    if (threadIdx.x == 0) {
        if (still_any) __stcg(&act_next[tile], 1);
        if ((touch & 1u) && o.tx > 0) __stcg(&act_next[tile - 1], 1);
        if ((touch & 2u) && o.tx + 1 < t.tiles_w) __stcg(&act_next[tile + 1], 1);
        if ((touch & 4u) && o.ty > 0) __stcg(&act_next[tile - t.tiles_w], 1);
        if ((touch & 8u) && o.ty + 1 < t.tiles_h) __stcg(&act_next[tile + t.tiles_w], 1);
    }
    __syncthreads();
}

// ------------------------------------------------------------ the solve ---

template <int NPT>
__global__ void __launch_bounds__(kTileThreads, 1) k_solve_tiled(SolveArgs a) {
    extern __shared__ int32_t smem[];
    const TileSmem m = tile_smem(smem, a.t.PN);
    Ctrl *ctrl = a.ctrl;
    const int T = a.t.T;
    long long relabels = 0, rounds = 0, passes = 0, visits = 0, sweep_visits = 0;
    long long my_sweep_visits = 0;
    const unsigned long long t_start = now_ns();
    long long relabel_ns_local = 0;
    unsigned long long t_relabel = 0, t_sweep = 0;
    long long active = 0;
    int converged = 0, overflow = 0, full = 0;
    __shared__ int s_work;
    for (long long outer = 0;; outer++) {
        if (a.mode == GS_MODE_EXACT && outer >= a.max_iters) break;
        // ---- global relabel: first pass (masks, heights reset, in-tile distances)
        unsigned long long t0 = now_ns();
        long long cnt = 0;
        for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
            cnt += relabel_init_tile<NPT>(a, m, tile);
            visits++;
            if (threadIdx.x == 0) {
                __stcg(&a.tile_dirty[tile], 0);
                __stcg(&a.tile_dirty[T + tile], 0);
                __stcg(&a.tile_act[T + tile], 0);
            }
        }
        active = grid_sync_sum(ctrl, threadIdx.x == 0 ? cnt : 0);
        passes++;
        if (aborted(ctrl)) break;
        // ---- later passes: every tile once, then only tiles whose halo changed.
        // An intermediate relabel stops after relabel_passes passes (heights of
        // nodes not reached stay infinite until the next relabel); the relabel
        // that can end the solve runs to its fixed point, which is exact.
        int conv = 0;
        for (int pass = 1;; pass++) {
            int changed = 0;
            long long delta = 0;
            int32_t *dcur = a.tile_dirty + (pass & 1) * T;
            int32_t *dnext = a.tile_dirty + ((pass + 1) & 1) * T;
            for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
                if (pass > 1) {
                    __syncthreads();
                    if (threadIdx.x == 0) s_work = ld(&dcur[tile]);
                    __syncthreads();
                    if (!s_work) continue;
                    if (threadIdx.x == 0) __stcg(&dcur[tile], 0);
                }
                delta += relabel_pass_tile<NPT>(a, m, tile, changed, dnext);
                visits++;
            }
            const Sum2 r = grid_sync_sum2(ctrl, threadIdx.x == 0 ? delta : 0,
                                          threadIdx.x == 0 ? changed : 0);
            passes++;
            active += r.a;
            if (aborted(ctrl)) break;
            if (r.b == 0) {
                conv = 1;
                break;
            }
            if (!full && pass >= a.relabel_passes) break;
        }
        // per-relabel log in the (otherwise idle during the solve) label-mark
        // buffer: passes | converged << 32, active nodes, tile visits, elapsed ns
        if (blockIdx.x == 0 && threadIdx.x == 0 && relabels < 256) {
            long long *log = (long long *)a.log;
            log[4 * relabels + 0] = passes | ((long long)conv << 32);
            log[4 * relabels + 1] = active;
            log[4 * relabels + 2] = sweep_visits;
            log[4 * relabels + 3] = (long long)(now_ns() - t0);
        }
        // the relabel's duration as block 0 saw it, shared through the next barrier sum
        relabel_ns_local = (long long)(now_ns() - t0);
        relabels++;
        t_relabel += now_ns() - t0;
        if (aborted(ctrl)) break;
        if (active == 0) {
            if (conv) {
                converged = 1;
                break;
            }
            full = 1;          // nothing active within reach: decide with an exact relabel
            continue;
        }
        full = 0;
        // ---- sweep rounds over tiles with work.  While many nodes are active a
        // relabel follows every sweeps_per_relabel rounds; in the tail (few
        // active nodes, cheap rounds) up to 8x as many; rounds stop early once
        // no tile has work.
        const bool tail = active * 64 <= (long long)a.g.N;
        long long n = tail ? 64ll * a.sweeps_per_relabel : a.sweeps_per_relabel;
        const long long last_relabel_ns =
            grid_sync_sum(ctrl, (blockIdx.x == 0 && threadIdx.x == 0) ? relabel_ns_local : 0);
        const int iters = tail ? a.tail_iters : a.local_iters;
        if (a.mode == GS_MODE_FIXED_SWEEPS) {
            n = min(n, a.fixed_sweeps - rounds);
            if (n <= 0) break;
        }
        t0 = now_ns();
        long long prev1_worked = 1ll << 40, prev2_worked = 1ll << 40;
        for (long long r = 0; r < n; r++) {
            const int cur = (int)(r & 1);
            long long worked = 0;
            for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
                __syncthreads();
                if (threadIdx.x == 0)
                    s_work = r == 0 ? (ld(&a.tile_cnt[tile]) > 0) : ld(&a.tile_act[cur * T + tile]);
                __syncthreads();
                if (threadIdx.x == 0) __stcg(&a.tile_act[cur * T + tile], 0);
                if (s_work) {
                    sweep_tile<NPT>(a, m, tile, cur, iters, overflow);
                    worked++;
                    my_sweep_visits++;
                }
            }
            // block 0's clock rides along the grid sum so every block takes the same
            // decision: in the tail, sweep on until the rounds have cost as much as
            // the last relabel and the number of tiles with work stopped falling
            // (the excess left is circling on stale heights)
            const Sum2 rs = grid_sync_sum2(
                ctrl, threadIdx.x == 0 ? worked : 0,
                (blockIdx.x == 0 && threadIdx.x == 0) ? (long long)(now_ns() - t0) : 0);
            const long long tot_worked = rs.a;
            const bool stalled = tail && r >= 2 && tot_worked * 10 > prev2_worked * 9 &&
                                 rs.b > last_relabel_ns;
            prev2_worked = prev1_worked;
            prev1_worked = tot_worked;
            if (blockIdx.x == 0 && threadIdx.x == 0 && rounds < 4096) {
                // per-round log after the per-relabel log: tiles worked, end time
                long long *log = (long long *)a.log + 1024;
                log[2 * rounds + 0] = tot_worked | ((long long)relabels << 32);
                log[2 * rounds + 1] = (long long)(now_ns() - t_start);
            }
            rounds++;
            sweep_visits += tot_worked;
            if (aborted(ctrl) || tot_worked == 0 || stalled) break;
        }
        t_sweep += now_ns() - t0;
        if (aborted(ctrl)) break;
    }
    if (__syncthreads_or(overflow) && threadIdx.x == 0)
        atomicCAS(&ctrl->status, GS_OK, GS_ERR_OVERFLOW);
    if (threadIdx.x == 0) {
        atomicAdd((unsigned long long *)&ctrl->visits_relabel, (unsigned long long)visits);
        atomicAdd((unsigned long long *)&ctrl->visits_sweep, (unsigned long long)my_sweep_visits);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctrl->stats[0] = relabels;
        ctrl->stats[1] = rounds;
        ctrl->stats[2] = passes;
        ctrl->stats[4] = active;
        ctrl->stats[5] = (long long)t_sweep;
        ctrl->stats[6] = (long long)t_relabel;
        ctrl->converged = converged;
        if (aborted(ctrl)) atomicCAS(&ctrl->status, GS_OK, GS_ERR_TIMEOUT);
        else if (!converged && a.mode == GS_MODE_EXACT) atomicCAS(&ctrl->status, GS_OK, GS_ERR_TIMEOUT);
    }
}

// ------------------------------------------------------------ labels ---

// Reads the cut of the solved state back as labels, in one cooperative launch.
// Exact mode: S_min = nodes reachable from positive excess over residual
// arcs (dir 1, sources = excess nodes); a site's label is the number of its
// chain nodes in S_min.  Fixed-sweep mode: the source side is the set of nodes
// that cannot reach sink capacity (dir 0, exact distances, label = number of
// chain nodes at infinite distance).  Both searches run to their fixed point.
// The flow value is the sink capacity used: initial minus remaining deficit.
template <int NPT>
__global__ void __launch_bounds__(kTileThreads, 1)
    k_extract_tiled(SolveArgs a, int32_t *labels, int64_t *flow, int32_t *status) {
    extern __shared__ int32_t smem[];
    const TileSmem m = tile_smem(smem, a.t.PN);
    Ctrl *ctrl = a.ctrl;
    const Geom &g = a.g;
    const TileGeom &t = a.t;
    const int T = t.T;
    __shared__ int s_work;
    long long passes = 1;
    for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
        relabel_init_tile<NPT>(a, m, tile);
        if (threadIdx.x == 0) {
            __stcg(&a.tile_dirty[tile], 0);
            __stcg(&a.tile_dirty[T + tile], 0);
        }
    }
    grid_sync_sum(ctrl, 0);
    for (int pass = 1; !aborted(ctrl); pass++) {
        int changed = 0;
        int32_t *dcur = a.tile_dirty + (pass & 1) * T;
        int32_t *dnext = a.tile_dirty + ((pass + 1) & 1) * T;
        for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
            if (pass > 1) {
                __syncthreads();
                if (threadIdx.x == 0) s_work = ld(&dcur[tile]);
                __syncthreads();
                if (!s_work) continue;
                if (threadIdx.x == 0) __stcg(&dcur[tile], 0);
            }
            relabel_pass_tile<NPT>(a, m, tile, changed, dnext);
        }
        const Sum2 r = grid_sync_sum2(ctrl, 0, threadIdx.x == 0 ? changed : 0);
        passes++;
        if (r.b == 0) break;
    }
    // labels of the tiles' sites and the sink capacity left
    unsigned long long deficit = 0;
    int bad = 0;
    for (int tile = blockIdx.x; tile < T; tile += gridDim.x) {
        const TileOrigin o = tile_origin(t, tile);
        for (int sidx = threadIdx.x; sidx < t.TW * t.TH; sidx += blockDim.x) {
            const int wl = sidx % t.TW, yl = sidx / t.TW;
            const int W = o.W0 + wl, y = o.y0 + yl;
            if (W >= g.ng || y >= g.h) continue;
            int64_t i = (int64_t)y * g.SY + W;
            int lab = 0, prev = 1;
            for (int j = 0; j < g.K; j++, i += g.P) {
                const int32_t h = ld(&a.hgt[i]);
                const int in = a.dir == 1 ? (h < kInfH) : (h >= kInfH);
                bad |= in && !prev;
                lab += in;
                prev = in;
                const int32_t e = ld(&a.s.ex[i]);
                if (e < 0) deficit += (unsigned long long)(-(int64_t)e);
            }
            labels[(int64_t)y * g.ng + W] = lab;
        }
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_LABELS);
    const long long tot = block_sum((long long)deficit);
    const long long all = grid_sync_sum(ctrl, threadIdx.x == 0 ? tot : 0);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *flow = (int64_t)a.s.hdr->init_deficit - all;
        ctrl->stats[3] = passes;
        if (aborted(ctrl)) atomicCAS(status, GS_OK, GS_ERR_TIMEOUT);
    }
}

// copy the solve's device status into the caller's word unless it holds an error
__global__ void k_publish_status(Ctrl *ctrl, int32_t *status, int launches) {
    if (*status == GS_OK && ctrl->status != GS_OK) *status = ctrl->status;
    ctrl->stats[7] = launches;
}

// ------------------------------------------------------------ host side ---

// Tile shape: whole chains (all K layers), TW sites x TH rows.  The shared
// memory holds 9 int32 fields over the tile and a one-site halo; at most 8
// nodes per thread (4 preferred).  Wider tiles first (coalesced rows of 32
// sites), then the tallest that fits up to TH = 4.
static bool pick_tile(const Geom &g, TileGeom &t, int &npt, size_t &smem) {
    const size_t budget = 200 * 1024;
    // squarish in sites first: a breadth-first path crosses fewer tile borders
    static const int cand[][2] = {{16, 8}, {32, 4}, {16, 4}, {32, 2}, {16, 2}, {8, 4},
                                  {16, 1}, {8, 2},  {8, 1},  {4, 2},  {4, 1}};
    for (int pass = 0; pass < 2; pass++) {
        const int max_nodes = (pass == 0 ? 4 : 8) * kTileThreads;
        for (const auto &c : cand) {
            const int TW = c[0], TH = c[1];
            const int TN = TH * g.K * TW;
            const int PN = (TH + 2) * g.K * (TW + 2);
            const size_t bytes = 9 * (size_t)PN * sizeof(int32_t);
            if (TN > max_nodes || TN > kMaxTileNodes || bytes > budget) continue;
            t.TW = TW;
            t.TH = TH;
            t.PW = TW + 2;
            t.SJ = t.PW;
            t.SYs = g.K * t.PW;
            t.PN = PN;
            t.TN = TN;
            t.tiles_w = (g.ng + TW - 1) / TW;
            t.tiles_h = (g.h + TH - 1) / TH;
            t.T = t.tiles_w * t.tiles_h;
            npt = pass == 0 ? 4 : 8;
            smem = bytes;
            return true;
        }
    }
    return false;
}

size_t tiled_work_extra(const Geom &g) {
    TileGeom t;
    int npt;
    size_t smem;
    if (!pick_tile(g, t, npt, smem)) return 0;
    return round_up(g.N * sizeof(uint16_t), 256) + round_up(5 * (int64_t)t.T * sizeof(int32_t), 256);
}

static int setup_args(const Geom &g, const State &s, const Work &w, SolveArgs &a, int &npt,
                      size_t &smem) {
    a.g = g;
    a.s = s;
    if (!pick_tile(g, a.t, npt, smem)) return GS_ERR_INVAL;
    char *extra = (char *)w.mark + round_up(g.N * sizeof(int32_t), 256);
    a.amask = (uint16_t *)extra;
    a.tile_act = (int32_t *)(extra + round_up(g.N * sizeof(uint16_t), 256));
    a.tile_dirty = a.tile_act + 2 * a.t.T;
    a.tile_cnt = a.tile_act + 4 * a.t.T;
    a.log = w.mark;
    a.ctrl = w.ctrl;
    return GS_OK;
}

// Cooperative launch of kern with the whole grid resident.
template <class... Args>
static int launch_coop(void (*kern)(Args...), size_t smem, int T, cudaStream_t st, void **args) {
    int dev = 0;
    GS_CUDA_TRY(cudaGetDevice(&dev));
    int sms = 0, coop = 0;
    GS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    GS_CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop) return GS_ERR_CUDA;
    GS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    GS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, smem));
    if (per_sm < 1) return GS_ERR_INVAL;
    const int grid = std::min(per_sm * sms, T);
    GS_CUDA_TRY(cudaLaunchCooperativeKernel((void *)kern, grid, kTileThreads, args, smem, st));
    count_launches(1);
    return GS_OK;
}

int tiled_solve(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                int32_t *status, cudaStream_t st) {
    SolveArgs a;
    int npt;
    size_t smem;
    int rc = setup_args(g, s, w, a, npt, smem);
    if (rc) return rc;
    a.hgt = s.ht;
    a.dir = 0;
    a.mode = o->mode;
    a.sweeps_per_relabel = o->sweeps_per_relabel;
    a.local_iters = o->local_iters > 0 ? o->local_iters : 8;
    a.relabel_passes = o->relabel_passes > 0 ? o->relabel_passes : 4;
    a.tail_iters = o->tail_iters > 0 ? o->tail_iters : 4 * a.local_iters;
    a.fixed_sweeps = o->fixed_sweeps;
    a.max_iters = o->max_iters;
    GS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), st));
    void *args[] = {&a};
    rc = npt == 4 ? launch_coop(k_solve_tiled<4>, smem, a.t.T, st, args)
                  : launch_coop(k_solve_tiled<8>, smem, a.t.T, st, args);
    if (rc) return rc;
    k_publish_status<<<1, 1, 0, st>>>(w.ctrl, status, 2);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int tiled_extract(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                  int32_t *labels, int64_t *flow, int32_t *status, cudaStream_t st) {
    SolveArgs a;
    int npt;
    size_t smem;
    int rc = setup_args(g, s, w, a, npt, smem);
    if (rc) return rc;
    a.hgt = w.mark;
    a.dir = o->mode == GS_MODE_EXACT ? 1 : 0;
    // control words only: keep the solve's statistics, reset the barrier
    GS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, offsetof(Ctrl, stats), st));
    void *args[] = {&a, &labels, &flow, &status};
    rc = npt == 4 ? launch_coop(k_extract_tiled<4>, smem, a.t.T, st, args)
                  : launch_coop(k_extract_tiled<8>, smem, a.t.T, st, args);
    if (rc) return rc;
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // namespace gs

extern "C" int gs_tile_info(const gs_params *p, int32_t *out) {
    gs::Geom g;
    if (gs::make_geom(p, &g) != GS_OK || !out) return GS_ERR_INVAL;
    gs::TileGeom t;
    int npt;
    size_t smem;
    if (!gs::pick_tile(g, t, npt, smem)) return GS_ERR_INVAL;
    out[0] = t.TW;
    out[1] = t.TH;
    out[2] = t.T;
    out[3] = (int32_t)smem;
    return GS_OK;
}
