// Graph construction (§3 / Fig. 4, terminals folded as in §4.4) and reading
// the cut back as labels (§3 "real cross points").
#include "arcs.cuh"

namespace gs {

__device__ __forceinline__ void block_sum_u64(unsigned long long v, unsigned long long *out) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __shared__ unsigned long long red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (wid == 0) {
        v = lane < (int)(blockDim.x >> 5) ? red[lane] : 0ull;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(out, v);
    }
}

__global__ void k_header(GraphHeader *hdr, Geom g, int inhibit, int vinhibit) {
    hdr->magic = kMagic;
    hdr->D = g.D;
    hdr->ng = g.ng;
    hdr->h = g.h;
    hdr->K = g.K;
    hdr->P = g.P;
    hdr->lam = g.lam;
    hdr->inhibit = inhibit;
    hdr->vinhibit = vinhibit;
    hdr->rev = 0;
    hdr->sum_first = 0;
    hdr->init_deficit = 0;
    hdr->src_total = 0;
    hdr->sum_last = 0;
    hdr->exact_heights = 0;
}

// Source capacity of each direction: sum of C(0) and of C(D-1).
__global__ void k_dir_sums(const int32_t *__restrict__ C, Geom g, GraphHeader *hdr) {
    unsigned long long a = 0, b = 0;
    const int64_t sites = (int64_t)g.ng * g.h;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < sites;
         v += (int64_t)gridDim.x * blockDim.x) {
        a += (unsigned long long)max(C[v * g.D], 0);
        b += (unsigned long long)max(C[v * g.D + g.D - 1], 0);
    }
    block_sum_u64(a, &hdr->sum_first);
    block_sum_u64(b, &hdr->sum_last);
}

__global__ void k_decide(GraphHeader *hdr, int direction) {
    hdr->rev = direction == 2 ? 1 : direction == 1 ? 0 : (hdr->sum_last < hdr->sum_first ? 1 : 0);
}

// One thread per node.  Chain node j = k-1 of site (W, y); its incoming data
// arc carries C(j) (from s when j = 0) and its outgoing one C(j+1) (to t when
// j = K-1).  The source arcs are folded in as excess and each chain starts
// with its own largest flow already pushed down it: node j receives
// F_j = min(C(0..j)) and forwards F_(j+1), so
//   ex = F_j - F_(j+1)  (j < K-1),   ex = F_(K-1) - C(D-1)  (j = K-1, negative
//                                     when sink capacity is left: a deficit)
//   rc = C(j+1) - F_(j+1)  residual of the outgoing data arc.
// This is a valid preflow (the flow of every chain taken alone, i.e. the cut
// with no interaction terms); the max-flow routes the rest.  Penalty residuals
// start at lambda (no flow) and inhibit residuals at h2.  Without the chain
// pre-pass (preflow = 0) only the source arcs are saturated: n_1 holds C(0),
// the last node's deficit is C(D-1), every data arc is unused.
__global__ void k_build(const int32_t *__restrict__ C, Geom g, State s, int32_t *status,
                        int preflow) {
    unsigned long long deficit = 0, src = 0;
    int bad = 0, big = 0;
    const bool rev = *(volatile int32_t *)&s.hdr->rev != 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const NodePos p = node_pos(g, i);
        if (p.W >= g.ng) {
            s.rc[i] = s.rr[i] = s.rd[i] = 0;
            s.ri0[i] = s.ri1[i] = s.ri2[i] = s.ri3[i] = 0;
            s.ex[i] = 0;
            s.ht[i] = kInfH;
            continue;
        }
        const int32_t *cs = C + ((int64_t)p.y * g.ng + p.W) * g.D;
        // cost of label l in the direction solved
        auto c = [&](int l) { return cs[rev ? g.D - 1 - l : l]; };
        int32_t F = c(0);                 // F_j
        bad |= F < 0;
        big |= F > kCapLimit;
        for (int q = 1; q <= p.j; q++) F = min(F, c(q));
        if (!preflow) F = p.j == 0 ? c(0) : 0;
        const int32_t cout = c(p.j + 1);  // outgoing arc capacity
        bad |= cout < 0;
        big |= cout > kCapLimit;
        int32_t e, rc;
        if (p.j < g.K - 1) {
            const int32_t F1 = preflow ? min(F, cout) : 0;
            e = F - F1;
            rc = cout - F1;
        } else {
            e = F - cout;
            rc = 0;
            deficit += (unsigned long long)max(cout, 0);
        }
        if (p.j == 0) src += (unsigned long long)max(c(0), 0);
        s.rc[i] = rc;
        s.ex[i] = e;
        s.rr[i] = (p.W < g.ng - 1) ? g.lam : 0;
        s.rd[i] = (p.y < g.h - 1) ? g.lam : 0;
        const bool dn = p.j > 0;
        s.ri0[i] = (dn && p.W > 0) ? g.h2h : 0;
        s.ri1[i] = (dn && p.W < g.ng - 1) ? g.h2h : 0;
        s.ri2[i] = (dn && p.y > 0) ? g.h2v : 0;
        s.ri3[i] = (dn && p.y < g.h - 1) ? g.h2v : 0;
        s.ht[i] = 0;
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_INVAL);
    }
    if (__syncthreads_or(big)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_OVERFLOW);
    }
    // flow value = (total sink capacity) - (sink capacity left at the end)
    block_sum_u64(deficit, &s.hdr->init_deficit);
    block_sum_u64(src, &s.hdr->src_total);
}

// Graph of the level-1 second cut (§4.5), one thread per node.  With bounds
// lo <= X <= hi a site's chain splits into nodes held on the source side
// (k <= lo), free nodes (lo < k <= hi) and nodes held on the sink side
// (k > hi).  Held nodes are contracted into the terminals: an arc from a
// source-held node into a free node is a source arc (saturated at once: its
// capacity is excess of the free node), an arc from a free node into a
// sink-held node is a sink arc (its capacity is a deficit), and arcs among
// held nodes are constants of the cut.  Residuals are set so that no
// capacity leaves the source-held region and none enters the sink-held one:
// source-held nodes can then never reach a deficit (their height stays
// infinite), sink-held nodes never receive flow, and only the free nodes
// carry the max-flow.  The free part of a chain is the chain of labels
// lo..hi (source arc C(lo), sink arc C(hi)) with the same chain-local
// preflow as k_build.  A source-held node keeps an excess of 1 so that label
// extraction finds it on the source side.
__device__ __forceinline__ int held(int lo, int hi, int k) { return k <= lo ? 0 : k > hi ? 2 : 1; }

__global__ void k_build_skin(const int32_t *__restrict__ C, const int32_t *__restrict__ lo,
                             const int32_t *__restrict__ hi, Geom g, State s, int32_t *status) {
    unsigned long long src = 0, snk = 0;
    int bad = 0, big = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const NodePos p = node_pos(g, i);
        if (p.W >= g.ng) {
            s.rc[i] = s.rr[i] = s.rd[i] = 0;
            s.ri0[i] = s.ri1[i] = s.ri2[i] = s.ri3[i] = 0;
            s.ex[i] = 0;
            s.ht[i] = kInfH;
            continue;
        }
        const int64_t v = (int64_t)p.y * g.ng + p.W;
        auto lo_of = [&](int64_t u) {
            const int a = lo[u], b = hi[u];
            return (a < 0 || a > b || b > g.D - 1) ? 0 : a;
        };
        auto hi_of = [&](int64_t u) {
            const int a = lo[u], b = hi[u];
            return (a < 0 || a > b || b > g.D - 1) ? g.D - 1 : b;
        };
        bad |= lo[v] < 0 || lo[v] > hi[v] || hi[v] > g.D - 1;
        const int a = lo_of(v), b = hi_of(v);
        const int k = p.j + 1;
        const int me = held(a, b, k);
        const int32_t *cs = C + v * g.D;
        // neighbours: W-1, W+1, y-1, y+1 (the inhibit directions ri0..ri3)
        const bool has[4] = {p.W > 0, p.W < g.ng - 1, p.y > 0, p.y < g.h - 1};
        const int64_t nb[4] = {v - 1, v + 1, v - g.ng, v + g.ng};
        const int32_t h2[4] = {g.h2h, g.h2h, g.h2v, g.h2v};
        int nlo[4], nhi[4];
        for (int q = 0; q < 4; q++) {
            nlo[q] = has[q] ? lo_of(nb[q]) : 0;
            nhi[q] = has[q] ? hi_of(nb[q]) : g.D - 1;
        }
        // data arc n_k -> n_(k+1) and the chain-local preflow of the free part
        long long ex = 0;
        int32_t rc = 0;
        if (me == 1) {
            int32_t F = cs[a];
            for (int l = a + 1; l < k; l++) F = min(F, cs[l]);
            if (k == a + 1) src += (unsigned long long)max(cs[a], 0);
            if (k < b) {
                const int32_t F1 = min(F, cs[k]);
                ex = (long long)F - F1;
                rc = cs[k] - F1;
            } else {
                ex = (long long)F - cs[b];
                snk += (unsigned long long)max(cs[b], 0);
            }
            for (int q = 0; q < 4; q++) {
                if (!has[q]) continue;
                const int hp = held(nlo[q], nhi[q], k);
                if (hp == 0) { ex += g.lam; src += g.lam; }               // source-held -> me
                if (hp == 2) { ex -= g.lam; snk += g.lam; }               // me -> sink-held
                if (k + 1 <= g.D - 1 && held(nlo[q], nhi[q], k + 1) == 0) {
                    ex += h2[q];                                          // inhibit into me
                    src += h2[q];
                }
                if (k >= 2 && held(nlo[q], nhi[q], k - 1) == 2) {
                    ex -= h2[q];                                          // inhibit out of me
                    snk += h2[q];
                }
            }
        } else if (me == 0) {
            ex = 1;
        }
        big |= ex > kCapLimit || ex < -(long long)kCapLimit;
        for (int l = 0; l < g.D; l++) bad |= cs[l] < 0;
        // penalty pairs stored at this node: right (rr) and down (rd); the value
        // is the residual of this node -> neighbour, the reverse is 2 lambda - r
        auto pair_res = [&](int su, int sv) -> int32_t {
            if (su == 1 && sv == 1) return g.lam;
            if ((su == 0 && sv != 0) || (su == 1 && sv == 2)) return 0;       // leaves S / enters T
            if ((su == 1 && sv == 0) || (su == 2 && sv != 2)) return g.lam2;  // the reverse does
            return g.lam;                                                     // both held alike
        };
        s.rc[i] = p.j < g.K - 1 ? rc : 0;
        s.rr[i] = has[1] ? pair_res(me, held(nlo[1], nhi[1], k)) : 0;
        s.rd[i] = has[3] ? pair_res(me, held(nlo[3], nhi[3], k)) : 0;
        int32_t ri[4];
        for (int q = 0; q < 4; q++) {
            ri[q] = 0;
            if (p.j == 0 || !has[q]) continue;
            const int hh = held(nlo[q], nhi[q], k - 1);
            // source-held tail into a free or sink-held head, free tail into a
            // sink-held head: folded into the terminals, no residual
            ri[q] = ((me == 0 && hh != 0) || (me == 1 && hh == 2)) ? 0 : h2[q];
        }
        s.ri0[i] = ri[0];
        s.ri1[i] = ri[1];
        s.ri2[i] = ri[2];
        s.ri3[i] = ri[3];
        s.ex[i] = (int32_t)max(min(ex, (long long)kCapLimit), -(long long)kCapLimit);
        s.ht[i] = 0;
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_INVAL);
    }
    if (__syncthreads_or(big)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_OVERFLOW);
    }
    block_sum_u64(snk, &s.hdr->init_deficit);
    block_sum_u64(src, &s.hdr->src_total);
}

__global__ void k_check_totals(const GraphHeader *hdr, int32_t *status) {
    if (hdr->src_total > (unsigned long long)kCapLimit ||
        hdr->init_deficit > (unsigned long long)kCapLimit)
        atomicCAS(status, GS_OK, GS_ERR_OVERFLOW);
}

// ---------------------------------------------------------------- labels ---

// S_min seed: nodes with positive excess.
__global__ void k_mark_init(Geom g, State s, int32_t *mark) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(i % g.P);
        mark[i] = (W < g.ng && s.ex[i] > 0) ? 1 : 0;
    }
}

// One pass of forward reachability: a marked node marks every head of a
// residual arc.  Writes are idempotent, so passes need no atomics.
__global__ void k_mark_pass(Geom g, State s, int32_t *mark, Ctrl *ctrl) {
    int changed = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (!mark[i]) continue;
        const NodePos p = node_pos(g, i);
        if (p.W >= g.ng) continue;
        int32_t r[kSlots];
        load_residuals(s, g, i, p, r);
#pragma unroll
        for (int q = 0; q < kSlots; q++) {
            if (r[q] > 0) {
                const int64_t v = i + slot_offset(g, q);
                if (!mark[v]) {
                    mark[v] = 1;
                    changed = 1;
                }
            }
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicExch(&ctrl->changed, 1);
}

// labels[y][W] = number of source-side nodes of the chain; the source side
// must be a prefix of the chain (mode 0: mark != 0, mode 1: ht == inf).
__global__ void k_labels(Geom g, State s, const int32_t *mark, int use_heights, int32_t *labels,
                         int32_t *status) {
    const int64_t sites = (int64_t)g.ng * g.h;
    int bad = 0;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < sites;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(v % g.ng), y = (int)(v / g.ng);
        int64_t i = (int64_t)y * g.SY + W;
        int a = 0, prev = 1;
        for (int j = 0; j < g.K; j++, i += g.P) {
            const int in = use_heights ? (s.ht[i] >= kInfH) : (mark[i] != 0);
            bad |= in && !prev;
            a += in;
            prev = in;
        }
        labels[v] = a;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_LABELS);
}

__global__ void k_flip_labels(int32_t *labels, int64_t n, int D) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x)
        labels[v] = D - 1 - labels[v];
}

__global__ void k_deficit(Geom g, State s, unsigned long long *out) {
    unsigned long long d = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = s.ex[i];
        if (e < 0) d += (unsigned long long)(-(int64_t)e);
    }
    block_sum_u64(d, out);
}

__global__ void k_flow(const GraphHeader *hdr, const Ctrl *ctrl, int64_t *flow) {
    *flow = (int64_t)hdr->init_deficit - (int64_t)ctrl->deficit_left;
}

}  // namespace gs

using namespace gs;


// Shared with solve.cu: run the global relabel to convergence (defined there).
namespace gs {
int global_relabel(const Geom &g, const State &s, const Work &w, cudaStream_t st, int64_t *passes);
}

extern "C" {

int gs_build_graph(const int32_t *cost, const gs_params *p, void *graph, int32_t *status,
                   void *stream) {
    return gs_build_graph_flags(cost, p, GS_BUILD_CHAIN_PREFLOW, graph, status, stream);
}

int gs_build_graph_flags(const int32_t *cost, const gs_params *p, int32_t flags, void *graph,
                         int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !graph || !status) return GS_ERR_INVAL;
    if (flags & ~GS_BUILD_CHAIN_PREFLOW) return GS_ERR_INVAL;
    if (((uintptr_t)graph & 255) != 0) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    State s = state_view(graph, g);
    GS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    k_header<<<1, 1, 0, st>>>(s.hdr, g, p->inhibit, p->vertical_inhibit);
    k_dir_sums<<<grid_for((int64_t)g.ng * g.h), 256, 0, st>>>(cost, g, s.hdr);
    k_decide<<<1, 1, 0, st>>>(s.hdr, p->direction);
    k_build<<<grid_for(g.N), 256, 0, st>>>(cost, g, s, status, flags & GS_BUILD_CHAIN_PREFLOW);
    k_check_totals<<<1, 1, 0, st>>>(s.hdr, status);
    count_launches(5);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_build_graph_skin(const int32_t *cost, const gs_params *p, const int32_t *lo,
                        const int32_t *hi, void *graph, int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !lo || !hi || !graph || !status)
        return GS_ERR_INVAL;
    if (((uintptr_t)graph & 255) != 0) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    State s = state_view(graph, g);
    GS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    k_header<<<1, 1, 0, st>>>(s.hdr, g, p->inhibit, p->vertical_inhibit);
    k_decide<<<1, 1, 0, st>>>(s.hdr, 1);
    k_build_skin<<<grid_for(g.N), 256, 0, st>>>(cost, lo, hi, g, s, status);
    k_check_totals<<<1, 1, 0, st>>>(s.hdr, status);
    count_launches(4);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_extract_labels(void *graph, const gs_params *p, const gs_solve_opts *o, void *workspace,
                      int32_t *labels, int64_t *flow, int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !o || !graph || !workspace || !labels || !flow || !status)
        return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    State s = state_view(graph, g);
    Work w = work_view(workspace, g);
    if (o->engine == GS_ENGINE_TILED) return tiled_extract(g, s, w, o, labels, flow, status, st);
    const int grid = grid_for(g.N);
    int32_t rev = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&rev, &s.hdr->rev, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    if (o->mode == GS_MODE_EXACT && !rev) {
        k_mark_init<<<grid, 256, 0, st>>>(g, s, w.mark);
        count_launches(1);
        int64_t passes = 0;
        for (;;) {
            GS_CUDA_TRY(cudaMemsetAsync(&w.ctrl->changed, 0, sizeof(int32_t), st));
            k_mark_pass<<<grid, 256, 0, st>>>(g, s, w.mark, w.ctrl);
            count_launches(1);
            int32_t changed = 0;
            GS_CUDA_TRY(cudaMemcpyAsync(&changed, &w.ctrl->changed, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, st));
            GS_CUDA_TRY(cudaStreamSynchronize(st));
            passes++;
            if (!changed) break;
        }
        long long lp = passes;
        GS_CUDA_TRY(cudaMemcpyAsync(&w.ctrl->stats[3], &lp, sizeof(long long),
                                    cudaMemcpyHostToDevice, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        k_labels<<<grid_for((int64_t)g.ng * g.h), 256, 0, st>>>(g, s, w.mark, 0, labels, status);
        count_launches(1);
    } else {
        int64_t passes = 0;
        int rc = global_relabel(g, s, w, st, &passes);
        if (rc) return rc;
        // the largest minimiser of the solved direction (nodes that cannot
        // reach sink capacity); for a label-reversed state it maps back to the
        // smallest minimiser of the original problem
        k_labels<<<grid_for((int64_t)g.ng * g.h), 256, 0, st>>>(g, s, w.mark, 1, labels, status);
        count_launches(1);
        if (rev) {
            k_flip_labels<<<grid_for((int64_t)g.ng * g.h), 256, 0, st>>>(labels, (int64_t)g.ng * g.h,
                                                                      g.D);
            count_launches(1);
        }
    }
    GS_CUDA_TRY(cudaMemsetAsync(&w.ctrl->deficit_left, 0, sizeof(unsigned long long), st));
    k_deficit<<<grid, 256, 0, st>>>(g, s, &w.ctrl->deficit_left);
    k_flow<<<1, 1, 0, st>>>(s.hdr, w.ctrl, flow);
    count_launches(3);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_solve_stats(const void *workspace, int64_t *host_stats, void *stream) {
    if (!workspace || !host_stats) return GS_ERR_INVAL;
    const Ctrl *c = (const Ctrl *)workspace;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemcpyAsync(host_stats, c->stats, 8 * sizeof(long long),
                                cudaMemcpyDeviceToHost, st));
    GS_CUDA_TRY(cudaMemcpyAsync(host_stats + 8, &c->visits_sweep, 2 * sizeof(long long),
                                cudaMemcpyDeviceToHost, st));
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    return GS_OK;
}

}  // extern "C"
