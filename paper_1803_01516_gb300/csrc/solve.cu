// Push-relabel max-flow with global relabelling (§4.4) on the chain graph.
#include "arcs.cuh"

namespace gs {

// ------------------------------------------------------- global relabel ---
// Heights become breadth-first distances, over residual arcs, to the nodes
// that still have sink capacity (negative excess); nodes that cannot reach
// one get kInfH.  Computed as a monotone relaxation
//     h(u) <- min(h(u), 1 + min_{residual (u,v)} h(v))
// from h = 0 on deficit nodes and kInfH elsewhere.  Every value stays an upper
// bound of the true distance, so any order of updates converges to the exact
// distances; a full pass without a change ends the loop.

__global__ void k_gr_init(Geom g, State s) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(i % g.P);
        s.ht[i] = (W < g.ng && s.ex[i] < 0) ? 0 : kInfH;
    }
}

__global__ void k_gr_relax(Geom g, State s, Ctrl *ctrl) {
    int changed = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const NodePos p = node_pos(g, i);
        if (p.W >= g.ng) continue;
        const int32_t hu = s.ht[i];
        if (hu == 0) continue;
        int32_t r[kSlots];
        load_residuals(s, g, i, p, r);
        int32_t hmin = kInfH;
#pragma unroll
        for (int q = 0; q < kSlots; q++)
            if (r[q] > 0) hmin = min(hmin, s.ht[i + slot_offset(g, q)]);
        if (hmin < kInfH && hmin + 1 < hu) {
            s.ht[i] = hmin + 1;
            changed = 1;
        }
    }
    if (__syncthreads_or(changed) && threadIdx.x == 0) atomicExch(&ctrl->changed, 1);
}

// Active nodes: positive excess and a finite height.
__global__ void k_count_active(Geom g, State s, Ctrl *ctrl) {
    int cnt = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(i % g.P);
        cnt += (W < g.ng && s.ex[i] > 0 && s.ht[i] < kInfH);
    }
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&ctrl->active, cnt);
}

// ---------------------------------------------------------------- sweep ---
// One discharge of every active node, concurrently and lock-free: push
// min(excess, residual) along every residual arc to a lower neighbour, then,
// if excess is left, relabel to one above the lowest residual neighbour.
// Pushes keep the state a valid preflow under any interleaving: only the owner
// lowers its excess and only the tail of an arc consumes its residual, while
// concurrent updates from other nodes can only add.  Heights read from
// neighbours may be stale; they only steer the pushes, and exactness is
// decided by the global relabel.
__global__ void k_sweep(Geom g, State s, Ctrl *ctrl) {
    int overflow = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.N;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = s.ex[i];
        if (e <= 0) continue;
        const int32_t hu = s.ht[i];
        if (hu >= kInfH) continue;
        const NodePos p = node_pos(g, i);
        if (p.W >= g.ng) continue;
        int32_t r[kSlots], hv[kSlots];
        load_residuals(s, g, i, p, r);
#pragma unroll
        for (int q = 0; q < kSlots; q++) hv[q] = r[q] > 0 ? s.ht[i + slot_offset(g, q)] : kInfH;
        int32_t left = e;
#pragma unroll
        for (int q = 0; q < kSlots; q++) {
            if (left > 0 && r[q] > 0 && hv[q] < hu) {
                const int32_t d = min(left, r[q]);
                const int32_t grown = push_residual(s, g, i, q, d);
                overflow |= grown > kCapLimit;
                const int32_t ev = atomicAdd(&s.ex[i + slot_offset(g, q)], d) + d;
                overflow |= ev > kCapLimit;
                r[q] -= d;
                left -= d;
            }
        }
        if (left != e) atomicSub(&s.ex[i], e - left);
        if (left > 0) {
            int32_t hmin = kInfH;
#pragma unroll
            for (int q = 0; q < kSlots; q++)
                if (r[q] > 0) hmin = min(hmin, hv[q]);
            s.ht[i] = hmin >= kInfH - 1 ? kInfH : hmin + 1;
        }
    }
    if (__syncthreads_or(overflow) && threadIdx.x == 0) atomicCAS(&ctrl->status, GS_OK, GS_ERR_OVERFLOW);
}

__global__ void k_add_stat(Ctrl *ctrl, int which, long long v) { ctrl->stats[which] += v; }


int global_relabel(const Geom &g, const State &s, const Work &w, cudaStream_t st, int64_t *passes) {
    const int grid = grid_for(g.N);
    k_gr_init<<<grid, 256, 0, st>>>(g, s);
    count_launches(1);
    for (;;) {
        GS_CUDA_TRY(cudaMemsetAsync(&w.ctrl->changed, 0, sizeof(int32_t), st));
        k_gr_relax<<<grid, 256, 0, st>>>(g, s, w.ctrl);
        count_launches(1);
        int32_t changed = 0;
        GS_CUDA_TRY(cudaMemcpyAsync(&changed, &w.ctrl->changed, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        (*passes)++;
        if (!changed) break;
    }
    return GS_OK;
}

// Event pair that times one phase on the solve's stream.
struct PhaseTimer {
    cudaEvent_t a = nullptr, b = nullptr;
    double ms = 0;
    bool pending = false;
    PhaseTimer() {
        cudaEventCreate(&a);
        cudaEventCreate(&b);
    }
    ~PhaseTimer() {
        cudaEventDestroy(a);
        cudaEventDestroy(b);
    }
    void start(cudaStream_t st) { cudaEventRecord(a, st); }
    void stop(cudaStream_t st) {
        cudaEventRecord(b, st);
        pending = true;
    }
    // call after the stream has been synchronised
    void collect() {
        if (!pending) return;
        float t = 0;
        if (cudaEventElapsedTime(&t, a, b) == cudaSuccess) ms += t;
        pending = false;
    }
};

}  // namespace gs

using namespace gs;

extern "C" int gs_check_solve_opts(const gs_solve_opts *o) {
    if (!o) return GS_ERR_INVAL;
    if (o->sweeps_per_relabel < 1 || o->max_iters < 1) return GS_ERR_INVAL;
    if (o->engine != GS_ENGINE_TILED && o->engine != GS_ENGINE_SIMPLE) return GS_ERR_INVAL;
    if (o->local_iters < 0 || o->relabel_passes < 0 || o->tail_iters < 0 || o->idle_limit_us < 0)
        return GS_ERR_INVAL;
    if (o->mode != GS_MODE_EXACT && o->mode != GS_MODE_FIXED_SWEEPS) return GS_ERR_INVAL;
    if (o->mode == GS_MODE_FIXED_SWEEPS && o->fixed_sweeps < 0) return GS_ERR_INVAL;
    if (o->cta_threads != 0 && o->cta_threads != 256 && o->cta_threads != 512) return GS_ERR_INVAL;
    return GS_OK;
}

extern "C" int gs_maxflow_solve(void *graph, const gs_params *p, const gs_solve_opts *o,
                                void *workspace, int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !o || !graph || !workspace || !status) return GS_ERR_INVAL;
    if (gs_check_solve_opts(o) != GS_OK) return GS_ERR_INVAL;
    if (((uintptr_t)workspace & 255) != 0) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    State s = state_view(graph, g);
    Work w = work_view(workspace, g);
    if (o->engine == GS_ENGINE_TILED) return tiled_solve(g, s, w, o, status, st);
    // this engine leaves no exact-height mark for the extraction to reuse
    GS_CUDA_TRY(cudaMemsetAsync(&s.hdr->exact_heights, 0, sizeof(int32_t), st));
    const int grid = grid_for(g.N);
    GS_CUDA_TRY(cudaMemsetAsync(w.ctrl, 0, sizeof(Ctrl), st));
    PhaseTimer t_sweep, t_relabel;
    const long long launches0 = gs_kernel_launches();
    int64_t relabels = 0, sweeps = 0, passes = 0, active = 0;
    bool done = false;
    for (int64_t it = 0; !done; it++) {
        if (o->mode == GS_MODE_EXACT && it >= o->max_iters) break;
        t_relabel.start(st);
        int rc = global_relabel(g, s, w, st, &passes);
        if (rc) return rc;
        t_relabel.stop(st);
        t_sweep.collect();
        relabels++;
        GS_CUDA_TRY(cudaMemsetAsync(&w.ctrl->active, 0, sizeof(int32_t), st));
        k_count_active<<<grid, 256, 0, st>>>(g, s, w.ctrl);
        count_launches(1);
        int32_t act = 0;
        GS_CUDA_TRY(cudaMemcpyAsync(&act, &w.ctrl->active, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost, st));
        GS_CUDA_TRY(cudaStreamSynchronize(st));
        t_relabel.collect();
        active = act;
        if (act == 0) { done = true; break; }
        int n = o->sweeps_per_relabel;
        if (o->mode == GS_MODE_FIXED_SWEEPS) {
            n = (int)std::min<int64_t>(n, o->fixed_sweeps - sweeps);
            if (n <= 0) { done = true; break; }
        }
        t_sweep.start(st);
        for (int k = 0; k < n; k++) k_sweep<<<grid, 256, 0, st>>>(g, s, w.ctrl);
        count_launches(n);
        t_sweep.stop(st);
        sweeps += n;
    }
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    t_sweep.collect();
    t_relabel.collect();
    long long stats[8] = {relabels, sweeps, passes, 0, active,
                          (long long)(t_sweep.ms * 1e6), (long long)(t_relabel.ms * 1e6),
                          gs_kernel_launches() - launches0};
    GS_CUDA_TRY(cudaMemcpyAsync(w.ctrl->stats, stats, sizeof(stats), cudaMemcpyHostToDevice, st));
    // status: keep an earlier error; else overflow seen by a sweep, else timeout
    int32_t dev = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&dev, &w.ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    int32_t mine = dev != GS_OK ? dev : (!done && o->mode == GS_MODE_EXACT ? GS_ERR_TIMEOUT : GS_OK);
    int32_t prev = 0;
    GS_CUDA_TRY(cudaMemcpyAsync(&prev, status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    if (prev == GS_OK && mine != GS_OK)
        GS_CUDA_TRY(cudaMemcpyAsync(status, &mine, sizeof(int32_t), cudaMemcpyHostToDevice, st));
    GS_CUDA_TRY(cudaStreamSynchronize(st));
    return GS_OK;
}
