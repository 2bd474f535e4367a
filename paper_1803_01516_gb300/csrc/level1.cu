// Level-1 hierarchical approximation (§4.5): the delegate problem and the
// thin skin around its cut.  The second cut's graph is built in graph.cu
// (gs_build_graph_skin); both cuts run through the exact solver.
#include "gs_internal.cuh"

namespace gs {

// One thread per (delegate site, delegate depth number): the sum over the
// block's sites of the smallest data term in the depth bin.
__global__ void k_delegate_cost(const int32_t *__restrict__ C, int ng, int h, int D, int b,
                                int ngc, int hc, int Dc, int32_t *__restrict__ Cc,
                                int32_t *status) {
    int bad = 0, big = 0;
    const int64_t n = (int64_t)hc * ngc * Dc;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int Lc = (int)(idx % Dc);
        const int64_t site = idx / Dc;
        const int Wc = (int)(site % ngc), yc = (int)(site / ngc);
        const int l0 = Lc * b, l1 = min(D, l0 + b);
        long long sum = 0;
        for (int y = yc * b; y < min(h, yc * b + b); y++)
            for (int W = Wc * b; W < min(ng, Wc * b + b); W++) {
                const int32_t *cs = C + ((int64_t)y * ng + W) * D;
                int32_t m = cs[l0];
                for (int l = l0 + 1; l < l1; l++) m = min(m, cs[l]);
                bad |= m < 0;
                sum += m;
            }
        big |= sum > kCapLimit;
        Cc[idx] = (int32_t)max(0ll, min(sum, (long long)kCapLimit));
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_INVAL);
    }
    if (__syncthreads_or(big)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_OVERFLOW);
    }
}

// One thread per site: the skin [b L - b, b L + 2b - 1] of its delegate's label.
__global__ void k_skin_bounds(const int32_t *__restrict__ Xc, int ng, int h, int D, int b,
                              int ngc, int Dc, int32_t *__restrict__ lo, int32_t *__restrict__ hi,
                              int32_t *status) {
    int bad = 0;
    const int64_t n = (int64_t)ng * h;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(v % ng), y = (int)(v / ng);
        const int L = Xc[(int64_t)(y / b) * ngc + W / b];
        if (L < 0 || L >= Dc) {
            bad = 1;
            lo[v] = 0;
            hi[v] = D - 1;
            continue;
        }
        lo[v] = max(0, b * L - b);
        hi[v] = min(D - 1, b * L + 2 * b - 1);
    }
    if (__syncthreads_or(bad)) {
        if (threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_LABELS);
    }
}

static int grid_sites(int64_t n) { return grid_for(n, 16); }

}  // namespace gs

using namespace gs;

extern "C" int gs_delegate_params(const gs_params *p, int32_t b, gs_params *out) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !out || b < 1 || b >= p->D) return GS_ERR_INVAL;
    const int Dc = (p->D + b - 1) / b;
    const int ngc = (g.ng + b - 1) / b, hc = (p->h + b - 1) / b;
    const long long lam = (long long)p->lambda * b, inh = (long long)p->inhibit * b;
    if (lam > (1 << 28) || inh > (1 << 29)) return GS_ERR_OVERFLOW;
    gs_params q = *p;
    q.D = Dc;
    q.dis0 = 2 * (Dc - 1);
    q.w = ngc + q.dis0;
    q.h = hc;
    q.lambda = (int32_t)lam;
    q.inhibit = (int32_t)inh;
    *out = q;
    return GS_OK;
}

extern "C" int gs_delegate_cost(const int32_t *cost, const gs_params *p, int32_t b, int32_t *coarse,
                                int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !coarse || !status || b < 1 || b >= p->D)
        return GS_ERR_INVAL;
    const int Dc = (p->D + b - 1) / b;
    const int ngc = (g.ng + b - 1) / b, hc = (p->h + b - 1) / b;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int32_t), st));
    k_delegate_cost<<<grid_sites((int64_t)hc * ngc * Dc), 256, 0, st>>>(
        cost, g.ng, g.h, g.D, b, ngc, hc, Dc, coarse, status);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_skin_bounds(const int32_t *coarse_labels, const gs_params *p, int32_t b,
                              int32_t *lo, int32_t *hi, int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !coarse_labels || !lo || !hi || !status || b < 1 ||
        b >= p->D)
        return GS_ERR_INVAL;
    const int Dc = (p->D + b - 1) / b;
    const int ngc = (g.ng + b - 1) / b;
    cudaStream_t st = (cudaStream_t)stream;
    k_skin_bounds<<<grid_sites((int64_t)g.ng * g.h), 256, 0, st>>>(coarse_labels, g.ng, g.h, g.D,
                                                                   b, ngc, Dc, lo, hi, status);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
