// Level-2 approximation (§4.5): after the level-1 delegate cut and thin skin,
// every b x b block of sites is cut exactly on its own, the pairs that leave
// the block taken against the neighbours' current labels, blocks updated in a
// two-colour order (see gs_block_descent in gazecut.h).
//
// A block problem is tiny (b <= 3: at most 3 x 3 sites, at most 3b labels in
// the skin), so one warp solves it exactly by min-sum dynamic programming over
// the block's rows: a row state is the labels of the row's sites (n^bw states
// for n labels), the row cost holds the sites' data and border terms and the
// pairs inside the row, and the pairs between consecutive rows -- a sum over
// the columns -- are applied one column at a time (a min-plus transform of one
// label digit), so moving from row to row costs bw * n^(bw+1) operations
// instead of n^(2 bw).  Forward and backward passes give every row state's
// min-marginal; the smallest label a site takes in any minimiser, read from
// the states whose min-marginal equals the minimum, is the site's label in the
// component-wise smallest minimiser (the minimisers of this convex-prior
// energy form a lattice under component-wise min), the same canonical answer
// as the minimal source set of the block's cut.
#include "gs_internal.cuh"

namespace gs {

constexpr int kL2Warps = 4;                       // warps (blocks in flight) per CTA
constexpr long long kL2Inf = 1ll << 50;           // data term outside a site's bounds

__device__ __forceinline__ long long htil(int d, long long lam, long long inh) {
    const long long a = d < 0 ? -d : d;
    return lam * a + (a > 1 ? inh * (a - 1) : 0);
}

struct L2Args {
    const int32_t *cost;    // [h][n_g][D]
    const int32_t *lo, *hi; // [h][n_g]
    int32_t *labels;        // [h][n_g], updated in place for the blocks of one colour
    int32_t *status;
    int ng, h, D, b, colour, nbx, nby, scap;
    long long lam, h2h, h2v;
};

// Min-plus transform of label digit c of every row state: out(s) = min over d
// of in(s with digit c = d) + h~_v(d - digit_c(s)).
__device__ __forceinline__ void col_transform(const long long *in, long long *out, int S, int n,
                                              int pw, long long lam, long long inh, int lane) {
    for (int s = lane; s < S; s += 32) {
        const int dc = (s / pw) % n;
        const int base = s - dc * pw;
        long long best = kL2Inf * 64;
        for (int d = 0; d < n; d++) best = min(best, in[base + d * pw] + htil(d - dc, lam, inh));
        out[s] = best;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * kL2Warps) k_block_descent(const L2Args a) {
    extern __shared__ long long l2sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S_cap = a.scap;
    long long *F = l2sm + (size_t)warp * (6 * S_cap + 96);   // F[3][S_cap]
    long long *Bk = F + 3 * S_cap;
    long long *A = Bk + S_cap;
    long long *Bb = A + S_cap;
    long long *U = Bb + S_cap;                                 // [bh][bw][n], at most 96
    const int nblocks = a.nbx * a.nby;
    for (int k = blockIdx.x * kL2Warps + warp; k < nblocks; k += gridDim.x * kL2Warps) {
        const int bx = k % a.nbx, by = k / a.nbx;
        if (((bx + by) & 1) != a.colour) continue;
        const int y0 = by * a.b, W0 = bx * a.b;
        const int bh = min(a.b, a.h - y0), bw = min(a.b, a.ng - W0);
        // the block's label range: the union of its sites' bounds
        int LO = a.D, HI = -1, bad = 0;
        for (int t = lane; t < bh * bw; t += 32) {
            const int64_t v = (int64_t)(y0 + t / bw) * a.ng + W0 + t % bw;
            const int l = a.lo[v], u = a.hi[v];
            bad |= l < 0 || l > u || u > a.D - 1;
            LO = min(LO, l);
            HI = max(HI, u);
        }
        for (int o = 16; o > 0; o >>= 1) {
            LO = min(LO, __shfl_xor_sync(0xffffffffu, LO, o));
            HI = max(HI, __shfl_xor_sync(0xffffffffu, HI, o));
            bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        }
        const int n = HI - LO + 1;
        int S = 1;
        for (int c = 0; c < bw && !bad; c++) {
            if (S > S_cap / max(n, 1)) bad = 1;
            S *= n;
        }
        if (bad || n < 1 || bh * bw * n > 96) {
            if (lane == 0) atomicCAS(a.status, GS_OK, GS_ERR_INVAL);
            continue;
        }
        // unary terms: data term inside the site's bounds, plus the pairs to
        // sites outside the block against their current labels
        for (int t = lane; t < bh * bw * n; t += 32) {
            const int kk = t % n, c = (t / n) % bw, r = t / (n * bw);
            const int y = y0 + r, W = W0 + c, l = LO + kk;
            const int64_t v = (int64_t)y * a.ng + W;
            long long u;
            if (l < a.lo[v] || l > a.hi[v]) {
                u = kL2Inf;
            } else {
                u = a.cost[v * a.D + l];
                if (W == W0 && W > 0) u += htil(l - a.labels[v - 1], a.lam, a.h2h);
                if (W == W0 + bw - 1 && W < a.ng - 1) u += htil(l - a.labels[v + 1], a.lam, a.h2h);
                if (y == y0 && y > 0) u += htil(l - a.labels[v - a.ng], a.lam, a.h2v);
                if (y == y0 + bh - 1 && y < a.h - 1) u += htil(l - a.labels[v + a.ng], a.lam, a.h2v);
            }
            U[t] = u;
        }
        __syncwarp();
        // row cost of state s in row r (data, border terms, pairs inside the row)
        auto row_cost = [&](int r, int s) {
            long long acc = 0;
            int prev = -1;
            for (int c = 0; c < bw; c++) {
                const int d = s % n;
                s /= n;
                acc += U[(r * bw + c) * n + d];
                if (c > 0) acc += htil(prev - d, a.lam, a.h2h);
                prev = d;
            }
            return acc;
        };
        // forward
        for (int s = lane; s < S; s += 32) F[s] = row_cost(0, s);
        __syncwarp();
        for (int r = 1; r < bh; r++) {
            const long long *src = F + (r - 1) * S_cap;
            long long *bufs[2] = {A, Bb};
            int pw = 1;
            for (int c = 0; c < bw; c++, pw *= n) {
                col_transform(c == 0 ? src : bufs[(c - 1) & 1], bufs[c & 1], S, n, pw, a.lam, a.h2v,
                              lane);
            }
            const long long *G = bufs[(bw - 1) & 1];
            for (int s = lane; s < S; s += 32) F[r * S_cap + s] = row_cost(r, s) + G[s];
            __syncwarp();
        }
        // minimum energy of the block problem
        long long Emin = kL2Inf * 64;
        for (int s = lane; s < S; s += 32) Emin = min(Emin, F[(bh - 1) * S_cap + s]);
        for (int o = 16; o > 0; o >>= 1) Emin = min(Emin, __shfl_xor_sync(0xffffffffu, Emin, o));
        // backward, with the smallest label of every site among the minimisers
        for (int s = lane; s < S; s += 32) Bk[s] = 0;
        __syncwarp();
        for (int r = bh - 1; r >= 0; r--) {
            if (r < bh - 1) {
                // Bk_r(s) = min over s' of V(s, s') + R_(r+1)(s') + Bk_(r+1)(s')
                for (int s = lane; s < S; s += 32) A[s] = row_cost(r + 1, s) + Bk[s];
                __syncwarp();
                long long *bufs[2] = {Bb, A};
                int pw = 1;
                for (int c = 0; c < bw; c++, pw *= n) {
                    col_transform(c == 0 ? A : bufs[(c - 1) & 1], bufs[c & 1], S, n, pw, a.lam,
                                  a.h2v, lane);
                }
                const long long *G = bufs[(bw - 1) & 1];
                for (int s = lane; s < S; s += 32) Bk[s] = G[s];
                __syncwarp();
            }
            for (int c = 0; c < bw; c++) {
                int best = n;
                int pw = 1;
                for (int q = 0; q < c; q++) pw *= n;
                for (int s = lane; s < S; s += 32)
                    if (F[r * S_cap + s] + Bk[s] == Emin) best = min(best, (s / pw) % n);
                for (int o = 16; o > 0; o >>= 1)
                    best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
                if (lane == 0) {
                    const int64_t v = (int64_t)(y0 + r) * a.ng + W0 + c;
                    if (best < n) a.labels[v] = LO + best;
                    else atomicCAS(a.status, GS_OK, GS_ERR_LABELS);
                }
            }
            __syncwarp();
        }
    }
}

// Start labels: each site's first argmin of the data term inside its
// delegate's depth bin [b Xc, min(b Xc + b, D) - 1].
__global__ void k_level2_start(const int32_t *__restrict__ cost, const int32_t *__restrict__ Xc,
                               int ng, int h, int D, int b, int ngc, int Dc,
                               int32_t *__restrict__ labels, int32_t *status) {
    int bad = 0;
    const int64_t sites = (int64_t)ng * h;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < sites;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int W = (int)(v % ng), y = (int)(v / ng);
        const int Lc = Xc[(int64_t)(y / b) * ngc + W / b];
        if (Lc < 0 || Lc >= Dc) {
            bad = 1;
            labels[v] = 0;
            continue;
        }
        const int a0 = b * Lc, z = min(a0 + b, D);
        int best = a0;
        int32_t bc = cost[v * D + a0];
        for (int l = a0 + 1; l < z; l++) {
            const int32_t c = cost[v * D + l];
            if (c < bc) {
                bc = c;
                best = l;
            }
        }
        labels[v] = best;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, GS_OK, GS_ERR_LABELS);
}

// Row states a block of b x b sites may need: (labels of the skin)^b.
static int state_cap(int b, int D) {
    const int n = std::min(3 * b, D);
    int S = 1;
    for (int c = 0; c < b; c++) S *= n;
    return S;
}

}  // namespace gs

using namespace gs;

extern "C" int gs_level2_start(const int32_t *cost, const gs_params *p, int32_t b,
                               const int32_t *coarse_labels, int32_t *labels, int32_t *status,
                               void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !coarse_labels || !labels || !status)
        return GS_ERR_INVAL;
    if (b < 1 || b >= g.D) return GS_ERR_INVAL;
    const int ngc = (g.ng + b - 1) / b, Dc = (g.D + b - 1) / b;
    const int64_t sites = (int64_t)g.ng * g.h;
    k_level2_start<<<grid_for(sites, 16), 256, 0, (cudaStream_t)stream>>>(
        cost, coarse_labels, g.ng, g.h, g.D, b, ngc, Dc, labels, status);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

extern "C" int gs_block_descent(const int32_t *cost, const gs_params *p, int32_t b,
                                const int32_t *lo, const int32_t *hi, int32_t *labels,
                                int32_t passes, int32_t *status, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !lo || !hi || !labels || !status)
        return GS_ERR_INVAL;
    if (b < 1 || b > 3 || passes < 0) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    L2Args a;
    a.cost = cost;
    a.lo = lo;
    a.hi = hi;
    a.labels = labels;
    a.status = status;
    a.ng = g.ng;
    a.h = g.h;
    a.D = g.D;
    a.b = b;
    a.nbx = (g.ng + b - 1) / b;
    a.nby = (g.h + b - 1) / b;
    a.scap = state_cap(b, g.D);
    a.lam = g.lam;
    a.h2h = g.h2h;
    a.h2v = g.h2v;
    const size_t smem = (size_t)kL2Warps * (6 * a.scap + 96) * sizeof(long long);
    GS_CUDA_TRY(cudaFuncSetAttribute(k_block_descent, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    const int64_t half = ((int64_t)a.nbx * a.nby + 1) / 2;
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>((half + kL2Warps - 1) / kL2Warps, 4 * (int64_t)device_sms()));
    for (int it = 0; it < passes; it++) {
        for (int colour = 0; colour < 2; colour++) {
            a.colour = colour;
            k_block_descent<<<grid, 32 * kL2Warps, smem, st>>>(a);
            count_launches(1);
        }
    }
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
