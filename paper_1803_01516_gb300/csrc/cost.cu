// Data term (§4.3), energy (§2) and the size queries of the C ABI.
#include "gs_internal.cuh"

#include <atomic>

namespace gs {

static std::atomic<long long> g_launches{0};
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

int make_geom(const gs_params *p, Geom *g) {
    if (!p) return GS_ERR_INVAL;
    if (p->w < 1 || p->h < 1 || p->D < 2) return GS_ERR_INVAL;
    if (p->dis0 < 2 * (p->D - 1) || p->w - p->dis0 < 1) return GS_ERR_INVAL;
    if (p->lambda < 0 || p->lambda > (1 << 28)) return GS_ERR_INVAL;
    if (p->inhibit < 0 || p->inhibit > (1 << 29)) return GS_ERR_INVAL;
    if (p->tau < 0) return GS_ERR_INVAL;
    if (p->direction < 0 || p->direction > 2) return GS_ERR_INVAL;
    g->ng = p->w - p->dis0;
    g->h = p->h;
    g->D = p->D;
    g->K = p->D - 1;
    g->P = (int32_t)round_up(g->ng, 32);
    g->SY = (int64_t)g->K * g->P;
    g->N = (int64_t)g->h * g->SY;
    g->lam = p->lambda;
    g->lam2 = 2 * p->lambda;
    g->h2h = p->inhibit;
    g->h2v = p->vertical_inhibit ? p->inhibit : 0;
    if (g->N > (int64_t)1 << 40) return GS_ERR_INVAL;
    return GS_OK;
}

int device_sms() {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return 1;
    return sms;
}

int grid_for(int64_t n, int per_sm) {
    const int64_t b = (n + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)per_sm * device_sms()));
}

size_t graph_bytes(const Geom &g) {
    return 256 + 9 * (size_t)round_up(g.N, 64) * sizeof(int32_t);
}

size_t work_bytes(const Geom &g) {
    return kWorkCtrlBytes + (size_t)round_up(g.N * sizeof(int32_t), 256) + tiled_work_extra(g);
}

State state_view(void *graph, const Geom &g) {
    State s;
    char *b = (char *)graph;
    size_t stride = (size_t)round_up(g.N, 64) * sizeof(int32_t);
    s.hdr = (GraphHeader *)b;
    b += 256;
    int32_t **arr[9] = {&s.rc, &s.rr, &s.rd, &s.ri0, &s.ri1, &s.ri2, &s.ri3, &s.ex, &s.ht};
    for (int i = 0; i < 9; i++) *arr[i] = (int32_t *)(b + i * stride);
    return s;
}

Work work_view(void *ws, const Geom &g) {
    Work w;
    w.ctrl = (Ctrl *)ws;
    w.mark = (int32_t *)((char *)ws + kWorkCtrlBytes);
    return w;
}

// Stage bytes [b0, b1) of an image row into shared memory (16-byte aligned
// dst).  With `vec` (the row starts on a 16-byte boundary) the 16-byte chunks
// from b0 rounded down that lie wholly inside the row's first row_end bytes
// are copied with 128-bit loads and stores, and the bytes past the last such
// chunk one at a time; nothing outside [0, row_end) is read.  Returns the
// position of byte b0 in dst.
__device__ __forceinline__ int stage_row(const uint8_t *__restrict__ row, int b0, int b1,
                                         int row_end, uint8_t *dst, bool vec) {
    if (!vec) {
        for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) dst[b - b0] = row[b];
        return 0;
    }
    const int a0 = b0 & ~15;
    const int vend = min((b1 + 15) & ~15, row_end & ~15);
    const int chunks = vend > a0 ? (vend - a0) >> 4 : 0;
    const uint4 *src = reinterpret_cast<const uint4 *>(row + a0);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    for (int c = threadIdx.x; c < chunks; c += blockDim.x) d[c] = __ldg(src + c);
    for (int b = max(vend, a0) + threadIdx.x; b < b1; b += blockDim.x) dst[b - a0] = row[b];
    return b0 - a0;
}

// Shared bytes for one staged span of n bytes (16-byte slack on each side).
__host__ __device__ __forceinline__ int span_bytes(int n) { return (n + 47) & ~15; }

// One block per (row y, tile of TW sites): the two image segments the tile
// touches are staged in shared memory (128-bit loads), then the [TW][D]
// output block, which is contiguous in the cost volume, is written with
// coalesced stores.
constexpr int kCostTW = 64;

__global__ void k_cost_volume(const uint8_t *__restrict__ L, const uint8_t *__restrict__ R,
                              int pitch, int w, int ng, int D, int dis0, int tau, int vec,
                              int32_t *__restrict__ cost) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int y = blockIdx.y;
    const int W0 = blockIdx.x * kCostTW;
    const int TW = min(kCostTW, ng - W0);
    const int span = TW + D - 1;
    uint8_t *sL = sm;                         // L[y][W0 + dis0 - (D-1) + t]
    uint8_t *sR = sm + span_bytes(span);      // R[y][W0 + t]
    const int xl0 = W0 + dis0 - (D - 1);
    const int oL = stage_row(L + (size_t)y * pitch, xl0, xl0 + span, w, sL, vec);
    const int oR = stage_row(R + (size_t)y * pitch, W0, W0 + span, w, sR, vec);
    __syncthreads();
    int32_t *out = cost + ((size_t)y * ng + W0) * D;
    const int n = TW * D;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int wi = e / D, S = e - wi * D;
        // x_l = W + dis0 - S  ->  sL index wi + (D-1) - S ; x_r = W + S -> sR index wi + S
        int d = (int)sL[oL + wi + (D - 1) - S] - (int)sR[oR + wi + S];
        d = d < 0 ? -d : d;
        out[e] = d < tau ? d : tau;
    }
}

// Colour data term of §4.3: sum over R, G, B of the absolute differences of
// the left pixel (x_l, y) and the right pixel (x_r, y), interleaved 8-bit
// RGB rows staged like the grayscale ones (3 bytes per pixel), truncated at
// tau (tau >= 765 gives the paper's plain sum).
__global__ void k_cost_volume_rgb(const uint8_t *__restrict__ L, const uint8_t *__restrict__ R,
                                  int pitch, int w, int ng, int D, int dis0, int tau, int vec,
                                  int32_t *__restrict__ cost) {
    extern __shared__ __align__(16) uint8_t sm[];
    const int y = blockIdx.y;
    const int W0 = blockIdx.x * kCostTW;
    const int TW = min(kCostTW, ng - W0);
    const int span = 3 * (TW + D - 1);
    uint8_t *sL = sm;
    uint8_t *sR = sm + span_bytes(span);
    const int xl0 = 3 * (W0 + dis0 - (D - 1));
    const int oL = stage_row(L + (size_t)y * pitch, xl0, xl0 + span, 3 * w, sL, vec);
    const int oR = stage_row(R + (size_t)y * pitch, 3 * W0, 3 * W0 + span, 3 * w, sR, vec);
    __syncthreads();
    int32_t *out = cost + ((size_t)y * ng + W0) * D;
    const int n = TW * D;
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        const int wi = e / D, S = e - wi * D;
        const uint8_t *lp = sL + oL + 3 * (wi + (D - 1) - S);
        const uint8_t *rp = sR + oR + 3 * (wi + S);
        const int sad = abs((int)lp[0] - (int)rp[0]) + abs((int)lp[1] - (int)rp[1]) +
                        abs((int)lp[2] - (int)rp[2]);
        out[e] = sad < tau ? sad : tau;
    }
}

__device__ __forceinline__ long long pair_term(int a, int b, int lam, int inh) {
    int d = a > b ? a - b : b - a;
    return (long long)lam * d + (d > 1 ? (long long)inh * (d - 1) : 0);
}

__global__ void k_energy(const int32_t *__restrict__ cost, const int32_t *__restrict__ X, int ng,
                         int h, int D, int lam, int h2h, int h2v,
                         unsigned long long *__restrict__ out) {
    long long acc = 0;
    const long long n = (long long)ng * h;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < n;
         v += (long long)gridDim.x * blockDim.x) {
        const int W = (int)(v % ng);
        const int y = (int)(v / ng);
        int a = X[v];
        if (a < 0 || a >= D) {       // invalid label: flag the result (sign bit) and skip
            atomicOr(out, 1ull << 63);
            a = 0;
        }
        acc += cost[v * D + a];
        if (W + 1 < ng) acc += pair_term(a, X[v + 1], lam, h2h);
        if (y + 1 < h) acc += pair_term(a, X[v + ng], lam, h2v);
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    __shared__ long long red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) atomicAdd(out, (unsigned long long)acc);
    }
}

}  // namespace gs

using namespace gs;

extern "C" {

int64_t gs_kernel_launches(void) { return g_launches.load(); }

int32_t gs_num_sites_w(const gs_params *p) {
    Geom g;
    return make_geom(p, &g) == GS_OK ? g.ng : 0;
}

size_t gs_cost_volume_bytes(const gs_params *p) {
    Geom g;
    if (make_geom(p, &g) != GS_OK) return 0;
    return (size_t)g.ng * g.h * g.D * sizeof(int32_t);
}

size_t gs_graph_bytes(const gs_params *p) {
    Geom g;
    return make_geom(p, &g) == GS_OK ? graph_bytes(g) : 0;
}

size_t gs_workspace_bytes(const gs_params *p, const gs_solve_opts *o) {
    Geom g;
    (void)o;
    return make_geom(p, &g) == GS_OK ? work_bytes(g) : 0;
}

int64_t gs_num_nodes(const gs_params *p) {
    Geom g;
    return make_geom(p, &g) == GS_OK ? (int64_t)g.ng * g.h * g.K : 0;
}

// 128-bit staging needs both images and every row on a 16-byte boundary.
static int rows_aligned(const uint8_t *L, const uint8_t *R, int32_t pitch) {
    return (((uintptr_t)L | (uintptr_t)R) & 15) == 0 && (pitch & 15) == 0;
}

int gs_stereo_cost_volume(const uint8_t *L, const uint8_t *R, int32_t pitch, const gs_params *p,
                          int32_t *cost, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !L || !R || !cost || pitch < p->w) return GS_ERR_INVAL;
    dim3 grid((g.ng + kCostTW - 1) / kCostTW, g.h);
    const size_t smem = 2 * (size_t)span_bytes(kCostTW + g.D - 1);
    if (smem > 48 * 1024) return GS_ERR_INVAL;
    k_cost_volume<<<grid, 256, smem, (cudaStream_t)stream>>>(
        L, R, pitch, p->w, g.ng, g.D, p->dis0, p->tau, rows_aligned(L, R, pitch), cost);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_stereo_cost_volume_rgb(const uint8_t *L, const uint8_t *R, int32_t pitch,
                              const gs_params *p, int32_t *cost, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !L || !R || !cost || pitch < 3 * (int64_t)p->w)
        return GS_ERR_INVAL;
    dim3 grid((g.ng + kCostTW - 1) / kCostTW, g.h);
    const size_t smem = 2 * (size_t)span_bytes(3 * (kCostTW + g.D - 1));
    if (smem > 48 * 1024) return GS_ERR_INVAL;
    k_cost_volume_rgb<<<grid, 256, smem, (cudaStream_t)stream>>>(
        L, R, pitch, p->w, g.ng, g.D, p->dis0, p->tau, rows_aligned(L, R, pitch), cost);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_energy(const int32_t *cost, const int32_t *labels, const gs_params *p, int64_t *energy,
              void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !labels || !energy) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(energy, 0, sizeof(int64_t), st));
    long long sites = (long long)g.ng * g.h;
    const int blocks = grid_for(sites, 4);
    k_energy<<<blocks, 256, 0, st>>>(cost, labels, g.ng, g.h, g.D, g.lam, g.h2h, g.h2v,
                                     (unsigned long long *)energy);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // extern "C"

// ------------------------------------------------- learned data term (FP32) ---
//
// c = w1 |L - R| + w2 |dxL - dxR| at the cross point, truncated at tau, then
// quantised to int32 at `scale` (round half to even).  dx is the central
// difference (I[x+1] - I[x-1]) / 2 with replicated borders.  Every product and
// sum is rounded separately (no fused multiply-add) so that the host reference
// computes the same integers.

namespace gs {

__device__ __forceinline__ float dx_at(const uint8_t *row, int x, int w) {
    const int xm = x > 0 ? x - 1 : 0, xp = x < w - 1 ? x + 1 : w - 1;
    return __fmul_rn(0.5f, (float)((int)row[xp] - (int)row[xm]));
}

// features of cross point (W, S) in row y: a = |L - R|, b = |dxL - dxR|
__device__ __forceinline__ void cross_features(const uint8_t *Lrow, const uint8_t *Rrow, int w,
                                               int W, int S, int dis0, float &fa, float &fb) {
    const int xr = W + S, xl = W + dis0 - S;
    fa = fabsf((float)((int)Lrow[xl] - (int)Rrow[xr]));
    fb = fabsf(__fsub_rn(dx_at(Lrow, xl, w), dx_at(Rrow, xr, w)));
}

__device__ __forceinline__ float learned_cost(float fa, float fb, float w1, float w2, float tau) {
    const float c = __fadd_rn(__fmul_rn(w1, fa), __fmul_rn(w2, fb));
    return fminf(c, tau);
}

__global__ void k_cost_volume_f32(const uint8_t *__restrict__ L, const uint8_t *__restrict__ R,
                                  int pitch, int w, int ng, int D, int dis0, float w1, float w2,
                                  float tau, float scale, int32_t *__restrict__ cost) {
    const int y = blockIdx.y;
    const uint8_t *Lrow = L + (size_t)y * pitch, *Rrow = R + (size_t)y * pitch;
    const int n = ng * D;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int W = e / D, S = e - W * D;
        float fa, fb;
        cross_features(Lrow, Rrow, w, W, S, dis0, fa, fb);
        const float c = learned_cost(fa, fb, w1, w2, tau);
        cost[(size_t)y * n + e] = __float2int_rn(__fmul_rn(scale, c));
    }
}

// Chain rule through the learned cost at the chosen labels: exact integer sums
//   out[0] = sum_v |L - R| [c < tau],  out[1] = sum_v 2|dxL - dxR| [c < tau],
//   out[2] = sum_v [c >= tau]
// (c at the label X_v).  dE/dw1 = out[0], dE/dw2 = out[1] / 2, dE/dtau = out[2]
// for the energy in cost units, the quantiser taken as the identity.
__global__ void k_cost_f32_backward(const uint8_t *__restrict__ L, const uint8_t *__restrict__ R,
                                    int pitch, int w, int ng, int h, int D, int dis0, float w1,
                                    float w2, float tau, const int32_t *__restrict__ X,
                                    unsigned long long *__restrict__ out) {
    unsigned long long sa = 0, sb = 0, st = 0;
    const long long sites = (long long)ng * h;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < sites;
         v += (long long)gridDim.x * blockDim.x) {
        const int W = (int)(v % ng), y = (int)(v / ng);
        const int S = min(max(X[v], 0), D - 1);
        float fa, fb;
        cross_features(L + (size_t)y * pitch, R + (size_t)y * pitch, w, W, S, dis0, fa, fb);
        const float c = __fadd_rn(__fmul_rn(w1, fa), __fmul_rn(w2, fb));
        if (c < tau) {
            sa += (unsigned long long)fa;
            sb += (unsigned long long)(2.0f * fb);
        } else {
            st += 1;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_down_sync(0xffffffffu, sa, o);
        sb += __shfl_down_sync(0xffffffffu, sb, o);
        st += __shfl_down_sync(0xffffffffu, st, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (sa) atomicAdd(&out[0], sa);
        if (sb) atomicAdd(&out[1], sb);
        if (st) atomicAdd(&out[2], st);
    }
}

// Adjoint of the minimum energy (§2) at the minimiser X: dE/dC[v][l] = [X_v = l]
// (written as grad * one-hot when dcost is given), dE/dlambda = sum |X_u - X_v|,
// dE/dinhibit = sum (|X_u - X_v| - 1)_+ over the pairs that carry the inhibit
// term.  E* is concave and piecewise linear in (C, lambda, inhibit); these are
// its gradients where X is the unique minimiser, and supergradients otherwise.
__global__ void k_energy_backward(const int32_t *__restrict__ X, int ng, int h, int D, int vinh,
                                  float grad, float *__restrict__ dcost,
                                  unsigned long long *__restrict__ counts) {
    unsigned long long jumps = 0, viol = 0;
    const long long sites = (long long)ng * h;
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < sites;
         v += (long long)gridDim.x * blockDim.x) {
        const int W = (int)(v % ng), y = (int)(v / ng);
        const int a = X[v];
        if (dcost)
            for (int l = 0; l < D; l++) dcost[v * D + l] = l == a ? grad : 0.0f;
        if (W + 1 < ng) {
            const int d = abs(a - X[v + 1]);
            jumps += d;
            viol += d > 1 ? d - 1 : 0;
        }
        if (y + 1 < h) {
            const int d = abs(a - X[v + ng]);
            jumps += d;
            if (vinh) viol += d > 1 ? d - 1 : 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        jumps += __shfl_down_sync(0xffffffffu, jumps, o);
        viol += __shfl_down_sync(0xffffffffu, viol, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (jumps) atomicAdd(&counts[0], jumps);
        if (viol) atomicAdd(&counts[1], viol);
    }
}

}  // namespace gs

extern "C" {

int gs_stereo_cost_volume_f32(const uint8_t *L, const uint8_t *R, int32_t pitch, const gs_params *p,
                              float w1, float w2, float tau, float scale, int32_t *cost,
                              void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !L || !R || !cost || pitch < p->w) return GS_ERR_INVAL;
    if (!(scale > 0.0f) || !(tau >= 0.0f) || !(w1 >= 0.0f) || !(w2 >= 0.0f)) return GS_ERR_INVAL;
    if ((double)scale * tau > (double)(1 << 30)) return GS_ERR_OVERFLOW;
    dim3 grid((g.ng * g.D + 255) / 256, g.h);
    k_cost_volume_f32<<<grid, 256, 0, (cudaStream_t)stream>>>(L, R, pitch, p->w, g.ng, g.D,
                                                              p->dis0, w1, w2, tau, scale, cost);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_cost_volume_f32_backward(const uint8_t *L, const uint8_t *R, int32_t pitch,
                                const gs_params *p, float w1, float w2, float tau,
                                const int32_t *labels, int64_t *sums, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !L || !R || !labels || !sums || pitch < p->w)
        return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(sums, 0, 3 * sizeof(int64_t), st));
    const long long sites = (long long)g.ng * g.h;
    const int blocks = grid_for(sites, 4);
    k_cost_f32_backward<<<blocks, 256, 0, st>>>(L, R, pitch, p->w, g.ng, g.h, g.D, p->dis0, w1, w2,
                                               tau, labels, (unsigned long long *)sums);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

int gs_energy_backward(const int32_t *labels, const gs_params *p, float grad, float *dcost,
                       int64_t *counts, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !labels || !counts) return GS_ERR_INVAL;
    cudaStream_t st = (cudaStream_t)stream;
    GS_CUDA_TRY(cudaMemsetAsync(counts, 0, 2 * sizeof(int64_t), st));
    const long long sites = (long long)g.ng * g.h;
    const int blocks = grid_for(sites, 16);
    k_energy_backward<<<blocks, 256, 0, st>>>(labels, g.ng, g.h, g.D, p->vertical_inhibit ? 1 : 0,
                                             grad, dcost, (unsigned long long *)counts);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}

}  // extern "C"

// Loss augmentation for structured learning: cost[v][labels[v]] += value.
namespace gs {
__global__ void k_cost_add_at_labels(int32_t *__restrict__ cost, const int32_t *__restrict__ X,
                                     long long sites, int D, int32_t value) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < sites;
         v += (long long)gridDim.x * blockDim.x) {
        const int a = X[v];
        if (a >= 0 && a < D) cost[v * D + a] += value;
    }
}
}  // namespace gs

extern "C" int gs_cost_add_at_labels(int32_t *cost, const int32_t *labels, const gs_params *p,
                                     int32_t value, void *stream) {
    Geom g;
    if (make_geom(p, &g) != GS_OK || !cost || !labels) return GS_ERR_INVAL;
    const long long sites = (long long)g.ng * g.h;
    const int blocks = grid_for(sites, 16);
    k_cost_add_at_labels<<<blocks, 256, 0, (cudaStream_t)stream>>>(cost, labels, sites, g.D, value);
    count_launches(1);
    GS_CUDA_TRY(cudaGetLastError());
    return GS_OK;
}
