// Internal layout of the solver state shared by the translation units of
// libgazecut.  Nothing here is visible through the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gazecut.h"

namespace gs {

// Height of a node that cannot reach the sink (distance "infinity").
constexpr int32_t kInfH = 0x3fffffff;
// Residual of the infinite reverse data arc n(v,k+1) -> n(v,k).
constexpr int32_t kInfR = 0x3fffffff;
// Bound on every stored capacity, excess and residual; larger values raise
// GS_ERR_OVERFLOW instead of wrapping.
constexpr int32_t kCapLimit = 1 << 30;

constexpr uint32_t kMagic = 0x47617a43u;  // "GazC"

// Node grid: rows y in [0,h), chain index j = k-1 in [0,K) (K = D-1), sites
// W in [0,n_g) padded to the pitch P (a multiple of 32).  Node index
//   i = (y*K + j)*P + W
// so a warp reads 32 consecutive sites of one depth layer, the chain
// neighbours are +-P and the vertical neighbours +-K*P.
struct Geom {
    int32_t ng, h, D, K, P;
    int64_t N;        // h*K*P (padded node count)
    int64_t SY;       // K*P, stride between rows
    int32_t lam, lam2;
    int32_t h2h, h2v; // inhibit capacity on horizontal / vertical pairs
};

// Header at the start of the graph buffer (256 bytes reserved).
// The graph may be built for the label-reversed problem C'(l) = C(D-1-l): it
// is the reversed graph (sources and sinks swapped, arcs reversed), has the
// same minimum energy, and its largest minimiser X'max gives the canonical
// smallest minimiser of the original as X = D-1-X'max.  build_graph picks the
// direction with the smaller total source capacity (less excess to route)
// unless the caller fixes it.
struct GraphHeader {
    uint32_t magic;
    int32_t D, ng, h, K, P, lam, inhibit, vinhibit;
    int32_t rev;                      // 1: the state is the label-reversed problem
    unsigned long long sum_first;     // sum of C(0) over sites
    unsigned long long init_deficit;  // total sink capacity left after folding
    unsigned long long src_total;     // total source capacity
    unsigned long long sum_last;      // sum of C(D-1) over sites
    int32_t exact_heights;            // 1: ht holds the exact distances of a finished solve
};

// Solver state: structure of arrays, each N int32, 256-byte aligned.
//   rc   residual of the data arc n(j) -> n(j+1) (the reverse arc is infinite)
//   rr   residual of the penalty arc to site W+1 (reverse = 2*lambda - rr)
//   rd   residual of the penalty arc to row y+1 (reverse = 2*lambda - rd)
//   ri[d] residual of the inhibit arc to neighbour d at layer j-1,
//        d = 0: W-1, 1: W+1, 2: y-1, 3: y+1 (reverse = h2_d - ri[d])
//   ex   excess (negative: sink capacity still unused)
//   ht   height (kInfH: cannot reach the sink)
struct State {
    GraphHeader *hdr;
    int32_t *rc, *rr, *rd, *ri0, *ri1, *ri2, *ri3, *ex, *ht;
};

// Workspace: control block, one int32 per node (label marks), then the
// tiled solver's per-node arc masks and per-tile flags.
struct Ctrl {
    int32_t status;
    int32_t changed;
    int32_t active;
    int32_t abort;
    int32_t converged;
    long long stats[8];   // relabels, sweeps, bfs passes, label passes, active at exit,
                          // sweep ns, relabel ns, launches
    unsigned long long deficit_left;
    long long visits_sweep;    // tile visits of the sweep rounds (all blocks)
    long long visits_relabel;  // tile visits of the relabel passes (all blocks)
    unsigned long long pad2;
};
static_assert(sizeof(Ctrl) <= 256, "ctrl block");

// Control region at the start of a workspace: the Ctrl block (256 bytes),
// then the persistent kernel's control words (an abort flag and a finished-
// pair count in a second Ctrl, then per pair its claim word, step, per-step
// sums and queue lengths, and state machine).
constexpr size_t kWorkCtrlBytes = 24576;

struct Work {
    Ctrl *ctrl;
    int32_t *mark;
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// Process-wide count of kernels this library has launched (diagnostics).
void count_launches(long long n);

// Tiled persistent solver (tile.cu): extra workspace bytes and the solve.
size_t tiled_work_extra(const Geom &g);
int tiled_solve(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                int32_t *status, cudaStream_t st);
int tiled_extract(const Geom &g, const State &s, const Work &w, const gs_solve_opts *o,
                  int32_t *labels, int64_t *flow, int32_t *status, cudaStream_t st);

// Validate params and fill the geometry.  Returns GS_OK or GS_ERR_INVAL.
int make_geom(const gs_params *p, Geom *g);
// Number of SMs of the current device (1 if the query fails).
int device_sms();
// Grid for a grid-stride kernel over n items with 256-thread blocks: enough
// blocks for n, at most per_sm resident blocks on every SM of the device.
int grid_for(int64_t n, int per_sm = 16);
size_t graph_bytes(const Geom &g);
size_t work_bytes(const Geom &g);
State state_view(void *graph, const Geom &g);
Work work_view(void *ws, const Geom &g);

}  // namespace gs

#define GS_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return GS_ERR_CUDA;          \
    } while (0)
