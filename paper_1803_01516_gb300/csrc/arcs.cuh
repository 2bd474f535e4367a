// The 14 residual arcs of one chain node of the gaze-line graph (§3, Fig. 4).
//
// Node u = (y, j, W) (j = k - 1).  Slots:
//   0  data arc up the chain      u -> (y, j+1, W)   residual rc[u]
//   1  reverse data arc           u -> (y, j-1, W)   infinite
//   2  penalty to W+1             residual rr[u]
//   3  penalty to W-1             2*lambda - rr[u-1]
//   4  penalty to y+1             rd[u]
//   5  penalty to y-1             2*lambda - rd[u-SY]
//   6+d inhibit u_k -> n_(k-1), neighbour d (0: W-1, 1: W+1, 2: y-1, 3: y+1)
//                                 residual ri_d[u]
//   10+d reverse of the inhibit arc n_(k+1) -> u_k of neighbour d
//                                 residual h2_d - ri_opp(d)[n at j+1]
// A slot whose arc does not exist (grid border, j = 0 or j = K-1) reports 0.
#pragma once

#include "gs_internal.cuh"

namespace gs {

constexpr int kSlots = 14;

__device__ __forceinline__ int32_t *ri_ptr(const State &s, int d) {
    return d == 0 ? s.ri0 : d == 1 ? s.ri1 : d == 2 ? s.ri2 : s.ri3;
}

// Offset from u to the head of each slot's arc.
__device__ __forceinline__ int64_t slot_offset(const Geom &g, int slot) {
    const int64_t P = g.P, SY = g.SY;
    switch (slot) {
        case 0: return P;
        case 1: return -P;
        case 2: return 1;
        case 3: return -1;
        case 4: return SY;
        case 5: return -SY;
        case 6: return -1 - P;
        case 7: return 1 - P;
        case 8: return -SY - P;
        case 9: return SY - P;
        case 10: return -1 + P;
        case 11: return 1 + P;
        case 12: return -SY + P;
        default: return SY + P;
    }
}

struct NodePos {
    int y, j, W;
};

__device__ __forceinline__ NodePos node_pos(const Geom &g, int64_t i) {
    NodePos p;
    p.W = (int)(i % g.P);
    const int64_t t = i / g.P;
    p.j = (int)(t % g.K);
    p.y = (int)(t / g.K);
    return p;
}

// Residuals of all 14 slots of node i (0 where the arc does not exist).
__device__ __forceinline__ void load_residuals(const State &s, const Geom &g, int64_t i,
                                               const NodePos &p, int32_t r[kSlots]) {
    const bool up = p.j < g.K - 1, dn = p.j > 0;
    const bool nb[4] = {p.W > 0, p.W < g.ng - 1, p.y > 0, p.y < g.h - 1};
    const int64_t P = g.P, SY = g.SY;
    r[0] = up ? s.rc[i] : 0;
    r[1] = dn ? kInfR : 0;
    r[2] = nb[1] ? s.rr[i] : 0;
    r[3] = nb[0] ? g.lam2 - s.rr[i - 1] : 0;
    r[4] = nb[3] ? s.rd[i] : 0;
    r[5] = nb[2] ? g.lam2 - s.rd[i - SY] : 0;
    r[6] = (dn && nb[0]) ? s.ri0[i] : 0;
    r[7] = (dn && nb[1]) ? s.ri1[i] : 0;
    r[8] = (dn && nb[2]) ? s.ri2[i] : 0;
    r[9] = (dn && nb[3]) ? s.ri3[i] : 0;
    // reverse inhibit: the arc (nbr, j+1) -> u is stored at the neighbour under
    // the direction pointing back to u
    r[10] = (up && nb[0]) ? g.h2h - s.ri1[i - 1 + P] : 0;
    r[11] = (up && nb[1]) ? g.h2h - s.ri0[i + 1 + P] : 0;
    r[12] = (up && nb[2]) ? g.h2v - s.ri3[i - SY + P] : 0;
    r[13] = (up && nb[3]) ? g.h2v - s.ri2[i + SY + P] : 0;
}

// Apply a push of delta along slot's arc to the residual state (atomically:
// the arc's other end may push the other way at the same time).  Returns the
// new value of a residual that grew, to let callers detect overflow.
__device__ __forceinline__ int32_t push_residual(const State &s, const Geom &g, int64_t i, int slot,
                                                 int32_t delta) {
    const int64_t P = g.P, SY = g.SY;
    switch (slot) {
        case 0: atomicSub(&s.rc[i], delta); return 0;
        case 1: return atomicAdd(&s.rc[i - P], delta) + delta;
        case 2: atomicSub(&s.rr[i], delta); return 0;
        case 3: return atomicAdd(&s.rr[i - 1], delta) + delta;
        case 4: atomicSub(&s.rd[i], delta); return 0;
        case 5: return atomicAdd(&s.rd[i - SY], delta) + delta;
        case 6: atomicSub(&s.ri0[i], delta); return 0;
        case 7: atomicSub(&s.ri1[i], delta); return 0;
        case 8: atomicSub(&s.ri2[i], delta); return 0;
        case 9: atomicSub(&s.ri3[i], delta); return 0;
        case 10: return atomicAdd(&s.ri1[i - 1 + P], delta) + delta;
        case 11: return atomicAdd(&s.ri0[i + 1 + P], delta) + delta;
        case 12: return atomicAdd(&s.ri3[i - SY + P], delta) + delta;
        default: return atomicAdd(&s.ri2[i + SY + P], delta) + delta;
    }
}

}  // namespace gs
