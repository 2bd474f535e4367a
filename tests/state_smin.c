/*
 * Canonical labels from a solved state of the chain graph (test infrastructure).
 *
 * Given a maximum preflow of the graph of §3 / Fig. 4 (terminal arcs folded
 * into node excess), the minimal source set of the minimum cut is the set of
 * nodes reachable, over arcs with residual capacity, from the nodes that still
 * hold excess (the source reaches them once the excess is returned to it).
 * The component-wise smallest minimiser of E is then X_v = |S_min ∩ chain(v)|.
 * For a state of the label-reversed problem C'(l) = C(D-1-l) (the reversed
 * graph) the canonical labels of the original are X = D-1-X'max, X'max read
 * from the maximal source set of the reversed problem: the nodes that cannot
 * reach remaining sink capacity (negative excess) over residual arcs.
 *
 * The arcs are taken from the graph's definition: per site a chain n_1..n_K
 * (K = D-1) with data arcs n_k -> n_(k+1) (residual stored at the tail) and
 * infinite reverse arcs; for every 4-neighbour pair (u, v) and layer k the
 * penalty pair u_k <-> v_k (capacity lambda each way; one residual stored at
 * the left / upper site, the other direction 2 lambda minus it); for every
 * ordered pair and k >= 2 the inhibit arc u_k -> v_(k-1) (residual stored at
 * the tail, the reverse is the capacity minus it).
 *
 * State layout (the library's): nine int32 arrays rc, rr, rd, ri0..ri3, ex,
 * ht over the node grid [h][K][P] (P = n_g rounded up to 32); ri_d holds the
 * inhibit arc towards neighbour d = 0: W-1, 1: W+1, 2: y-1, 3: y+1.
 *
 * Returns 0, or 1 when a chain's side is not a prefix (not a cut of the
 * chain graph), 2 on bad sizes, 3 when memory runs out.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    const int32_t *rc, *rr, *rd, *ri[4], *ex;
    int64_t h, K, P, ng;
    int64_t lam2, h2h, h2v;
} graph_t;

static inline int64_t node(const graph_t *g, int64_t y, int64_t j, int64_t W) {
    return (y * g->K + j) * g->P + W;
}

/* Residual of the arc a -> b between nodes (y,j,W) and (y2,j2,W2), which the
 * caller knows to exist.  Only the arc kinds of the graph occur. */
static int64_t residual(const graph_t *g, int64_t y, int64_t j, int64_t W, int64_t y2, int64_t j2,
                        int64_t W2) {
    const int64_t a = node(g, y, j, W), b = node(g, y2, j2, W2);
    if (y2 == y && W2 == W) {                        /* chain */
        if (j2 == j + 1) return g->rc[a];
        return (int64_t)1 << 40;                     /* infinite reverse data arc */
    }
    if (j2 == j) {                                   /* penalty pair */
        if (y2 == y && W2 == W + 1) return g->rr[a];
        if (y2 == y && W2 == W - 1) return g->lam2 - g->rr[b];
        if (y2 == y + 1) return g->rd[a];
        return g->lam2 - g->rd[b];                   /* y2 == y - 1 */
    }
    /* inhibit: the arc from layer j to layer j-1 is stored at its tail */
    const int d = W2 == W - 1 ? 0 : W2 == W + 1 ? 1 : y2 == y - 1 ? 2 : 3;
    if (j2 == j - 1) return g->ri[d][a];
    /* j2 == j + 1: reverse of the inhibit arc b -> a, stored at b towards a */
    const int back = d ^ 1;                          /* 0 <-> 1, 2 <-> 3 */
    const int64_t cap = d < 2 ? g->h2h : g->h2v;
    return cap - g->ri[back][b];
}

/* Visit the neighbours of node (y, j, W) along arcs with positive residual in
 * the given direction (forward: arcs leaving the node; backward: arcs
 * entering it), pushing unmarked ones on the queue. */
static void expand(const graph_t *g, int64_t y, int64_t j, int64_t W, int forward, uint8_t *mark,
                   int32_t *queue, int64_t *tail) {
    static const int dW[4] = {-1, 1, 0, 0}, dy[4] = {0, 0, -1, 1};
    int64_t nb[14][3];
    int n = 0;
    if (j + 1 < g->K) { nb[n][0] = y; nb[n][1] = j + 1; nb[n][2] = W; n++; }
    if (j > 0) { nb[n][0] = y; nb[n][1] = j - 1; nb[n][2] = W; n++; }
    for (int d = 0; d < 4; d++) {
        const int64_t y2 = y + dy[d], W2 = W + dW[d];
        if (y2 < 0 || y2 >= g->h || W2 < 0 || W2 >= g->ng) continue;
        nb[n][0] = y2; nb[n][1] = j; nb[n][2] = W2; n++;
        if (j > 0) { nb[n][0] = y2; nb[n][1] = j - 1; nb[n][2] = W2; n++; }
        if (j + 1 < g->K) { nb[n][0] = y2; nb[n][1] = j + 1; nb[n][2] = W2; n++; }
    }
    for (int q = 0; q < n; q++) {
        const int64_t y2 = nb[q][0], j2 = nb[q][1], W2 = nb[q][2];
        const int64_t r = forward ? residual(g, y, j, W, y2, j2, W2)
                                  : residual(g, y2, j2, W2, y, j, W);
        if (r <= 0) continue;
        const int64_t b = node(g, y2, j2, W2);
        if (mark[b]) continue;
        mark[b] = 1;
        queue[(*tail)++] = (int32_t)b;
    }
}

int smin_labels(const int32_t *const arrays[9], int64_t h, int64_t ng, int64_t D, int64_t lam,
                int64_t h2h, int64_t h2v, int rev, int32_t *labels) {
    if (h < 1 || ng < 1 || D < 2) return 2;
    graph_t g;
    g.rc = arrays[0];
    g.rr = arrays[1];
    g.rd = arrays[2];
    for (int d = 0; d < 4; d++) g.ri[d] = arrays[3 + d];
    g.ex = arrays[7];
    g.h = h;
    g.K = D - 1;
    g.P = (ng + 31) / 32 * 32;
    g.ng = ng;
    g.lam2 = 2 * lam;
    g.h2h = h2h;
    g.h2v = h2v;
    const int64_t N = h * g.K * g.P;
    if (N >= ((int64_t)1 << 31)) return 2;
    uint8_t *mark = calloc((size_t)N, 1);
    int32_t *queue = malloc((size_t)N * sizeof(int32_t));
    if (!mark || !queue) {
        free(mark);
        free(queue);
        return 3;
    }
    /* seeds: excess (forward search) or remaining sink capacity (backward) */
    int64_t head = 0, tail = 0;
    for (int64_t y = 0; y < h; y++)
        for (int64_t j = 0; j < g.K; j++)
            for (int64_t W = 0; W < ng; W++) {
                const int64_t a = node(&g, y, j, W);
                if (rev ? g.ex[a] < 0 : g.ex[a] > 0) {
                    mark[a] = 1;
                    queue[tail++] = (int32_t)a;
                }
            }
    while (head < tail) {
        const int64_t a = queue[head++];
        const int64_t W = a % g.P, t = a / g.P, j = t % g.K, y = t / g.K;
        expand(&g, y, j, W, !rev, mark, queue, &tail);
    }
    int bad = 0;
    for (int64_t y = 0; y < h; y++)
        for (int64_t W = 0; W < ng; W++) {
            /* source side: marked (forward) / not marked (backward) */
            int64_t cnt = 0;
            int prev = 1;
            for (int64_t j = 0; j < g.K; j++) {
                const int in = rev ? !mark[node(&g, y, j, W)] : mark[node(&g, y, j, W)];
                if (in && !prev) bad = 1;
                cnt += in;
                prev = in;
            }
            labels[y * ng + W] = (int32_t)(rev ? D - 1 - cnt : cnt);
        }
    free(mark);
    free(queue);
    return bad;
}
