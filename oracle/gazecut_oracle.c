/*
 * CPU oracle for the gaze-line / depth-number stereo min-cut.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header, table or helper with the CUDA
 * library: it is written straight from the paper's definitions and is meant
 * to be read side by side with them.
 *
 *   cost volume   data term g_v, §4.3 (grayscale truncated absolute difference
 *                 at the cross point (x_l, x_r, y), §3)
 *   graph         Ishikawa chain graph of the convex prior, §2 Eq. 1, §3
 *                 (h~(δ) = h~1|δ| + h~2 (|δ|-1) T(|δ|>1)), Fig. 4
 *   max-flow      Boykov-Kolmogorov search trees (the CPU solver of §4.4,
 *                 written from the published description: growth, augment,
 *                 adoption) and Dinic blocking flows as an independent second
 *                 solver
 *   min cut       S_min = nodes reachable from s in the final residual graph;
 *                 label X_v = |S_min ∩ chain(v)| (the "real cross points" of §3)
 *   energy        E(X) = Σ_v g_v(X_v) + Σ_(u,v) h~(X_u - X_v), §2
 *
 * Conventions (the paper omits the cuboid offsets, §4.1): sites (W, y) with
 * W in [0, n_g), n_g = w - dis0; depth number S in [0, D); the cross point
 * (W, S, y) pairs right pixel x_r = W + S with left pixel x_l = W + dis0 - S,
 * i.e. disparity dis(S) = dis0 - 2S.  Chain node n(v, k), k in [1, D-1];
 * n(v, 0) = s and n(v, D) = t.  Label a  <=>  n(v,1..a) on the source side.
 *
 * Everything is int64; "infinite" capacities are OR_INF.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

#define OR_INF ((i64)1 << 50)

/* ---------------------------------------------------------------- cost --- */

/* Data term at every cross point: C[(y*n_g + W)*D + S] = min(|L(x_l,y) - R(x_r,y)|, tau). */
int or_cost_volume(const uint8_t *L, const uint8_t *R, int w, int h, int D, int dis0,
                   int tau, int32_t *C)
{
    int ng = w - dis0;
    if (D < 2 || h < 1 || dis0 < 2 * (D - 1) || ng < 1) return 1;
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++)
            for (int S = 0; S < D; S++) {
                int xr = W + S;
                int xl = W + dis0 - S;
                int d = (int)L[(size_t)y * w + xl] - (int)R[(size_t)y * w + xr];
                if (d < 0) d = -d;
                C[((size_t)y * ng + W) * D + S] = d < tau ? d : tau;
            }
    return 0;
}

/* Colour data term of §4.3 at every cross point: the sum over the three
 * channels of the absolute difference between left pixel (x_l, y) and right
 * pixel (x_r, y), 0..765, then truncated at tau (tau >= 765: the paper's
 * plain sum).  L, R: interleaved 8-bit RGB, h rows of w pixels (3w bytes). */
int or_cost_volume_rgb(const uint8_t *L, const uint8_t *R, int w, int h, int D, int dis0,
                       int tau, int32_t *C)
{
    int ng = w - dis0;
    if (D < 2 || h < 1 || dis0 < 2 * (D - 1) || ng < 1) return 1;
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++)
            for (int S = 0; S < D; S++) {
                const uint8_t *lp = L + ((size_t)y * w + (W + dis0 - S)) * 3;
                const uint8_t *rp = R + ((size_t)y * w + (W + S)) * 3;
                int sad = 0;
                for (int c = 0; c < 3; c++) {
                    int d = (int)lp[c] - (int)rp[c];
                    sad += d < 0 ? -d : d;
                }
                C[((size_t)y * ng + W) * D + S] = sad < tau ? sad : tau;
            }
    return 0;
}

/* -------------------------------------------------------------- energy --- */

static i64 pair_term(int a, int b, i64 lam, i64 inh)
{
    i64 d = a > b ? a - b : b - a;
    return lam * d + (d > 1 ? inh * (d - 1) : 0);
}

/* E(X) over the 4-connected site grid; vertical pairs carry the inhibit term
 * only when vinhibit != 0. */
i64 or_energy(const int32_t *C, const int32_t *X, int ng, int h, int D, int lam,
              int inhibit, int vinhibit)
{
    i64 E = 0;
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++) {
            size_t v = (size_t)y * ng + W;
            E += C[v * D + X[v]];
            if (W + 1 < ng) E += pair_term(X[v], X[v + 1], lam, inhibit);
            if (y + 1 < h) E += pair_term(X[v], X[v + ng], lam, vinhibit ? inhibit : 0);
        }
    return E;
}

/* --------------------------------------------------------------- graph --- */

typedef struct {
    int n, m, mcap;         /* nodes, arcs used, arcs allocated */
    int *first, *next, *head;
    i64 *res, *cap0;
} graph_t;

static int g_init(graph_t *g, int n, int mcap)
{
    memset(g, 0, sizeof(*g));
    g->n = n;
    g->mcap = mcap;
    g->first = (int *)malloc(sizeof(int) * (size_t)n);
    g->next = (int *)malloc(sizeof(int) * (size_t)mcap);
    g->head = (int *)malloc(sizeof(int) * (size_t)mcap);
    g->res = (i64 *)malloc(sizeof(i64) * (size_t)mcap);
    g->cap0 = (i64 *)malloc(sizeof(i64) * (size_t)mcap);
    if (!g->first || !g->next || !g->head || !g->res || !g->cap0) return 1;
    for (int i = 0; i < n; i++) g->first[i] = -1;
    return 0;
}

static void g_free(graph_t *g)
{
    free(g->first); free(g->next); free(g->head); free(g->res); free(g->cap0);
    memset(g, 0, sizeof(*g));
}

/* Arc 2i is u->v with capacity cuv, arc 2i+1 is v->u with capacity cvu. */
static void g_edge(graph_t *g, int u, int v, i64 cuv, i64 cvu)
{
    int a = g->m;
    g->head[a] = v; g->res[a] = cuv; g->cap0[a] = cuv; g->next[a] = g->first[u]; g->first[u] = a;
    g->head[a + 1] = u; g->res[a + 1] = cvu; g->cap0[a + 1] = cvu; g->next[a + 1] = g->first[v];
    g->first[v] = a + 1;
    g->m += 2;
}

#define SRC 0
#define SNK 1

static int node_id(int ng, int D, int W, int y, int k)
{
    /* k in [1, D-1]; k = 0 is s, k = D is t */
    if (k <= 0) return SRC;
    if (k >= D) return SNK;
    return 2 + (int)(((size_t)y * ng + W) * (D - 1) + (k - 1));
}

/* The chain graph of Fig. 4 extended to the 4-connected grid:
 *   data      n(v,k) -> n(v,k+1), k in [0, D-1], capacity C_v(k); reverse infinite
 *             (the reverse arcs make every cut cross each chain exactly once);
 *   penalty   u_k <-> v_k, k in [1, D-1], capacity h~1 each way;
 *   inhibit   u_k -> v_(k-1), k in [2, D-1], capacity h~2, for both orders of
 *             every neighbouring pair (horizontal always, vertical when vinhibit).
 * For labels a = X_u, b = X_v the cut penalty arcs number |a-b| and the cut
 * inhibit arcs (|a-b|-1)_+, which reproduces h~ of §3 exactly. */
static int build(graph_t *g, const int32_t *C, int ng, int h, int D, int lam, int inhibit,
                 int vinhibit, long long extra)
{
    long long sites = (long long)ng * h;
    long long hp = (long long)(ng - 1) * h, vp = (long long)ng * (h - 1);
    long long ip = inhibit > 0 ? hp + (vinhibit ? vp : 0) : 0;
    long long edges = sites * D + (hp + vp) * (D - 1) + 2 * ip * (D > 2 ? D - 2 : 0);
    long long n = 2 + sites * (D - 1);
    if (n > 2000000000LL || 2 * (edges + extra) > 2000000000LL) return 2;
    if (g_init(g, (int)n, (int)(2 * (edges + extra)))) return 3;
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++) {
            const int32_t *c = C + ((size_t)y * ng + W) * D;
            for (int k = 0; k < D; k++) {
                int a = node_id(ng, D, W, y, k), b = node_id(ng, D, W, y, k + 1);
                g_edge(g, a, b, c[k], (a == SRC || b == SNK) ? 0 : OR_INF);
            }
        }
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++)
            for (int dir = 0; dir < 2; dir++) {
                int W2 = W + (dir == 0), y2 = y + (dir == 1);
                if (W2 >= ng || y2 >= h) continue;
                i64 h2 = (dir == 0 || vinhibit) ? inhibit : 0;
                for (int k = 1; k <= D - 1; k++)
                    g_edge(g, node_id(ng, D, W, y, k), node_id(ng, D, W2, y2, k), lam, lam);
                if (h2 > 0)
                    for (int k = 2; k <= D - 1; k++) {
                        g_edge(g, node_id(ng, D, W, y, k), node_id(ng, D, W2, y2, k - 1), h2, 0);
                        g_edge(g, node_id(ng, D, W2, y2, k), node_id(ng, D, W, y, k - 1), h2, 0);
                    }
            }
    return g->m == 2 * edges ? 0 : 4;
}

/* ------------------------------------------------------ Boykov-Kolmogorov --- */
/* Two search trees, S rooted at s and T rooted at t.  A tree arc of S runs
 * parent -> child, a tree arc of T runs child -> parent; both must be
 * residual.  Stages: growth (active nodes claim free neighbours until the trees
 * touch), augmentation (push the bottleneck along s ~> t, saturated tree arcs
 * turn their child into an orphan), adoption (an orphan finds a new parent in
 * its own tree whose root path is intact, or becomes free and orphans its
 * children). */

enum { FREE = 0, TS_ = 1, TT_ = 2 };
#define P_NONE (-1)     /* orphan / free */
#define P_ROOT (-2)     /* terminal */

typedef struct {
    graph_t *g;
    unsigned char *tree;
    int *parent;        /* arc index linking node and parent, or P_NONE / P_ROOT */
    int *stamp, *dist;  /* origin-check cache: valid at time stamp with root distance */
    int time;
    int *aq; size_t aq_head, aq_tail, aq_cap; unsigned char *inq;   /* active FIFO */
    int *oq; size_t oq_n, oq_cap;                                     /* orphan stack */
} bk_t;

static int tail_of(const graph_t *g, int a) { return g->head[a ^ 1]; }

static void bk_activate(bk_t *b, int u)
{
    if (b->inq[u]) return;
    if (b->aq_tail == b->aq_cap) {
        /* compact */
        size_t live = b->aq_tail - b->aq_head;
        memmove(b->aq, b->aq + b->aq_head, live * sizeof(int));
        b->aq_head = 0; b->aq_tail = live;
        if (live == b->aq_cap) { b->aq_cap *= 2; b->aq = (int *)realloc(b->aq, b->aq_cap * sizeof(int)); }
    }
    b->aq[b->aq_tail++] = u;
    b->inq[u] = 1;
}

static void bk_orphan(bk_t *b, int u)
{
    b->parent[u] = P_NONE;
    if (b->oq_n == b->oq_cap) { b->oq_cap *= 2; b->oq = (int *)realloc(b->oq, b->oq_cap * sizeof(int)); }
    b->oq[b->oq_n++] = u;
}

/* Residual capacity of the arc that would link q as parent of p in tree tr. */
static i64 tree_cap_to(const graph_t *g, int a_from_p, int tr)
{
    /* a_from_p is an arc p -> q.  For S, the parent arc is q -> p = a^1;
     * for T, the parent arc is p -> q = a. */
    return tr == TS_ ? g->res[a_from_p ^ 1] : g->res[a_from_p];
}

/* Is the root path of q intact?  Returns its distance to the root or -1. */
static int bk_origin(bk_t *b, int q)
{
    const graph_t *g = b->g;
    int d = 0, u = q;
    while (1) {
        if (b->stamp[u] == b->time) { d += b->dist[u]; break; }
        int pa = b->parent[u];
        if (pa == P_ROOT) { break; }
        if (pa == P_NONE) return -1;
        /* parent node of u */
        u = (b->tree[u] == TS_) ? tail_of(g, pa) : g->head[pa];
        d++;
    }
    /* refresh the cache along the verified path */
    int dd = d;
    u = q;
    while (1) {
        if (b->stamp[u] == b->time) break;
        b->stamp[u] = b->time;
        b->dist[u] = dd;
        int pa = b->parent[u];
        if (pa == P_ROOT) break;
        u = (b->tree[u] == TS_) ? tail_of(g, pa) : g->head[pa];
        dd--;
    }
    return d;
}

static void bk_augment(bk_t *b, int a_mid, i64 *flow)
{
    graph_t *g = b->g;
    /* a_mid: residual arc p -> q with p in S and q in T */
    i64 bott = g->res[a_mid];
    int u = tail_of(g, a_mid);
    while (b->parent[u] != P_ROOT) { int pa = b->parent[u]; if (g->res[pa] < bott) bott = g->res[pa]; u = tail_of(g, pa); }
    u = g->head[a_mid];
    while (b->parent[u] != P_ROOT) { int pa = b->parent[u]; if (g->res[pa] < bott) bott = g->res[pa]; u = g->head[pa]; }

    g->res[a_mid] -= bott; g->res[a_mid ^ 1] += bott;
    u = tail_of(g, a_mid);
    while (b->parent[u] != P_ROOT) {
        int pa = b->parent[u];
        int par = tail_of(g, pa);
        g->res[pa] -= bott; g->res[pa ^ 1] += bott;
        if (g->res[pa] == 0) bk_orphan(b, u);
        u = par;
    }
    u = g->head[a_mid];
    while (b->parent[u] != P_ROOT) {
        int pa = b->parent[u];
        int par = g->head[pa];
        g->res[pa] -= bott; g->res[pa ^ 1] += bott;
        if (g->res[pa] == 0) bk_orphan(b, u);
        u = par;
    }
    *flow += bott;
}

static void bk_adopt(bk_t *b)
{
    graph_t *g = b->g;
    while (b->oq_n > 0) {
        int p = b->oq[--b->oq_n];
        int tr = b->tree[p];
        int best = P_NONE, bestd = 0x7fffffff;
        for (int a = g->first[p]; a >= 0; a = g->next[a]) {
            int q = g->head[a];
            if (b->tree[q] != tr || tree_cap_to(g, a, tr) <= 0) continue;
            int d = bk_origin(b, q);
            if (d >= 0 && d < bestd) { bestd = d; best = (tr == TS_) ? (a ^ 1) : a; }
        }
        if (best != P_NONE) {
            b->parent[p] = best;
            b->stamp[p] = b->time;
            b->dist[p] = bestd + 1;
            continue;
        }
        /* no parent: p becomes free */
        for (int a = g->first[p]; a >= 0; a = g->next[a]) {
            int q = g->head[a];
            if (b->tree[q] != tr) continue;
            if (tree_cap_to(g, a, tr) > 0) bk_activate(b, q);
            int pq = b->parent[q];
            if (pq >= 0) {
                int par = (tr == TS_) ? tail_of(g, pq) : g->head[pq];
                if (par == p) bk_orphan(b, q);
            }
        }
        b->tree[p] = FREE;
    }
}

static i64 bk_maxflow(graph_t *g)
{
    bk_t b;
    memset(&b, 0, sizeof(b));
    b.g = g;
    int n = g->n;
    b.tree = (unsigned char *)calloc((size_t)n, 1);
    b.inq = (unsigned char *)calloc((size_t)n, 1);
    b.parent = (int *)malloc(sizeof(int) * (size_t)n);
    b.stamp = (int *)calloc((size_t)n, sizeof(int));
    b.dist = (int *)calloc((size_t)n, sizeof(int));
    b.aq_cap = 1024; b.aq = (int *)malloc(b.aq_cap * sizeof(int));
    b.oq_cap = 1024; b.oq = (int *)malloc(b.oq_cap * sizeof(int));
    for (int i = 0; i < n; i++) b.parent[i] = P_NONE;
    b.time = 1;
    b.tree[SRC] = TS_; b.parent[SRC] = P_ROOT; b.stamp[SRC] = b.time; b.dist[SRC] = 0;
    b.tree[SNK] = TT_; b.parent[SNK] = P_ROOT; b.stamp[SNK] = b.time; b.dist[SNK] = 0;
    bk_activate(&b, SRC);
    bk_activate(&b, SNK);
    i64 flow = 0;
    while (b.aq_head < b.aq_tail) {
        int p = b.aq[b.aq_head];
        if (b.tree[p] == FREE) { b.inq[p] = 0; b.aq_head++; continue; }
        int found = -1;
        int tr = b.tree[p];
        for (int a = g->first[p]; a >= 0; a = g->next[a]) {
            int q = g->head[a];
            /* growth along residual p -> q (S) or q -> p (T) */
            i64 r = (tr == TS_) ? g->res[a] : g->res[a ^ 1];
            if (r <= 0) continue;
            if (b.tree[q] == FREE) {
                b.tree[q] = (unsigned char)tr;
                b.parent[q] = (tr == TS_) ? a : (a ^ 1);
                b.stamp[q] = b.stamp[p];
                b.dist[q] = b.dist[p] + 1;
                bk_activate(&b, q);
            } else if (b.tree[q] != tr) {
                found = (tr == TS_) ? a : (a ^ 1);   /* arc from the S side to the T side */
                break;
            }
        }
        if (found < 0) { b.inq[p] = 0; b.aq_head++; continue; }
        b.time++;
        bk_augment(&b, found, &flow);
        bk_adopt(&b);
        /* p stays at the head of the queue and is scanned again */
    }
    free(b.tree); free(b.inq); free(b.parent); free(b.stamp); free(b.dist); free(b.aq); free(b.oq);
    return flow;
}

/* ----------------------------------------------------------------- Dinic --- */

static int dinic_bfs(graph_t *g, int *level, int *queue)
{
    for (int i = 0; i < g->n; i++) level[i] = -1;
    int qh = 0, qt = 0;
    level[SRC] = 0; queue[qt++] = SRC;
    while (qh < qt) {
        int u = queue[qh++];
        for (int a = g->first[u]; a >= 0; a = g->next[a])
            if (g->res[a] > 0 && level[g->head[a]] < 0) {
                level[g->head[a]] = level[u] + 1;
                queue[qt++] = g->head[a];
            }
    }
    return level[SNK] >= 0;
}

static i64 dinic_maxflow(graph_t *g)
{
    int n = g->n;
    int *level = (int *)malloc(sizeof(int) * (size_t)n);
    int *queue = (int *)malloc(sizeof(int) * (size_t)n);
    int *it = (int *)malloc(sizeof(int) * (size_t)n);
    int *stk = (int *)malloc(sizeof(int) * (size_t)n);   /* arcs of the current path */
    i64 flow = 0;
    while (dinic_bfs(g, level, queue)) {
        memcpy(it, g->first, sizeof(int) * (size_t)n);
        int top = 0, u = SRC;
        while (1) {
            if (u == SNK) {
                i64 bott = OR_INF;
                for (int i = 0; i < top; i++) if (g->res[stk[i]] < bott) bott = g->res[stk[i]];
                int cut = -1;
                for (int i = 0; i < top; i++) {
                    g->res[stk[i]] -= bott; g->res[stk[i] ^ 1] += bott;
                    if (cut < 0 && g->res[stk[i]] == 0) cut = i;
                }
                flow += bott;
                top = cut;
                u = tail_of(g, stk[cut]);
                continue;
            }
            int a = it[u];
            while (a >= 0 && !(g->res[a] > 0 && level[g->head[a]] == level[u] + 1)) a = g->next[a];
            it[u] = a;
            if (a >= 0) { stk[top++] = a; u = g->head[a]; continue; }
            /* dead end: retreat */
            level[u] = -1;
            if (u == SRC) break;
            int pa = stk[--top];
            u = tail_of(g, pa);
            it[u] = g->next[it[u]];
        }
    }
    free(level); free(queue); free(it); free(stk);
    return flow;
}

/* ------------------------------------------------------------- min cut --- */

/* S_min: nodes reachable from s in the residual graph of a maximum flow. */
static void reach_from_source(const graph_t *g, unsigned char *inS)
{
    int *queue = (int *)malloc(sizeof(int) * (size_t)g->n);
    memset(inS, 0, (size_t)g->n);
    int qh = 0, qt = 0;
    inS[SRC] = 1; queue[qt++] = SRC;
    while (qh < qt) {
        int u = queue[qh++];
        for (int a = g->first[u]; a >= 0; a = g->next[a])
            if (g->res[a] > 0 && !inS[g->head[a]]) { inS[g->head[a]] = 1; queue[qt++] = g->head[a]; }
    }
    free(queue);
}

static i64 cut_capacity(const graph_t *g, const unsigned char *inS)
{
    i64 c = 0;
    for (int a = 0; a < g->m; a++)
        if (inS[tail_of(g, a)] && !inS[g->head[a]]) c += g->cap0[a];
    return c;
}

/*
 * Exact minimum of E(X) by max-flow on the chain graph.
 *   method 0 = Boykov-Kolmogorov, 1 = Dinic.
 * Outputs: flow value, canonical labels X_min (from S_min, the smallest
 * minimiser), the capacity of the cut S_min, and X_max read from the largest
 * source set (nodes that cannot reach t).
 * Returns 0, or non-zero on bad sizes / allocation failure / a source set that
 * is not a prefix of some chain (which a correct max flow never produces).
 */
int or_solve(const int32_t *C, int ng, int h, int D, int lam, int inhibit, int vinhibit,
             int method, i64 *flow_out, int32_t *labels, i64 *cut_out, int32_t *labels_max)
{
    if (D < 2 || ng < 1 || h < 1 || lam < 0 || inhibit < 0) return 1;
    for (size_t i = 0; i < (size_t)ng * h * D; i++) if (C[i] < 0) return 1;
    graph_t g;
    int rc = build(&g, C, ng, h, D, lam, inhibit, vinhibit, 0);
    if (rc) { g_free(&g); return 10 + rc; }
    i64 flow = method == 0 ? bk_maxflow(&g) : dinic_maxflow(&g);
    unsigned char *inS = (unsigned char *)malloc((size_t)g.n);
    reach_from_source(&g, inS);
    if (inS[SNK]) { free(inS); g_free(&g); return 5; }
    *flow_out = flow;
    *cut_out = cut_capacity(&g, inS);
    int bad = 0;
    for (size_t v = 0; v < (size_t)ng * h; v++) {
        int W = (int)(v % ng), y = (int)(v / ng);
        int a = 0;
        while (a + 1 <= D - 1 && inS[node_id(ng, D, W, y, a + 1)]) a++;
        for (int k = a + 1; k <= D - 1; k++) if (inS[node_id(ng, D, W, y, k)]) bad = 1;
        labels[v] = a;
    }
    if (labels_max) {
        /* T side: nodes that can reach t; reverse BFS over residual arcs */
        unsigned char *inT = (unsigned char *)calloc((size_t)g.n, 1);
        int *queue = (int *)malloc(sizeof(int) * (size_t)g.n);
        int qh = 0, qt = 0;
        inT[SNK] = 1; queue[qt++] = SNK;
        while (qh < qt) {
            int u = queue[qh++];
            for (int a = g.first[u]; a >= 0; a = g.next[a]) {
                /* arc a: u -> x; residual x -> u is res[a^1] */
                int x = g.head[a];
                if (g.res[a ^ 1] > 0 && !inT[x]) { inT[x] = 1; queue[qt++] = x; }
            }
        }
        for (size_t v = 0; v < (size_t)ng * h; v++) {
            int W = (int)(v % ng), y = (int)(v / ng);
            int a = 0;
            while (a + 1 <= D - 1 && !inT[node_id(ng, D, W, y, a + 1)]) a++;
            for (int k = a + 1; k <= D - 1; k++) if (!inT[node_id(ng, D, W, y, k)]) bad = 1;
            labels_max[v] = a;
        }
        free(inT); free(queue);
    }
    free(inS);
    g_free(&g);
    return bad ? 6 : 0;
}

/*
 * The second cut of the level-1 approximation (§4.5): the exact minimum of
 * E(X) over labelings with lo_v <= X_v <= hi_v at every site (the "thin skin"
 * around the first cut).  The bounds pin chain nodes to a side: X_v >= lo_v
 * puts n(v,1..lo_v) on the source side (an infinite arc s -> n(v,lo_v); the
 * infinite reverse chain arcs carry it down the chain), X_v <= hi_v puts
 * n(v,hi_v+1..D-1) on the sink side (an infinite arc n(v,hi_v+1) -> t).
 * lo, hi: int32 [h][n_g], 0 <= lo <= hi <= D-1.  Outputs as or_solve (the
 * flow value is that of the pinned graph, i.e. E of the labels).  Returns 1 on
 * bad bounds, else as or_solve.
 */
int or_solve_band(const int32_t *C, int ng, int h, int D, int lam, int inhibit, int vinhibit,
                  const int32_t *lo, const int32_t *hi, int method, i64 *flow_out,
                  int32_t *labels)
{
    if (D < 2 || ng < 1 || h < 1 || lam < 0 || inhibit < 0) return 1;
    for (size_t i = 0; i < (size_t)ng * h * D; i++) if (C[i] < 0) return 1;
    for (size_t v = 0; v < (size_t)ng * h; v++)
        if (lo[v] < 0 || lo[v] > hi[v] || hi[v] > D - 1) return 1;
    graph_t g;
    int rc = build(&g, C, ng, h, D, lam, inhibit, vinhibit, 2LL * ng * h);
    if (rc) { g_free(&g); return 10 + rc; }
    for (int y = 0; y < h; y++)
        for (int W = 0; W < ng; W++) {
            size_t v = (size_t)y * ng + W;
            if (lo[v] >= 1) g_edge(&g, SRC, node_id(ng, D, W, y, lo[v]), OR_INF, 0);
            if (hi[v] <= D - 2) g_edge(&g, node_id(ng, D, W, y, hi[v] + 1), SNK, OR_INF, 0);
        }
    i64 flow = method == 0 ? bk_maxflow(&g) : dinic_maxflow(&g);
    unsigned char *inS = (unsigned char *)malloc((size_t)g.n);
    reach_from_source(&g, inS);
    if (inS[SNK]) { free(inS); g_free(&g); return 5; }
    *flow_out = flow;
    int bad = 0;
    for (size_t v = 0; v < (size_t)ng * h; v++) {
        int W = (int)(v % ng), y = (int)(v / ng);
        int a = 0;
        while (a + 1 <= D - 1 && inS[node_id(ng, D, W, y, a + 1)]) a++;
        for (int k = a + 1; k <= D - 1; k++) if (inS[node_id(ng, D, W, y, k)]) bad = 1;
        labels[v] = a;
    }
    free(inS);
    g_free(&g);
    return bad ? 6 : 0;
}

/* Number of nodes and arcs of the chain graph (for sizing and for tests). */
void or_graph_size(int ng, int h, int D, int vinhibit, i64 *nodes, i64 *edges)
{
    long long sites = (long long)ng * h;
    long long hp = (long long)(ng - 1) * h, vp = (long long)ng * (h - 1);
    *nodes = 2 + sites * (D - 1);
    *edges = sites * D + (hp + vp) * (D - 1) + 2 * (hp + (vinhibit ? vp : 0)) * (D > 2 ? D - 2 : 0);
}
