/*
 * FP64 CPU oracle for the layout method of "Graph Visualization for
 * Blockchain Data" (Dietl, Gemuend, Oeltz, Thiele, Werner, 2024).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled on its own with gcc and is
 * called only by the tests, by the smoke check and by the CPU-baseline leg of
 * the benchmark.  It shares no code, header or table with the CUDA library,
 * and the library never calls it.
 *
 * Everything is written as the plain definition, in double precision, with
 * no blocking or reordering beyond what the definition states:
 *
 *   Section 2   bipartite address/transaction graph             orc_graph_build
 *               undirected simple adjacency, degrees            orc_undirected_csr
 *   Section 4   connected components (directions ignored)       orc_components
 *               components ordered for the size split           orc_component_order
 *   Section 3.1 all-pairs graph distances (BFS; Floyd-Warshall) orc_bfs_apsp, orc_floyd_warshall
 *               Kamada-Kawai energy, gradient, Hessian          orc_kk_energy, orc_kk_grad_hess
 *               Newton-Raphson minimisation (Gauss-Seidel)      orc_kk_run
 *   Section 3.2 ForceAtlas2 forces: edge attraction, gravity,   orc_fa2_forces
 *               all-pairs repulsion; layout energy              orc_fa2_energy
 *               swing / traction adaptive speed and update      orc_fa2_run
 *   initial positions (SplitMix64, a counter-based generator)   orc_init_positions
 *
 * The Fast Multipole Method of Section 3.2.1 approximates the exact
 * repulsion sum; its reference is orc_fa2_forces' exact sum.
 *
 * Readings of the paper where it is silent (each also listed in the design
 * notes):
 *   - repulsion kr * m_i * m_j / d with mass m = degree + 1 (ForceAtlas2's
 *     degree weighting), attraction coefficient 1, gravity -kg * m_i * p_i
 *     toward the component origin;
 *   - swing and traction exactly as printed in Section 3.2 (unweighted sums)
 *     unless variant 1 (ForceAtlas2's degree-weighted, halved traction);
 *   - global speed s_G = min(tau * trc / swg, 1.5 * s_G), s_G starts at 1,
 *     F_{-1} = 0; per-node speed ks * s_G / (1 + s_G sqrt(|F_t - F_{t-1}|)),
 *     capped so that no node moves farther than ksmax;
 *   - coincident points (distance 0) exert no repulsion on each other;
 *   - KK: k_ij = d_ij^-2, l_ij = l d_ij, one sweep = one 2x2 Newton step per
 *     node in ascending id order using positions already updated in the
 *     sweep; where H is not positive definite its non-positive eigenvalues
 *     are replaced by max(|l|, 0.1 max|l|), and steps are no longer than l
 *     (a safeguarded Newton-Raphson step: the plain step diverges from
 *     random starts where H is indefinite).
 * "parity unpinned": none.  Every function has a pin in tests/test_oracle.py;
 * the safeguarded KK step (orc_kk_step) by hand-worked 2x2 cases
 * (tests/golden/kk_newton_step.json: plain, shortened, isotropic,
 * indefinite, floored, a small positive eigenvalue kept, zero), both
 * swing/traction variants by a hand-worked iteration of a three-node path
 * with unequal masses (tests/golden/fa2_swing_variants.json), the iteration
 * off the axes with tau != 1, s_G != 1 and both caps by six hand-worked cases
 * (tests/golden/fa2_iteration_2d.json).  Every single-operator, constant or
 * statement mutation of this file that changes a result on valid input
 * fails one of the pins.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* SplitMix64 (Steele, Lea, Flood, OOPSLA 2014), used for the initial   */
/* positions.                                                           */
/* ------------------------------------------------------------------ */
static uint64_t orc_splitmix64(uint64_t *state)
{
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* first n outputs of SplitMix64 from the given seed (for its published test vector) */
void orc_splitmix64_stream(uint64_t seed, int64_t n, uint64_t *out)
{
    uint64_t s = seed;
    for (int64_t i = 0; i < n; ++i) out[i] = orc_splitmix64(&s);
}

/*
 * Initial position of node `id`: a fresh SplitMix64 stream with state
 * seed XOR (id * 0x9E3779B97F4A7C15); x from its first output, y from its
 * second, each as ((h >> 40) * 2^-24) * 2 - 1, uniform on [-1, 1).
 */
void orc_init_positions(uint64_t seed, int64_t n, const int64_t *ids, double *x, double *y)
{
    for (int64_t i = 0; i < n; ++i) {
        uint64_t s = seed ^ ((uint64_t)ids[i] * 0x9E3779B97F4A7C15ULL);
        uint64_t hx = orc_splitmix64(&s);
        uint64_t hy = orc_splitmix64(&s);
        x[i] = ldexp((double)(hx >> 40), -24) * 2.0 - 1.0;
        y[i] = ldexp((double)(hy >> 40), -24) * 2.0 - 1.0;
    }
}

/* ------------------------------------------------------------------ */
/* Section 2: the bipartite transaction graph                           */
/* ------------------------------------------------------------------ */

typedef struct {
    uint64_t *key;
    int64_t *val;
    unsigned char *used;
    int64_t cap;
} orc_map;

static uint64_t orc_hash(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xFF51AFD7ED558CCDULL;
    k ^= k >> 33;
    return k;
}

/* value stored for `key`, or -1 */
static int64_t orc_map_get(const orc_map *m, uint64_t key)
{
    uint64_t h = orc_hash(key) & (uint64_t)(m->cap - 1);
    while (m->used[h]) {
        if (m->key[h] == key) return m->val[h];
        h = (h + 1) & (uint64_t)(m->cap - 1);
    }
    return -1;
}

static void orc_map_put(orc_map *m, uint64_t key, int64_t val)
{
    uint64_t h = orc_hash(key) & (uint64_t)(m->cap - 1);
    while (m->used[h]) h = (h + 1) & (uint64_t)(m->cap - 1);
    m->used[h] = 1;
    m->key[h] = key;
    m->val[h] = val;
}

typedef struct { int32_t a, b; } orc_pair;

static int orc_pair_cmp(const void *p, const void *q)
{
    const orc_pair *x = (const orc_pair *)p, *y = (const orc_pair *)q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return 0;
}

/*
 * Section 2: vertices are addresses and transactions.  An edge address -> tx
 * exists when the address is an input of the tx; an edge tx -> address when
 * it is an output.
 *
 * Node ids: transaction t has id t; an address has id n_tx + (its rank of
 * first appearance when scanning tx 0 inputs, tx 0 outputs, tx 1 inputs, ...).
 * Exact duplicate directed edges are kept once.  Directed edges are returned
 * sorted by (src, dst).  Buffers addr_out, src_out, dst_out need room for
 * in_off[n_tx] + out_off[n_tx] entries.  Returns the number of addresses;
 * *n_edges receives the number of directed edges.
 */
int64_t orc_graph_build(int64_t n_tx, const int64_t *in_off, const uint64_t *in_addr,
                        const int64_t *out_off, const uint64_t *out_addr, uint64_t *addr_out,
                        int32_t *src_out, int32_t *dst_out, int64_t *n_edges)
{
    int64_t total = in_off[n_tx] + out_off[n_tx];
    orc_map m;
    m.cap = 16;
    while (m.cap < 2 * total + 16) m.cap <<= 1;
    m.key = (uint64_t *)calloc((size_t)m.cap, sizeof(uint64_t));
    m.val = (int64_t *)calloc((size_t)m.cap, sizeof(int64_t));
    m.used = (unsigned char *)calloc((size_t)m.cap, 1);
    orc_pair *e = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(total > 0 ? total : 1));
    int64_t n_addr = 0, ne = 0;
    for (int64_t t = 0; t < n_tx; ++t) {
        for (int side = 0; side < 2; ++side) {
            const int64_t *off = side == 0 ? in_off : out_off;
            const uint64_t *addr = side == 0 ? in_addr : out_addr;
            for (int64_t k = off[t]; k < off[t + 1]; ++k) {
                int64_t id = orc_map_get(&m, addr[k]);
                if (id < 0) {
                    id = n_addr;
                    addr_out[n_addr++] = addr[k];
                    orc_map_put(&m, addr[k], id);
                }
                int32_t a = (int32_t)(n_tx + id);
                if (side == 0) { e[ne].a = a; e[ne].b = (int32_t)t; }   /* input: address -> tx */
                else { e[ne].a = (int32_t)t; e[ne].b = a; }             /* output: tx -> address */
                ++ne;
            }
        }
    }
    qsort(e, (size_t)ne, sizeof(orc_pair), orc_pair_cmp);
    int64_t w = 0;
    for (int64_t k = 0; k < ne; ++k) {
        if (w > 0 && src_out[w - 1] == e[k].a && dst_out[w - 1] == e[k].b) continue;
        src_out[w] = e[k].a;
        dst_out[w] = e[k].b;
        ++w;
    }
    *n_edges = w;
    free(m.key); free(m.val); free(m.used); free(e);
    return n_addr;
}

/*
 * Undirected simple graph of a directed edge list (directions ignored, as in
 * Section 4): one undirected edge per unordered pair {u, v}, u != v.  Rows
 * of the CSR (off[n+1], adj[2E]) list neighbours in ascending id; the degree
 * of v is off[v+1] - off[v], the number of distinct neighbours.  adj needs
 * room for 2m entries.  Returns E.
 */
int64_t orc_undirected_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                           int64_t *off, int32_t *adj)
{
    orc_pair *p = (orc_pair *)malloc(sizeof(orc_pair) * (size_t)(2 * m > 0 ? 2 * m : 1));
    int64_t np = 0;
    for (int64_t k = 0; k < m; ++k) {
        if (src[k] == dst[k]) continue;
        p[np].a = src[k]; p[np].b = dst[k]; ++np;
        p[np].a = dst[k]; p[np].b = src[k]; ++np;
    }
    qsort(p, (size_t)np, sizeof(orc_pair), orc_pair_cmp);
    for (int64_t v = 0; v <= n; ++v) off[v] = 0;
    int64_t w = 0;
    for (int64_t k = 0; k < np; ++k) {
        if (w > 0 && p[k].a == p[w - 1].a && p[k].b == p[w - 1].b) continue;
        p[w++] = p[k];
    }
    for (int64_t k = 0; k < w; ++k) off[p[k].a + 1] += 1;
    for (int64_t v = 0; v < n; ++v) off[v + 1] += off[v];
    for (int64_t k = 0; k < w; ++k) adj[k] = p[k].b;   /* rows already in (a, b) order */
    free(p);
    return w / 2;
}

/* ------------------------------------------------------------------ */
/* Section 4: components                                                */
/* ------------------------------------------------------------------ */

static int64_t orc_find(int64_t *parent, int64_t v)
{
    while (parent[v] != v) {
        parent[v] = parent[parent[v]];
        v = parent[v];
    }
    return v;
}

/* Connected components by union-find; label = smallest node id of the component. */
int64_t orc_components(int64_t n, const int64_t *off, const int32_t *adj, int32_t *label)
{
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; ++v) parent[v] = v;
    for (int64_t v = 0; v < n; ++v)
        for (int64_t k = off[v]; k < off[v + 1]; ++k) {
            int64_t a = orc_find(parent, v), b = orc_find(parent, adj[k]);
            if (a != b) {
                if (a < b) parent[b] = a;
                else parent[a] = b;
            }
        }
    int64_t nc = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t r = orc_find(parent, v);
        label[v] = (int32_t)r;     /* the root is always the smallest id: unions keep the smaller root */
        if (r == v) ++nc;
    }
    free(parent);
    return nc;
}

typedef struct { int64_t size; int32_t label; } orc_comp;

static int orc_comp_cmp(const void *p, const void *q)
{
    const orc_comp *x = (const orc_comp *)p, *y = (const orc_comp *)q;
    if (x->size != y->size) return x->size > y->size ? -1 : 1;   /* larger first */
    if (x->label != y->label) return x->label < y->label ? -1 : 1;
    return 0;
}

/*
 * Components in the order used for the size split (Section 4): by node
 * count descending, then by label ascending.  comp_off[c]..comp_off[c+1]
 * indexes nodes[] for component c; nodes of a component in ascending id.
 * comp_label[c] receives the component's label.  Returns the count.
 */
int64_t orc_component_order(int64_t n, const int32_t *label, int64_t *comp_off, int32_t *comp_label,
                            int32_t *nodes)
{
    int64_t *size = (int64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
    for (int64_t v = 0; v < n; ++v) size[label[v]] += 1;
    int64_t nc = 0;
    for (int64_t v = 0; v < n; ++v) if (size[v] > 0) ++nc;
    orc_comp *c = (orc_comp *)malloc(sizeof(orc_comp) * (size_t)(nc > 0 ? nc : 1));
    int64_t k = 0;
    for (int64_t v = 0; v < n; ++v) if (size[v] > 0) { c[k].size = size[v]; c[k].label = (int32_t)v; ++k; }
    qsort(c, (size_t)nc, sizeof(orc_comp), orc_comp_cmp);
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    comp_off[0] = 0;
    for (int64_t i = 0; i < nc; ++i) {
        comp_label[i] = c[i].label;
        comp_off[i + 1] = comp_off[i] + c[i].size;
        slot[c[i].label] = comp_off[i];
    }
    for (int64_t v = 0; v < n; ++v) nodes[slot[label[v]]++] = (int32_t)v;
    free(size); free(c); free(slot);
    return nc;
}

/* ------------------------------------------------------------------ */
/* Section 3.1: graph distances                                         */
/* ------------------------------------------------------------------ */

/* BFS from every node of a graph given by CSR (local ids 0..n-1).
 * d[s*n + v] = hop distance, -1 if unreachable.  Unit weights make this equal
 * to Floyd-Warshall's all-pairs shortest paths. */
void orc_bfs_apsp(int64_t n, const int64_t *off, const int32_t *adj, int32_t *d)
{
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t s = 0; s < n; ++s) {
        int32_t *row = d + s * n;
        for (int64_t v = 0; v < n; ++v) row[v] = -1;
        int64_t head = 0, tail = 0;
        row[s] = 0;
        queue[tail++] = (int32_t)s;
        while (head < tail) {
            int32_t v = queue[head++];
            for (int64_t k = off[v]; k < off[v + 1]; ++k) {
                int32_t w = adj[k];
                if (row[w] < 0) {
                    row[w] = row[v] + 1;
                    queue[tail++] = w;
                }
            }
        }
    }
    free(queue);
}

/* Floyd-Warshall all-pairs shortest paths with unit edge weights (Section 3.1). */
void orc_floyd_warshall(int64_t n, const int64_t *off, const int32_t *adj, int32_t *d)
{
    const int32_t INF = 1 << 29;
    for (int64_t i = 0; i < n * n; ++i) d[i] = INF;
    for (int64_t i = 0; i < n; ++i) {
        d[i * n + i] = 0;
        for (int64_t k = off[i]; k < off[i + 1]; ++k) d[i * n + adj[k]] = 1;
    }
    for (int64_t k = 0; k < n; ++k)
        for (int64_t i = 0; i < n; ++i)
            for (int64_t j = 0; j < n; ++j)
                if (d[i * n + k] + d[k * n + j] < d[i * n + j]) d[i * n + j] = d[i * n + k] + d[k * n + j];
    for (int64_t i = 0; i < n * n; ++i) if (d[i] >= INF) d[i] = -1;
}

/* ------------------------------------------------------------------ */
/* Section 3.1: Kamada-Kawai                                             */
/* ------------------------------------------------------------------ */

/* E = sum_{i<j} d_ij^-2 (|p_i - p_j| - l d_ij)^2 over pairs with d_ij > 0. */
double orc_kk_energy(int64_t n, const double *x, const double *y, const int32_t *d, double l)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            int32_t dij = d[i * n + j];
            if (dij <= 0) continue;
            double r = hypot(x[i] - x[j], y[i] - y[j]);
            double t = r - l * dij;
            e += t * t / ((double)dij * dij);
        }
    return e;
}

/*
 * Half-gradient and half-Hessian of the KK energy with respect to p_m
 * (the common factor 2 cancels in the Newton step):
 *   g   = sum_i k (dx - l_mi dx / r, dy - l_mi dy / r)
 *   Hxx = sum_i k (1 - l_mi dy^2 / r^3),  Hyy = sum_i k (1 - l_mi dx^2 / r^3),
 *   Hxy = sum_i k l_mi dx dy / r^3,
 * with dx = x_m - x_i, dy = y_m - y_i, r = |p_m - p_i|, k = d_mi^-2,
 * l_mi = l d_mi.  A coincident pair (r = 0) is skipped.
 * out = {gx, gy, Hxx, Hxy, Hyy}.
 */
void orc_kk_grad_hess(int64_t n, const double *x, const double *y, const int32_t *d, double l,
                      int64_t m, double *out)
{
    double gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i == m) continue;
        int32_t dmi = d[m * n + i];
        if (dmi <= 0) continue;
        double dx = x[m] - x[i], dy = y[m] - y[i];
        double r = sqrt(dx * dx + dy * dy);
        if (r == 0.0) continue;
        double k = 1.0 / ((double)dmi * dmi);
        double lm = l * dmi;
        double r3 = r * r * r;
        gx += k * (dx - lm * dx / r);
        gy += k * (dy - lm * dy / r);
        hxx += k * (1.0 - lm * dy * dy / r3);
        hyy += k * (1.0 - lm * dx * dx / r3);
        hxy += k * lm * dx * dy / r3;
    }
    out[0] = gx; out[1] = gy; out[2] = hxx; out[3] = hxy; out[4] = hyy;
}

/*
 * One safeguarded Newton-Raphson step for node m (the minimisation step of
 * Section 3.1): with g the half-gradient and H = l1 P1 + l2 P2 the symmetric
 * 2x2 half-Hessian (eigenvalues l1 >= l2, P1, P2 the orthogonal projectors
 * onto their eigenvectors), the step is
 *   delta = -(P1 g / e1 + P2 g / e2),
 *   e_i = l_i if l_i > 1e-12 max|l|, else max(|l_i|, 0.1 max|l|),
 * shortened to length l when longer.  Where H is positive definite and the
 * step is shorter than l this is the plain Newton step; elsewhere the
 * directions of non-positive curvature are treated as positive (the plain
 * step there climbs the energy and throws nodes away from random starts).
 * H = 0 gives no step (returns 0).  o = {g_x, g_y, H_xx, H_xy, H_yy}.
 */
int orc_kk_step(const double *o, double l, double *dxm, double *dym)
{
    double gx = o[0], gy = o[1], a = o[2], b = o[3], c = o[4];
    double tr = 0.5 * (a + c);
    double dd = hypot(0.5 * (a - c), b);
    double l1 = tr + dd, l2 = tr - dd;
    double big = fabs(l1) > fabs(l2) ? fabs(l1) : fabs(l2);
    if (big == 0.0) return 0;
    double fl = 0.1 * big;
    double e1 = l1 > 1e-12 * big ? l1 : (fabs(l1) > fl ? fabs(l1) : fl);
    double e2 = l2 > 1e-12 * big ? l2 : (fabs(l2) > fl ? fabs(l2) : fl);
    double sx, sy;
    if (dd == 0.0) {            /* H = tr I */
        sx = -gx / e1;
        sy = -gy / e1;
    } else {
        /* P1 = (H - l2 I) / (l1 - l2),  P2 = I - P1, with l1 - l2 = 2 dd and
           a - l2 = (a - c)/2 + dd, c - l2 = (c - a)/2 + dd */
        double h = 0.5 * (a - c);
        double p1x = ((h + dd) * gx + b * gy) / (2.0 * dd);
        double p1y = (b * gx + (dd - h) * gy) / (2.0 * dd);
        double p2x = gx - p1x, p2y = gy - p1y;
        sx = -(p1x / e1 + p2x / e2);
        sy = -(p1y / e1 + p2y / e2);
    }
    double len = hypot(sx, sy);
    if (len > l) {
        sx *= l / len;
        sy *= l / len;
    }
    *dxm = sx;
    *dym = sy;
    return 1;
}

/*
 * Newton-Raphson minimisation of the KK energy (Section 3.1), Gauss-Seidel
 * order: one sweep visits m = 0..n-1 and moves p_m by orc_kk_step, using
 * positions already moved in this sweep.  `sweeps` sweeps are run; if
 * tol > 0 the run stops after a sweep in which every node had |g| < tol.
 * energy (may be NULL) receives the energy after each sweep.
 * Returns the number of node steps skipped (H = 0); *sweeps_done the sweeps run.
 */
int64_t orc_kk_run(int64_t n, double *x, double *y, const int32_t *d, double l, int64_t sweeps,
                   double tol, double *energy, int64_t *sweeps_done)
{
    int64_t skipped = 0, s = 0;
    for (s = 0; s < sweeps; ++s) {
        double gmax = 0.0;
        for (int64_t m = 0; m < n; ++m) {
            double o[5], dxm, dym;
            orc_kk_grad_hess(n, x, y, d, l, m, o);
            double gn = hypot(o[0], o[1]);
            if (gn > gmax) gmax = gn;
            if (!orc_kk_step(o, l, &dxm, &dym)) { ++skipped; continue; }
            x[m] += dxm;
            y[m] += dym;
        }
        if (energy) energy[s] = orc_kk_energy(n, x, y, d, l);
        if (tol > 0.0 && gmax < tol) { ++s; break; }
    }
    if (sweeps_done) *sweeps_done = s;
    return skipped;
}

/* ------------------------------------------------------------------ */
/* Section 4: assembly of the component layouts                          */
/* ------------------------------------------------------------------ */

/*
 * Kamada-Kawai on a graph whose pair distances d_ij are real (the path
 * lengths of the weighted tree of components): energy
 *   E = sum_{i<j} d_ij^-2 (|p_i - p_j| - d_ij)^2,
 * i.e. the Section 3.1 energy with l d_ij replaced by the weighted d_ij.
 */
double orc_kkw_energy(int64_t n, const double *x, const double *y, const double *d)
{
    double e = 0.0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double dij = d[i * n + j];
            if (!(dij > 0.0)) continue;
            double t = hypot(x[i] - x[j], y[i] - y[j]) - dij;
            e += t * t / (dij * dij);
        }
    return e;
}

/* half-gradient and half-Hessian with respect to p_m, as orc_kk_grad_hess
   with k = d_mi^-2 and l_mi = d_mi */
void orc_kkw_grad_hess(int64_t n, const double *x, const double *y, const double *d, int64_t m, double *out)
{
    double gx = 0, gy = 0, hxx = 0, hxy = 0, hyy = 0;
    for (int64_t i = 0; i < n; ++i) {
        if (i == m) continue;
        double dmi = d[m * n + i];
        if (!(dmi > 0.0)) continue;
        double dx = x[m] - x[i], dy = y[m] - y[i];
        double r = sqrt(dx * dx + dy * dy);
        if (r == 0.0) continue;
        double k = 1.0 / (dmi * dmi);
        double r3 = r * r * r;
        gx += k * (dx - dmi * dx / r);
        gy += k * (dy - dmi * dy / r);
        hxx += k * (1.0 - dmi * dy * dy / r3);
        hyy += k * (1.0 - dmi * dx * dx / r3);
        hxy += k * dmi * dx * dy / r3;
    }
    out[0] = gx; out[1] = gy; out[2] = hxx; out[3] = hxy; out[4] = hyy;
}

/* Gauss-Seidel sweeps of the safeguarded Newton step (orc_kk_step), steps
   capped at `cap`; returns the node steps skipped */
int64_t orc_kkw_run(int64_t n, double *x, double *y, const double *d, double cap, int64_t sweeps, double *energy)
{
    int64_t skipped = 0;
    for (int64_t s = 0; s < sweeps; ++s) {
        for (int64_t m = 0; m < n; ++m) {
            double o[5], dxm, dym;
            orc_kkw_grad_hess(n, x, y, d, m, o);
            if (!orc_kk_step(o, cap, &dxm, &dym)) { ++skipped; continue; }
            x[m] += dxm;
            y[m] += dym;
        }
        if (energy) energy[s] = orc_kkw_energy(n, x, y, d);
    }
    return skipped;
}

/*
 * Path lengths in a tree given by parent links (parent[k] < k, -1 for the
 * root k = 0) and edge lengths len[k] (edge k - parent[k]): d[i * m + j],
 * by walking from every node, plainly O(m^2).
 */
void orc_tree_distances(int64_t m, const int64_t *parent, const double *len, double *d)
{
    for (int64_t i = 0; i < m * m; ++i) d[i] = -1.0;
    for (int64_t s = 0; s < m; ++s) {
        d[s * m + s] = 0.0;
        /* repeat relaxations along tree edges until nothing changes */
        int changed = 1;
        while (changed) {
            changed = 0;
            for (int64_t k = 1; k < m; ++k) {
                int64_t p = parent[k];
                double a = d[s * m + k], b = d[s * m + p];
                if (b >= 0.0 && a < 0.0) { d[s * m + k] = b + len[k]; changed = 1; }
                if (a >= 0.0 && b < 0.0) { d[s * m + p] = a + len[k]; changed = 1; }
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Section 3.2: ForceAtlas2 forces                                      */
/* ------------------------------------------------------------------ */

/*
 * Forces on the targets tgt[0..nt) (local ids; NULL = all n nodes) of one
 * component with positions (x, y), masses m = degree + 1 and CSR (off, adj):
 *   repulsion  F_rep(i)  = kr m_i sum_{j != i} m_j (p_i - p_j) / |p_i - p_j|^2
 *              (a coincident pair contributes nothing)
 *   attraction F_att(i)  = - sum_{j in N(i)} (p_i - p_j)
 *   gravity    F_grav(i) = - kg m_i p_i
 * Outputs are indexed by target position k (0..nt).  sabs[k] (may be NULL)
 * is the sum of the magnitudes of every individual contribution, the scale
 * used for relative force errors; srep[k] (may be NULL) the same sum over
 * the repulsion terms only, kr m_i sum_j m_j / |p_i - p_j|, the scale of the
 * Fast Multipole error (Section 3.2.1).
 */
void orc_fa2_forces(int64_t n, const double *x, const double *y, const double *mass,
                    const int64_t *off, const int32_t *adj, double kr, double kg,
                    int64_t nt, const int64_t *tgt, double *frx, double *fry, double *fax,
                    double *fay, double *fgx, double *fgy, double *sabs, double *srep)
{
    if (!tgt) nt = n;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < nt; ++k) {
        int64_t i = tgt ? tgt[k] : k;
        double rx = 0, ry = 0, ax = 0, ay = 0, s = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j];
            double d2 = dx * dx + dy * dy;
            if (d2 == 0.0) continue;
            double w = kr * mass[i] * mass[j] / d2;
            rx += w * dx;
            ry += w * dy;
            s += kr * mass[i] * mass[j] / sqrt(d2);
        }
        if (srep) srep[k] = s;
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            int64_t j = adj[e];
            double dx = x[i] - x[j], dy = y[i] - y[j];
            ax -= dx;
            ay -= dy;
            s += sqrt(dx * dx + dy * dy);
        }
        double gx = -kg * mass[i] * x[i], gy = -kg * mass[i] * y[i];
        s += sqrt(gx * gx + gy * gy);
        frx[k] = rx; fry[k] = ry;
        fax[k] = ax; fay[k] = ay;
        fgx[k] = gx; fgy[k] = gy;
        if (sabs) sabs[k] = s;
    }
}

/*
 * Layout energy whose negative gradient is the force above:
 *   E = 1/2 sum_{edges} |p_i - p_j|^2 - kr sum_{i<j} m_i m_j ln |p_i - p_j|
 *       + 1/2 kg sum_i m_i |p_i|^2      (coincident pairs omitted)
 */
double orc_fa2_energy(int64_t n, const double *x, const double *y, const double *mass,
                      const int64_t *off, const int32_t *adj, double kr, double kg)
{
    double e_att = 0, e_rep = 0, e_grav = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t e = off[i]; e < off[i + 1]; ++e) {
            int64_t j = adj[e];
            if (j <= i) continue;
            double dx = x[i] - x[j], dy = y[i] - y[j];
            e_att += 0.5 * (dx * dx + dy * dy);
        }
        for (int64_t j = i + 1; j < n; ++j) {
            double d2 = (x[i] - x[j]) * (x[i] - x[j]) + (y[i] - y[j]) * (y[i] - y[j]);
            if (d2 == 0.0) continue;
            e_rep -= kr * mass[i] * mass[j] * 0.5 * log(d2);
        }
        e_grav += 0.5 * kg * mass[i] * (x[i] * x[i] + y[i] * y[i]);
    }
    return e_att + e_rep + e_grav;
}

/* ------------------------------------------------------------------ */
/* Section 3.2: swing / traction and the position update                */
/* ------------------------------------------------------------------ */

/*
 * `iters` ForceAtlas2 iterations on one component with exact repulsion.
 * State: positions (x, y), previous forces (fpx, fpy; zero before the first
 * iteration) and global speed *sg (1 before the first iteration).
 * Per iteration t:
 *   F_t       = F_rep + F_att + F_grav                (orc_fa2_forces)
 *   variant 0 (as printed in Section 3.2):
 *     swg = sum_n |F_t(n) - F_{t-1}(n)|,  trc = sum_n |F_t(n) + F_{t-1}(n)|
 *   variant 1 (ForceAtlas2): the same sums weighted by m_n, traction halved
 *   s_G       = min(tau trc / swg, 1.5 s_G)   (1.5 s_G when swg = 0)
 *   s_n       = ks s_G / (1 + s_G sqrt(|F_t(n) - F_{t-1}(n)|)),
 *               reduced to ksmax / |F_t(n)| if larger
 *   p_n      += s_n F_t(n);   F_{t-1} <- F_t
 * stats (may be NULL) receives {swg, trc, s_G} per iteration.
 */
void orc_fa2_run(int64_t n, double *x, double *y, const double *mass, const int64_t *off,
                 const int32_t *adj, double kr, double kg, double ks, double ksmax, double tau,
                 int32_t variant, int64_t iters, double *fpx, double *fpy, double *sg, double *stats)
{
    size_t sz = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double *rx = malloc(sz), *ry = malloc(sz), *ax = malloc(sz), *ay = malloc(sz);
    double *gx = malloc(sz), *gy = malloc(sz);
    for (int64_t t = 0; t < iters; ++t) {
        orc_fa2_forces(n, x, y, mass, off, adj, kr, kg, n, NULL, rx, ry, ax, ay, gx, gy, NULL, NULL);
        double swg = 0.0, trc = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            double fx = rx[i] + ax[i] + gx[i], fy = ry[i] + ay[i] + gy[i];
            double sw = hypot(fx - fpx[i], fy - fpy[i]);
            double tr = hypot(fx + fpx[i], fy + fpy[i]);
            if (variant == 1) { swg += mass[i] * sw; trc += 0.5 * mass[i] * tr; }
            else { swg += sw; trc += tr; }
        }
        double s_new = swg > 0.0 ? tau * trc / swg : 1.5 * (*sg);
        if (s_new > 1.5 * (*sg)) s_new = 1.5 * (*sg);
        *sg = s_new;
        for (int64_t i = 0; i < n; ++i) {
            double fx = rx[i] + ax[i] + gx[i], fy = ry[i] + ay[i] + gy[i];
            double sw = hypot(fx - fpx[i], fy - fpy[i]);
            double s = ks * (*sg) / (1.0 + (*sg) * sqrt(sw));
            double fn = hypot(fx, fy);
            if (fn > 0.0 && s > ksmax / fn) s = ksmax / fn;
            x[i] += s * fx;
            y[i] += s * fy;
            fpx[i] = fx;
            fpy[i] = fy;
        }
        if (stats) { stats[3 * t] = swg; stats[3 * t + 1] = trc; stats[3 * t + 2] = *sg; }
    }
    free(rx); free(ry); free(ax); free(ay); free(gx); free(gy);
}

/* number of OpenMP threads the force loop uses (1 without OpenMP) */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
