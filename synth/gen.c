/*
 * Seeded synthetic inputs shaped like the paper's workloads.
 *
 * The paper lays out daily bitcoin transaction graphs (Section 2, Section 4:
 * Fig. 4 with about 1.5e4 nodes, Fig. 5 with about 2e5 nodes).  Those data are
 * not available, so this generator produces transaction lists with the same
 * structure: each transaction has a list of input addresses and a list of
 * output addresses, addresses are reused preferentially, and the bipartite
 * address/transaction graph of Section 2 is built from them by the library
 * (and by the oracle).  This file holds none of the layout method's
 * arithmetic; both the CUDA path and the oracle read what it writes.
 *
 * Pseudo-random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).
 *
 * Transaction recipe:
 *   inputs per tx  : Geometric(1/2) on {1,2,...}, redrawn above 20
 *   outputs per tx : 2 with probability 0.7, else Geometric(1/2), redrawn above 50
 *   each endpoint  : with probability 0.4 reuse an existing address chosen by
 *                    Zipf(s = 1.2) over creation rank (rank 1 = oldest), else a
 *                    new address.  The very first endpoint is always new.
 * Geometric(1/2) is 1 + ctz(u) for a uniform nonzero 64-bit word u.
 * Zipf draws use rejection-inversion (Hoermann and Derflinger, "Rejection-
 * inversion to generate variates from monotone discrete distributions",
 * ACM TOMACS 6(3), 1996) with hat H(x) = (x^(1-s) - 1)/(1-s).
 *
 * Address keys are opaque 64-bit values: key = SplitMix64 finaliser of
 * (creation rank + salt), so they look like hashes and are not ordered by
 * creation.
 *
 * Counts and endpoint choices come from two independent streams so the
 * sizes can be computed without drawing the endpoints.
 */
#include <stdint.h>
#include <math.h>
#include <stdlib.h>

typedef struct { uint64_t s; } sm64;

static uint64_t sm64_next(sm64 *g)
{
    uint64_t z = (g->s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform double in [0,1) with 53 random bits */
static double sm64_u01(sm64 *g) { return (double)(sm64_next(g) >> 11) * 0x1.0p-53; }

static int64_t geo_half(sm64 *g, int64_t maxv)
{
    for (;;) {
        uint64_t u = sm64_next(g);
        if (u == 0) continue;
        int64_t k = 1 + (int64_t)__builtin_ctzll(u);
        if (k <= maxv) return k;
    }
}

static const double ZIPF_S = 1.2;

static double zipf_H(double x) { return (pow(x, 1.0 - ZIPF_S) - 1.0) / (1.0 - ZIPF_S); }
static double zipf_Hinv(double u) { return pow(1.0 + u * (1.0 - ZIPF_S), 1.0 / (1.0 - ZIPF_S)); }
static double zipf_h(double x) { return pow(x, -ZIPF_S); }

/* Zipf(s) on {1..N}: P(k) proportional to k^-s. */
static int64_t zipf_draw(sm64 *g, int64_t N)
{
    const double lo = zipf_H(1.5) - 1.0;            /* so that k = 1 owns mass h(1) = 1 */
    const double hi = zipf_H((double)N + 0.5);
    for (;;) {
        double u = hi + sm64_u01(g) * (lo - hi);    /* uniform in (lo, hi] */
        double x = zipf_Hinv(u);
        int64_t k = (int64_t)(x + 0.5);
        if (k < 1) k = 1;
        if (k > N) k = N;
        if (u >= zipf_H((double)k + 0.5) - zipf_h((double)k)) return k;
    }
}

static const uint64_t SALT_COUNTS = 0xC0FFEE0000000001ULL;
static const uint64_t SALT_ENDPTS = 0xE11D0B1A00000002ULL;
static const uint64_t SALT_KEYS = 0xADD4E55000000003ULL;

static uint64_t mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void draw_counts(sm64 *g, int64_t *nin, int64_t *nout)
{
    *nin = geo_half(g, 20);
    if (sm64_u01(g) < 0.7) *nout = 2;
    else *nout = geo_half(g, 50);
}

/* Total inputs and outputs of the n_tx transactions for this seed. */
void synth_tx_sizes(uint64_t seed, int64_t n_tx, int64_t *n_in, int64_t *n_out)
{
    sm64 gc = { seed ^ SALT_COUNTS };
    int64_t a = 0, b = 0;
    for (int64_t t = 0; t < n_tx; ++t) {
        int64_t i, o;
        draw_counts(&gc, &i, &o);
        a += i;
        b += o;
    }
    *n_in = a;
    *n_out = b;
}

/* Fill CSR lists: in_off[n_tx+1], in_addr[n_in], out_off[n_tx+1], out_addr[n_out].
 * Returns the number of distinct addresses created. */
int64_t synth_tx_generate(uint64_t seed, int64_t n_tx, int64_t *in_off, uint64_t *in_addr,
                          int64_t *out_off, uint64_t *out_addr)
{
    sm64 gc = { seed ^ SALT_COUNTS };
    sm64 ge = { seed ^ SALT_ENDPTS };
    int64_t n_addr = 0;
    in_off[0] = 0;
    out_off[0] = 0;
    for (int64_t t = 0; t < n_tx; ++t) {
        int64_t ni, no;
        draw_counts(&gc, &ni, &no);
        in_off[t + 1] = in_off[t] + ni;
        out_off[t + 1] = out_off[t] + no;
        for (int64_t e = 0; e < ni + no; ++e) {
            int64_t rank;
            if (n_addr > 0 && sm64_u01(&ge) < 0.4) {
                rank = zipf_draw(&ge, n_addr);
            } else {
                rank = ++n_addr;
            }
            uint64_t key = mix64((uint64_t)rank + (seed ^ SALT_KEYS));
            if (e < ni) in_addr[in_off[t] + e] = key;
            else out_addr[out_off[t] + (e - ni)] = key;
        }
    }
    return n_addr;
}

/*
 * Batched small components (forest of independent components).
 * Component sizes n = round(exp(U[ln a, ln b])).  Each component is a random
 * recursive tree (node k > 0 attaches to a uniform j < k) plus
 * round(0.1 (n - 1)) extra distinct edges between distinct nodes that are not
 * already adjacent (fewer if the component is too dense to hold them).
 * Node ids are consecutive per component.
 */
void synth_forest_sizes(uint64_t seed, int64_t n_comp, double a, double b, int64_t *sizes,
                        int64_t *n_nodes, int64_t *n_edges)
{
    sm64 g = { seed ^ SALT_COUNTS };
    int64_t nn = 0, ne = 0;
    for (int64_t c = 0; c < n_comp; ++c) {
        double u = sm64_u01(&g);
        int64_t n = (int64_t)llround(exp(log(a) + u * (log(b) - log(a))));
        if (n < 1) n = 1;
        sizes[c] = n;
        int64_t extra = (int64_t)llround(0.1 * (double)(n - 1));
        int64_t room = n * (n - 1) / 2 - (n - 1);
        if (extra > room) extra = room;
        nn += n;
        ne += (n - 1) + extra;
    }
    *n_nodes = nn;
    *n_edges = ne;
}

/* open-addressing set of unordered pairs, local to one component */
typedef struct { uint64_t *slot; int64_t cap; } pairset;

static uint64_t pair_key(int32_t a, int32_t b)
{
    uint32_t lo = (uint32_t)(a < b ? a : b), hi = (uint32_t)(a < b ? b : a);
    return ((uint64_t)hi << 32 | lo) + 1;   /* +1 keeps 0 as the empty marker */
}

static int pairset_insert(pairset *s, uint64_t k)    /* 1 if newly inserted */
{
    uint64_t h = mix64(k) & (uint64_t)(s->cap - 1);
    while (s->slot[h] != 0) {
        if (s->slot[h] == k) return 0;
        h = (h + 1) & (uint64_t)(s->cap - 1);
    }
    s->slot[h] = k;
    return 1;
}

/* Edges (u[e], v[e]) with global node ids; sizes[] from synth_forest_sizes. */
void synth_forest_edges(uint64_t seed, int64_t n_comp, const int64_t *sizes, int32_t *u, int32_t *v)
{
    sm64 g = { seed ^ SALT_ENDPTS };
    int64_t base = 0, e = 0;
    for (int64_t c = 0; c < n_comp; ++c) {
        int64_t n = sizes[c];
        int64_t extra = (int64_t)llround(0.1 * (double)(n - 1));
        int64_t room = n * (n - 1) / 2 - (n - 1);
        if (extra > room) extra = room;
        pairset s;
        s.cap = 16;
        while (s.cap < 4 * (n + extra)) s.cap <<= 1;
        s.slot = (uint64_t *)calloc((size_t)s.cap, sizeof(uint64_t));
        for (int64_t k = 1; k < n; ++k) {
            int64_t j = (int64_t)(sm64_u01(&g) * (double)k);
            u[e] = (int32_t)(base + j);
            v[e] = (int32_t)(base + k);
            pairset_insert(&s, pair_key(u[e], v[e]));
            ++e;
        }
        for (int64_t x = 0; x < extra;) {
            int32_t a = (int32_t)(base + (int64_t)(sm64_u01(&g) * (double)n));
            int32_t b = (int32_t)(base + (int64_t)(sm64_u01(&g) * (double)n));
            if (a == b || !pairset_insert(&s, pair_key(a, b))) continue;
            u[e] = a;
            v[e] = b;
            ++e;
            ++x;
        }
        free(s.slot);
        base += n;
    }
}

/* Test hooks of the two samplers above (the generator's own streams are
 * unchanged by them): the first n outputs of SplitMix64 from state `seed`,
 * and n Zipf(1.2) draws on {1..N} from the stream with state `seed`. */
void synth_splitmix64_stream(uint64_t seed, int64_t n, uint64_t *out)
{
    sm64 g = { seed };
    for (int64_t i = 0; i < n; ++i) out[i] = sm64_next(&g);
}

void synth_zipf_sample(uint64_t seed, int64_t N, int64_t n, int64_t *out)
{
    sm64 g = { seed };
    for (int64_t i = 0; i < n; ++i) out[i] = zipf_draw(&g, N);
}
