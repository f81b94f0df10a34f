/*
 * graphgen.c -- seeded synthetic graph generators (inputs only).
 *
 * This module produces the symmetric, self-loop-free, duplicate-free int32 CSR
 * graphs that both the CPU oracle and the GPU library are fed.  It contains no
 * coloring arithmetic at all.  Workload shapes follow the paper's evaluation
 * (Sect. 4, Table 1): R-MAT graphs with (a,b,c,d) parameters, uniform random
 * (Erdos-Renyi style, the paper's "rmat-er") graphs, and regular meshes, for
 * which lattice stencils stand in.
 *
 * Random numbers: splitmix64 (Steele, Lea and Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014) expands the user seed into the
 * 256-bit state of xoshiro256** (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2018).  Both are integer-only, so the same
 * seed yields the same graph on every platform.
 *
 * Every generated row is sorted ascending and holds distinct neighbours.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ PRNG */

typedef struct { uint64_t s[4]; } gg_rng;

static uint64_t gg_splitmix64(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static void gg_seed(gg_rng *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = gg_splitmix64(&x);
}

static inline uint64_t gg_rotl(uint64_t v, int k) { return (v << k) | (v >> (64 - k)); }

static inline uint64_t gg_next(gg_rng *r) {
    uint64_t *s = r->s;
    const uint64_t out = gg_rotl(s[1] * 5u, 7) * 9u;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = gg_rotl(s[3], 45);
    return out;
}

/* uniform integer in [0, bound) by the multiply-high method (Lemire, 2019),
 * without the rejection step: the bias is below 2^-32 for our bounds. */
static inline uint64_t gg_below(gg_rng *r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)gg_next(r) * bound) >> 64);
}

/* exported for the tests: the first outputs of the generator for a seed */
int gg_rng_stream(uint64_t seed, int64_t count, uint64_t *out) {
    gg_rng r;
    gg_seed(&r, seed);
    for (int64_t i = 0; i < count; ++i) out[i] = gg_next(&r);
    return 0;
}

/* ------------------------------------------------------------------ CSR */

typedef struct {
    int32_t n;
    int64_t m;
    int32_t *ro; /* n + 1 */
    int32_t *ci; /* m */
} gg_graph;

/* In-place ascending sort of int32 (quicksort with median-of-three pivots,
 * recursing on the smaller side, insertion sort below 24 elements). */
static void sort_i32(int32_t *a, int64_t n) {
    while (n > 24) {
        int64_t mid = n / 2;
        int32_t x = a[0], y = a[mid], z = a[n - 1];
        int32_t piv = (x < y) ? ((y < z) ? y : ((x < z) ? z : x)) : ((x < z) ? x : ((y < z) ? z : y));
        int64_t i = 0, j = n - 1;
        while (i <= j) {
            while (a[i] < piv) i++;
            while (a[j] > piv) j--;
            if (i <= j) {
                int32_t t = a[i];
                a[i] = a[j];
                a[j] = t;
                i++;
                j--;
            }
        }
        /* [0, j] <= piv <= [i, n) */
        if (j + 1 < n - i) {
            sort_i32(a, j + 1);
            a += i;
            n -= i;
        } else {
            sort_i32(a + i, n - i);
            n = j + 1;
        }
    }
    for (int64_t i = 1; i < n; ++i) {
        int32_t v = a[i];
        int64_t k = i - 1;
        while (k >= 0 && a[k] > v) {
            a[k + 1] = a[k];
            k--;
        }
        a[k + 1] = v;
    }
}

/* Build a symmetric CSR from `cnt` undirected pairs (u[i], v[i]).  Self-loops
 * are dropped, both directions are inserted, rows are sorted and deduplicated.
 * Returns NULL on allocation failure or if the result would not fit int32. */
static gg_graph *gg_from_pairs(int32_t n, int64_t cnt, const int32_t *u, const int32_t *v) {
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    if (!g) return NULL;
    int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!deg) { free(g); return NULL; }
    int64_t tot = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (u[i] == v[i]) continue;
        deg[u[i]]++;
        deg[v[i]]++;
        tot += 2;
    }
    int64_t *pos = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int32_t *tmp = (int32_t *)malloc((size_t)(tot > 0 ? tot : 1) * sizeof(int32_t));
    if (!pos || !tmp) { free(deg); free(pos); free(tmp); free(g); return NULL; }
    pos[0] = 0;
    for (int32_t i = 0; i < n; ++i) pos[i + 1] = pos[i] + deg[i];
    memcpy(deg, pos, ((size_t)n + 1) * sizeof(int64_t)); /* deg now = write cursor */
    for (int64_t i = 0; i < cnt; ++i) {
        if (u[i] == v[i]) continue;
        tmp[deg[u[i]]++] = v[i];
        tmp[deg[v[i]]++] = u[i];
    }
    /* sort + dedupe each row in place, compacting into tmp */
    int64_t w = 0;
    int32_t *ro = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!ro) { free(deg); free(pos); free(tmp); free(g); return NULL; }
    ro[0] = 0;
    for (int32_t i = 0; i < n; ++i) {
        int64_t a = pos[i], b = pos[i + 1];
        if (b - a > 1) sort_i32(tmp + a, b - a);
        int64_t start = w;
        for (int64_t k = a; k < b; ++k) {
            if (k > a && tmp[k] == tmp[k - 1]) continue;
            tmp[w++] = tmp[k];
        }
        if (w > INT32_MAX) { free(deg); free(pos); free(tmp); free(ro); free(g); return NULL; }
        ro[i + 1] = (int32_t)w;
        (void)start;
    }
    free(deg);
    free(pos);
    int32_t *ci = (int32_t *)realloc(tmp, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
    g->n = n;
    g->m = w;
    g->ro = ro;
    g->ci = ci ? ci : tmp;
    return g;
}

void gg_free(void *h) {
    gg_graph *g = (gg_graph *)h;
    if (!g) return;
    free(g->ro);
    free(g->ci);
    free(g);
}

int32_t gg_n(void *h) { return ((gg_graph *)h)->n; }
int64_t gg_m(void *h) { return ((gg_graph *)h)->m; }

/* copy the CSR out into caller buffers of n+1 and m int32 entries */
int gg_export(void *h, int32_t *ro, int32_t *ci) {
    gg_graph *g = (gg_graph *)h;
    memcpy(ro, g->ro, ((size_t)g->n + 1) * sizeof(int32_t));
    if (g->m) memcpy(ci, g->ci, (size_t)g->m * sizeof(int32_t));
    return 0;
}

/* ----------------------------------------------------------- generators */

/* Uniform random graph: `pairs` endpoint pairs drawn uniformly from [0,n)^2,
 * then symmetrised with self-loops and duplicates removed (the paper's
 * rmat-er has a=b=c=d=0.25, which is this distribution). */
void *gg_uniform(int32_t n, int64_t pairs, uint64_t seed) {
    if (n <= 0 || pairs < 0) return NULL;
    gg_rng r;
    gg_seed(&r, seed);
    int32_t *u = (int32_t *)malloc((size_t)(pairs > 0 ? pairs : 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(pairs > 0 ? pairs : 1) * sizeof(int32_t));
    if (!u || !v) { free(u); free(v); return NULL; }
    for (int64_t i = 0; i < pairs; ++i) {
        u[i] = (int32_t)gg_below(&r, (uint64_t)n);
        v[i] = (int32_t)gg_below(&r, (uint64_t)n);
    }
    gg_graph *g = gg_from_pairs(n, pairs, u, v);
    free(u);
    free(v);
    return g;
}

/* R-MAT (Chakrabarti, Zhan and Faloutsos, SDM 2004): each edge descends
 * `scale` levels of the 2^scale x 2^scale adjacency matrix, picking a quadrant
 * with probabilities (a, b, c, 1-a-b-c) given to 16-bit precision (four
 * levels per 64-bit draw).  No noise is added.  An edge with an endpoint at or
 * above n is drawn again, so `draws` edges land in [0, n)^2 (n = 2^scale keeps
 * all of them).  Vertex ids are then relabelled by a seeded Fisher-Yates
 * permutation of [0, n). */
void *gg_rmat(int32_t scale, int32_t n, int64_t draws, double a, double b, double c,
              uint64_t seed) {
    if (scale < 1 || scale > 30) return NULL;
    int64_t N = (int64_t)1 << scale;
    if (n <= 0 || n > N || draws < 0) return NULL;
    gg_rng r;
    gg_seed(&r, seed);
    const uint32_t ta = (uint32_t)(a * 65536.0);
    const uint32_t tb = (uint32_t)((a + b) * 65536.0);
    const uint32_t tc = (uint32_t)((a + b + c) * 65536.0);
    int32_t *u = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    int32_t *v = (int32_t *)malloc((size_t)(draws > 0 ? draws : 1) * sizeof(int32_t));
    int32_t *perm = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!u || !v || !perm) { free(u); free(v); free(perm); return NULL; }
    uint64_t bits = 0;
    int left = 0;
    for (int64_t i = 0; i < draws;) {
        int64_t x = 0, y = 0;
        for (int l = 0; l < scale; ++l) {
            if (left == 0) {
                bits = gg_next(&r);
                left = 4;
            }
            const uint32_t q = (uint32_t)(bits & 0xFFFFu);
            bits >>= 16;
            left--;
            const int bx = q >= tb, by = (q >= ta && q < tb) || q >= tc;
            x = (x << 1) | bx;
            y = (y << 1) | by;
        }
        if (x >= n || y >= n) continue; /* redraw */
        u[i] = (int32_t)x;
        v[i] = (int32_t)y;
        i++;
    }
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)gg_below(&r, (uint64_t)(i + 1));
        int32_t t = perm[i];
        perm[i] = perm[j];
        perm[j] = t;
    }
    for (int64_t i = 0; i < draws; ++i) {
        u[i] = perm[u[i]];
        v[i] = perm[v[i]];
    }
    free(perm);
    gg_graph *g = gg_from_pairs(n, draws, u, v);
    free(u);
    free(v);
    return g;
}

/* Lattice stencil graph on nx*ny*nz points in natural lexicographic order
 * (id = (z*ny + y)*nx + x).  kind: 5 = 2-D 5-point, 9 = 2-D 9-point (nz must
 * be 1), 7 = 3-D 7-point, 27 = 3-D 27-point.  Each point is linked to the
 * stencil offsets that stay inside the box; rows come out sorted. */
void *gg_stencil(int32_t nx, int32_t ny, int32_t nz, int32_t kind) {
    if (nx <= 0 || ny <= 0 || nz <= 0) return NULL;
    if ((kind == 5 || kind == 9) && nz != 1) return NULL;
    if (kind != 5 && kind != 9 && kind != 7 && kind != 27) return NULL;
    int64_t n64 = (int64_t)nx * ny * nz;
    if (n64 > INT32_MAX - 1) return NULL;
    int32_t n = (int32_t)n64;
    /* offsets in increasing id order: dz major, then dy, then dx */
    int dxs[26], dys[26], dzs[26], no = 0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int nnz = (dx != 0) + (dy != 0) + (dz != 0);
                int ok = 0;
                if (kind == 27) ok = 1;
                if (kind == 9) ok = (dz == 0);
                if (kind == 7) ok = (nnz == 1);
                if (kind == 5) ok = (dz == 0 && nnz == 1);
                if (!ok) continue;
                dxs[no] = dx; dys[no] = dy; dzs[no] = dz; no++;
            }
    gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
    int32_t *ro = (int32_t *)malloc(((size_t)n + 1) * sizeof(int32_t));
    if (!g || !ro) { free(g); free(ro); return NULL; }
    int64_t m = 0;
    ro[0] = 0;
    for (int32_t z = 0, id = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x, ++id) {
                for (int k = 0; k < no; ++k) {
                    int32_t X = x + dxs[k], Y = y + dys[k], Z = z + dzs[k];
                    if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                    m++;
                }
                if (m > INT32_MAX) { free(g); free(ro); return NULL; }
                ro[id + 1] = (int32_t)m;
            }
    int32_t *ci = (int32_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
    if (!ci) { free(g); free(ro); return NULL; }
    int64_t w = 0;
    for (int32_t z = 0; z < nz; ++z)
        for (int32_t y = 0; y < ny; ++y)
            for (int32_t x = 0; x < nx; ++x)
                for (int k = 0; k < no; ++k) {
                    int32_t X = x + dxs[k], Y = y + dys[k], Z = z + dzs[k];
                    if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
                    ci[w++] = (Z * ny + Y) * nx + X;
                }
    g->n = n;
    g->m = m;
    g->ro = ro;
    g->ci = ci;
    return g;
}

/* Symmetric CSR from caller pairs (for hand-built test graphs). */
void *gg_from_edges(int32_t n, int64_t cnt, const int32_t *u, const int32_t *v) {
    if (n < 0) return NULL;
    for (int64_t i = 0; i < cnt; ++i)
        if (u[i] < 0 || v[i] < 0 || u[i] >= n || v[i] >= n) return NULL;
    if (n == 0) {
        gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
        if (!g) return NULL;
        g->ro = (int32_t *)calloc(1, sizeof(int32_t));
        g->ci = (int32_t *)calloc(1, sizeof(int32_t));
        return g;
    }
    return gg_from_pairs(n, cnt, u, v);
}
