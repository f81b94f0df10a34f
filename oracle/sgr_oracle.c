/*
 * sgr_oracle.c -- plain CPU oracle for speculative-greedy graph coloring.
 *
 * TEST INFRASTRUCTURE.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg may load this code.  It shares nothing with the GPU
 * library: no headers, no helpers, no tables.
 *
 * It computes, slowly and literally:
 *   - orc_serial_greedy: the sequential first-fit greedy of Algorithm 1
 *     (Sect. 2.1): vertices in order 0..n-1, each taking the smallest color
 *     i > 0 not held by a neighbour, found with a colorMask array stamped with
 *     the current vertex id (initial stamp value -1, which is not a vertex).
 *   - orc_det_sgr: the data-driven speculative greedy loop of Algorithm 7
 *     (Sect. 3.1) with FirstFit (Algorithm 4) and ConflictResolve
 *     (Algorithm 5), made deterministic by two readings:
 *       * every FirstFit of a round reads the colors frozen at the start of
 *         that round (vertices on the worklist hold 0 there);
 *       * conflicts are judged after all tentative colors of the round are
 *         written, before any is cleared; of two neighbours holding the same
 *         color, the one that loses under `rule` is cleared to 0 and pushed
 *         onto the next worklist (Algorithm 5's clearing, Sect. 3.1 "Color
 *         Clearing").
 *     rule ORC_RULE_LOW_KEEPS: the lower vertex id keeps its color.
 *     rule ORC_RULE_LOW_LOSES: the lower id is recolored, as printed in
 *       Algorithm 2 and Algorithm 5 (v < w => color[v] <- 0).
 *     rule ORC_RULE_DEGREE: the heuristic of Sect. 3.2 ("Heuristic Conflict
 *       Resolve"): the larger degree keeps its color; on equal degree the
 *       smaller vertex id keeps it.
 *     The next worklist is kept in ascending vertex order.
 *   - orc_check: counts monochrome adjacencies and out-of-range colors.
 *
 * Colors are 1..k; 0 means uncolored (Sect. 2.1).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_RULE_LOW_KEEPS = 0, ORC_RULE_LOW_LOSES = 1, ORC_RULE_DEGREE = 2 };
enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_NOMEM = -3, ORC_ERR_NO_CONVERGENCE = -5 };

typedef struct {
    int64_t rounds;       /* iterations of the while loop of Algorithm 7 */
    int64_t sum_w;        /* sum over rounds of |W_r| */
    int64_t sum_d;        /* sum over rounds of the degrees of W_r (edges scanned by FirstFit) */
    int64_t sum_d_low;    /* sum over rounds of the lower-id neighbours of W_r */
    int64_t sum_next;     /* sum over rounds of |W_{r+1}| */
    int32_t num_colors;   /* max color */
    int32_t max_degree;
} orc_stats;

static int32_t max_degree(int32_t n, const int32_t *ro) {
    int32_t d = 0;
    for (int32_t v = 0; v < n; ++v)
        if (ro[v + 1] - ro[v] > d) d = ro[v + 1] - ro[v];
    return d;
}

/* Algorithm 1.  Returns the number of colors (max color), 0 for n == 0. */
int32_t orc_serial_greedy(int32_t n, const int32_t *ro, const int32_t *ci, int32_t *color) {
    if (n <= 0) return 0;
    int32_t maxd = max_degree(n, ro);
    int32_t *colorMask = (int32_t *)malloc(((size_t)maxd + 2) * sizeof(int32_t));
    if (!colorMask) return ORC_ERR_NOMEM;
    for (int32_t i = 0; i < maxd + 2; ++i) colorMask[i] = -1;
    for (int32_t v = 0; v < n; ++v) color[v] = 0;
    int32_t k = 0;
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t e = ro[v]; e < ro[v + 1]; ++e) {
            int32_t cw = color[ci[e]];
            if (cw <= maxd + 1) colorMask[cw] = v; /* colors above deg(v)+1 cannot matter */
        }
        int32_t c = 1;
        while (colorMask[c] == v) ++c;
        color[v] = c;
        if (c > k) k = c;
    }
    free(colorMask);
    return k;
}

static int loses(int rule, int32_t v, int32_t w, const int32_t *ro) {
    if (rule == ORC_RULE_LOW_KEEPS) return w < v;
    if (rule == ORC_RULE_LOW_LOSES) return v < w;
    int32_t dv = ro[v + 1] - ro[v], dw = ro[w + 1] - ro[w];
    if (dw != dv) return dw > dv;
    return w < v;
}

/*
 * Algorithm 7 under the readings above.  `max_rounds` <= 0 means n + 1.
 * trace_w / trace_d (optional, capacity trace_cap) receive |W_r| and the
 * degree sum of W_r per round.  Returns ORC_OK or ORC_ERR_NO_CONVERGENCE.
 */
int orc_det_sgr(int32_t n, const int32_t *ro, const int32_t *ci, int rule, int64_t max_rounds,
                int32_t *color, orc_stats *st, int64_t *trace_w, int64_t *trace_d,
                int64_t trace_cap) {
    memset(st, 0, sizeof(*st));
    if (n < 0 || (rule != ORC_RULE_LOW_KEEPS && rule != ORC_RULE_LOW_LOSES && rule != ORC_RULE_DEGREE))
        return ORC_ERR_ARG;
    if (n == 0) return ORC_OK;
    if (max_rounds <= 0) max_rounds = (int64_t)n + 1;
    int32_t maxd = max_degree(n, ro);
    st->max_degree = maxd;
    int32_t *F = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *tent = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *W = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *Lose = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *colorMask = (int32_t *)malloc(((size_t)maxd + 2) * sizeof(int32_t));
    if (!F || !tent || !W || !Lose || !colorMask) {
        free(F); free(tent); free(W); free(Lose); free(colorMask);
        return ORC_ERR_NOMEM;
    }
    for (int32_t i = 0; i < maxd + 2; ++i) colorMask[i] = -1;
    for (int32_t v = 0; v < n; ++v) { color[v] = 0; W[v] = v; }
    int64_t nw = n;
    int rc = ORC_OK;
    while (nw > 0) {
        if (st->rounds == max_rounds) { rc = ORC_ERR_NO_CONVERGENCE; break; }
        st->rounds++;
        memcpy(F, color, (size_t)n * sizeof(int32_t));
        int64_t d = 0, dlow = 0;
        /* FirstFit (Algorithm 4) on the frozen colors F */
        for (int64_t i = 0; i < nw; ++i) {
            int32_t v = W[i];
            for (int32_t e = ro[v]; e < ro[v + 1]; ++e) {
                int32_t cw = F[ci[e]];
                if (cw <= maxd + 1) colorMask[cw] = v;
                if (ci[e] < v) dlow++;
            }
            d += ro[v + 1] - ro[v];
            int32_t c = 1;
            while (colorMask[c] == v) ++c;
            tent[v] = c;
        }
        for (int64_t i = 0; i < nw; ++i) color[W[i]] = tent[W[i]];
        /* ConflictResolve (Algorithm 5), judged on the committed colors */
        int64_t nl = 0;
        for (int64_t i = 0; i < nw; ++i) {
            int32_t v = W[i];
            int conflict = 0;
            for (int32_t e = ro[v]; e < ro[v + 1] && !conflict; ++e) {
                int32_t w = ci[e];
                if (color[w] == color[v] && loses(rule, v, w, ro)) conflict = 1;
            }
            if (conflict) Lose[nl++] = v; /* W ascending => Lose ascending */
        }
        for (int64_t i = 0; i < nl; ++i) color[Lose[i]] = 0;
        if (trace_w && st->rounds <= trace_cap) trace_w[st->rounds - 1] = nw;
        if (trace_d && st->rounds <= trace_cap) trace_d[st->rounds - 1] = d;
        st->sum_w += nw;
        st->sum_d += d;
        st->sum_d_low += dlow;
        st->sum_next += nl;
        memcpy(W, Lose, (size_t)nl * sizeof(int32_t));
        nw = nl;
    }
    int32_t k = 0;
    for (int32_t v = 0; v < n; ++v)
        if (color[v] > k) k = color[v];
    st->num_colors = k;
    free(F); free(tent); free(W); free(Lose); free(colorMask);
    return rc;
}

/*
 * Validity of a coloring (Sect. 2: no two neighbouring vertices share a
 * color).  Returns the number of directed CSR entries (v, w) with
 * color[v] == color[w]; *bad_range receives the number of vertices whose
 * color is outside [1, k] where k = max color, and *k_out the max color.
 */
int64_t orc_check(int32_t n, const int32_t *ro, const int32_t *ci, const int32_t *color,
                  int64_t *bad_range, int32_t *k_out) {
    int64_t mono = 0, bad = 0;
    int32_t k = 0;
    for (int32_t v = 0; v < n; ++v)
        if (color[v] > k) k = color[v];
    for (int32_t v = 0; v < n; ++v) {
        if (color[v] < 1 || color[v] > k) bad++;
        for (int32_t e = ro[v]; e < ro[v + 1]; ++e)
            if (color[ci[e]] == color[v]) mono++;
    }
    if (bad_range) *bad_range = bad;
    if (k_out) *k_out = k;
    return mono;
}
