/*
 * motif.c -- fast twin of workloads.graphs.motif_graph_py (the motif graphs
 * of the batched and serving workloads).  It draws the same splitmix64
 * values in the same order and makes the same choices, so for equal inputs
 * it returns the same graph, edge for edge; a CPU test checks that.  Input
 * generation only: no payload, condition hash or digest of the task-graph
 * method is in here.
 *
 * Build: gcc -O2 -shared -fPIC -o libmotif.so motif.c -lm
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define WL_K 12            /* candidates drawn per row before the fallback */
#define WL_CHUNK (1u << 20) /* rows whose candidates are drawn together */

enum { WL_OK = 0, WL_ERR_SMALL = -1, WL_ERR_CAP = -2, WL_ERR_NOMEM = -3 };

typedef struct {
    uint64_t state, pos;
} wl_stream;

/* splitmix64 output function (Steele, Lea & Flood 2014). */
static uint64_t wl_mix64(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* value i of a stream is mix64(state + (i + 1) * gamma) */
static uint64_t wl_next(wl_stream *s)
{
    s->pos++;
    return wl_mix64(s->state + s->pos * 0x9E3779B97F4A7C15ull);
}

/* integer in [0, span), span <= 2^32: multiply-high of the top 32 bits */
static uint64_t wl_below(wl_stream *s, uint64_t span) { return ((wl_next(s) >> 32) * span) >> 32; }

typedef struct {
    uint64_t key;
    uint32_t idx;
} wl_pair;

static int wl_pair_cmp(const void *a, const void *b)
{
    const wl_pair *x = (const wl_pair *)a, *y = (const wl_pair *)b;
    if (x->key != y->key)
        return x->key < y->key ? -1 : 1;
    return x->idx < y->idx ? -1 : (x->idx > y->idx);
}

static int wl_less(const wl_pair *x, const wl_pair *y)
{
    return x->key < y->key || (x->key == y->key && x->idx < y->idx);
}

/* Move the k smallest pairs (key, then index) to the front, in ascending
 * order: quickselect, then a sort of the front.  Equals the first k entries
 * of a stable argsort of the keys. */
static void wl_smallest(wl_pair *a, uint32_t n, uint32_t k)
{
    if (k == 0 || n == 0)
        return;
    uint32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        /* median of three as pivot */
        if (wl_less(&a[mid], &a[lo])) { wl_pair t = a[mid]; a[mid] = a[lo]; a[lo] = t; }
        if (wl_less(&a[hi], &a[lo])) { wl_pair t = a[hi]; a[hi] = a[lo]; a[lo] = t; }
        if (wl_less(&a[hi], &a[mid])) { wl_pair t = a[hi]; a[hi] = a[mid]; a[mid] = t; }
        const wl_pair pv = a[mid];
        uint32_t i = lo, j = hi;
        while (i <= j) {
            while (wl_less(&a[i], &pv))
                i++;
            while (wl_less(&pv, &a[j]))
                j--;
            if (i <= j) {
                wl_pair t = a[i];
                a[i] = a[j];
                a[j] = t;
                i++;
                if (j == 0)
                    break;
                j--;
            }
        }
        if (k - 1 <= j)
            hi = j;
        else if (k - 1 >= i)
            lo = i;
        else
            break;
    }
    qsort(a, k, sizeof(wl_pair), wl_pair_cmp);
}

/*
 * One motif graph with n tasks and n_c loop motifs (the caller rounds
 * cond_frac * n; it must be >= 1), drawn from the stream (state, pos).
 *   rounds >= 0: every task takes `rounds`; rounds < 0: U{r_lo..r_hi} each
 *   d_lo..d_hi: in-degree range of the layered part; trip_max: trips U{1..}
 * Outputs: kinds[n], params[n], src/dst[edge_cap] (edge count in *m),
 * ks[n_c], anchors[n_c], trips[n_c], *n_d, and *pos_out (the stream's new
 * position).  Returns WL_OK, WL_ERR_SMALL (too few tasks for the motifs),
 * WL_ERR_CAP (edge_cap too small) or WL_ERR_NOMEM.
 */
int wl_motif_graph(uint64_t state, uint64_t pos, uint32_t n, uint32_t n_c, int32_t rounds, uint32_t r_lo,
                   uint32_t r_hi, uint32_t d_lo, uint32_t d_hi, uint32_t trip_max, uint8_t *kinds, uint32_t *params,
                   uint32_t *src, uint32_t *dst, uint64_t edge_cap, uint64_t *m, uint32_t *ks, uint32_t *anchors,
                   uint32_t *trips, uint32_t *n_d_out, uint64_t *pos_out)
{
    wl_stream st = {state, pos};
    uint64_t motif_nodes = 0;
    for (uint32_t i = 0; i < n_c; ++i) {
        ks[i] = 2u + (uint32_t)wl_below(&st, 3);
        motif_nodes += ks[i] + 1u;
    }
    if (motif_nodes > n || n - motif_nodes < n_c)
        return WL_ERR_SMALL;
    const uint32_t n_d = (uint32_t)(n - motif_nodes);
    uint32_t w = (uint32_t)lround(sqrt((double)n_d));
    if (w < 1)
        w = 1;
    uint64_t e = 0;
    /* layered part: every task past the first level draws d distinct
     * predecessors of the level before it (a full level of width w) */
    if (n_d > w) {
        const uint32_t rows = n_d - w;
        uint32_t *d = (uint32_t *)malloc((size_t)rows * sizeof(uint32_t));
        uint32_t *pick = (uint32_t *)malloc((size_t)rows * 8u * sizeof(uint32_t));
        uint64_t *cand = (uint64_t *)malloc((size_t)(rows < WL_CHUNK ? rows : WL_CHUNK) * WL_K * sizeof(uint64_t));
        if (!d || !pick || !cand || d_hi > 8u) {
            free(d);
            free(pick);
            free(cand);
            return WL_ERR_NOMEM;
        }
        for (uint32_t r = 0; r < rows; ++r) {
            uint32_t dd = d_lo + (uint32_t)wl_below(&st, (uint64_t)(d_hi - d_lo + 1u));
            d[r] = dd < w ? dd : w;
        }
        for (uint32_t c0 = 0; c0 < rows; c0 += WL_CHUNK) {
            const uint32_t c1 = rows - c0 < WL_CHUNK ? rows : c0 + WL_CHUNK;
            for (uint64_t i = 0; i < (uint64_t)(c1 - c0) * WL_K; ++i)
                cand[i] = wl_below(&st, w);
            /* the first d distinct candidates in draw order */
            for (uint32_t r = c0; r < c1; ++r) {
                const uint64_t *cr = cand + (uint64_t)(r - c0) * WL_K;
                uint32_t got = 0;
                for (uint32_t j = 0; j < WL_K && got < d[r]; ++j) {
                    int seen = 0;
                    for (uint32_t q = 0; q < got; ++q)
                        if (pick[(uint64_t)r * 8u + q] == (uint32_t)cr[j]) {
                            seen = 1;
                            break;
                        }
                    if (!seen)
                        pick[(uint64_t)r * 8u + got++] = (uint32_t)cr[j];
                }
                if (got < d[r])
                    pick[(uint64_t)r * 8u] = 0xFFFFFFFFu;   /* fallback below */
            }
            /* rows whose candidates held too few distinct values: the first
             * d entries of a random permutation, in row order */
            for (uint32_t r = c0; r < c1; ++r) {
                if (pick[(uint64_t)r * 8u] != 0xFFFFFFFFu || d[r] == 0)
                    continue;
                wl_pair *pp = (wl_pair *)malloc((size_t)w * sizeof(wl_pair));
                if (!pp) {
                    free(d);
                    free(pick);
                    free(cand);
                    return WL_ERR_NOMEM;
                }
                for (uint32_t q = 0; q < w; ++q) {
                    pp[q].key = wl_next(&st);
                    pp[q].idx = q;
                }
                wl_smallest(pp, w, d[r]);
                for (uint32_t q = 0; q < d[r]; ++q)
                    pick[(uint64_t)r * 8u + q] = pp[q].idx;
                free(pp);
            }
        }
        for (uint32_t r = 0; r < rows; ++r) {
            const uint32_t node = w + r;
            const uint32_t prev0 = (node / w - 1u) * w;
            for (uint32_t q = 0; q < d[r]; ++q) {
                if (e >= edge_cap) {
                    free(d);
                    free(pick);
                    free(cand);
                    return WL_ERR_CAP;
                }
                src[e] = prev0 + pick[(uint64_t)r * 8u + q];
                dst[e] = node;
                e++;
            }
        }
        free(d);
        free(pick);
        free(cand);
    }
    /* anchors: n_c distinct layered tasks, the first entries of a random
     * permutation */
    {
        wl_pair *pp = (wl_pair *)malloc((size_t)(n_d ? n_d : 1) * sizeof(wl_pair));
        if (!pp)
            return WL_ERR_NOMEM;
        for (uint32_t q = 0; q < n_d; ++q) {
            pp[q].key = wl_next(&st);
            pp[q].idx = q;
        }
        wl_smallest(pp, n_d, n_c);
        for (uint32_t i = 0; i < n_c; ++i)
            anchors[i] = pp[i].idx;
        free(pp);
    }
    for (uint32_t i = 0; i < n_c; ++i)
        trips[i] = 1u + (uint32_t)wl_below(&st, trip_max);
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t R = rounds >= 0 ? (uint32_t)rounds : r_lo + (uint32_t)wl_below(&st, (uint64_t)(r_hi - r_lo + 1u));
        params[v] = R & 0xFFFFu;
        kinds[v] = 0;
    }
    /* motif i occupies [h, c, arm_1 .. arm_{k-1}] after the layered part */
    const uint64_t need = e + 2ull * n_c + (motif_nodes - n_c);
    if (need > edge_cap)
        return WL_ERR_CAP;
    uint32_t base = n_d;
    for (uint32_t i = 0; i < n_c; ++i) {   /* anchor -> h */
        src[e] = anchors[i];
        dst[e] = base;
        e++;
        base += ks[i] + 1u;
    }
    base = n_d;
    for (uint32_t i = 0; i < n_c; ++i) {   /* h -> c */
        src[e] = base;
        dst[e] = base + 1u;
        e++;
        base += ks[i] + 1u;
    }
    base = n_d;
    for (uint32_t i = 0; i < n_c; ++i) {   /* c -> [h, arms], its successor order */
        const uint32_t c = base + 1u;
        kinds[c] = 2;   /* loop condition */
        params[c] |= (trips[i] & 0xFFu) << 16;
        src[e] = c;
        dst[e] = base;
        e++;
        for (uint32_t j = 1; j < ks[i]; ++j) {
            src[e] = c;
            dst[e] = base + 1u + j;
            e++;
        }
        base += ks[i] + 1u;
    }
    *m = e;
    *n_d_out = n_d;
    *pos_out = st.pos;
    return WL_OK;
}
