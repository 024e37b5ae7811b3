/*
 * oracle.c -- plain single-threaded CPU oracle for the 3-way joins.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file; it shares no code, header, hash function or table with
 * the CUDA library.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it.
 *
 * What it computes (bag semantics: a tuple that occurs m times counts m
 * times, Section 1, Example 1's footnote on duplicates):
 *
 *   linear  (Section 3, Algorithm 1's result):
 *       Out = { (a,b,c,d) : (a,b) in R, (b,c) in S, (c,d) in T }
 *   cyclic  (Section 3 and Section 5):
 *       Out = { (a,b,c)   : (a,b) in R, (b,c) in S, (c,a) in T }
 *
 * in three output modes: COUNT(*) of Out, COUNT(*) GROUP BY A as a dense
 * array over [0, a_domain), and the rows of Out sorted lexicographically.
 *
 * The evaluation is an ordinary hash join written out: group R by B into
 * lists of A; group T by C (linear: lists of D) or count the (C,A) pairs of
 * T (cyclic); then walk S once and combine.  For COUNT and GROUP BY the
 * innermost enumeration over T's matching tuples is replaced by the number
 * of those tuples, which is the same sum.  Counts accumulate modulo 2^64
 * (unsigned wraparound); the paper fixes no width.
 *
 * Return codes: 0 ok, 1 bad argument, 2 an A value outside [0, a_domain),
 * 3 more rows than the capacity (n_rows still holds the exact count),
 * 4 out of host memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { O_COUNT = 0, O_GROUP_BY_A = 1, O_MATERIALIZE = 2 };

/* ---------- a small open-addressing map: 64-bit key -> dense index ------- */

typedef struct {
    uint64_t *key;
    int64_t *idx;    /* -1 = empty */
    uint64_t mask;
    int64_t n;       /* number of distinct keys inserted */
} omap;

static uint64_t omix(uint64_t z) {            /* SplitMix64 finaliser */
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int omap_init(omap *m, int64_t expected) {
    uint64_t cap = 16;
    while (cap < (uint64_t)expected * 2 + 16) cap <<= 1;
    m->key = (uint64_t *)malloc(cap * sizeof(uint64_t));
    m->idx = (int64_t *)malloc(cap * sizeof(int64_t));
    if (!m->key || !m->idx) { free(m->key); free(m->idx); return 4; }
    for (uint64_t i = 0; i < cap; ++i) m->idx[i] = -1;
    m->mask = cap - 1;
    m->n = 0;
    return 0;
}

static void omap_free(omap *m) { free(m->key); free(m->idx); }

/* index of key, inserting it with the next dense index if absent */
static int64_t omap_get_or_add(omap *m, uint64_t k) {
    uint64_t s = omix(k) & m->mask;
    for (;;) {
        if (m->idx[s] < 0) { m->key[s] = k; m->idx[s] = m->n++; return m->idx[s]; }
        if (m->key[s] == k) return m->idx[s];
        s = (s + 1) & m->mask;
    }
}

static int64_t omap_find(const omap *m, uint64_t k) {
    uint64_t s = omix(k) & m->mask;
    for (;;) {
        if (m->idx[s] < 0) return -1;
        if (m->key[s] == k) return m->idx[s];
        s = (s + 1) & m->mask;
    }
}

static uint64_t key32(int32_t v) { return (uint64_t)(uint32_t)v; }
static uint64_t key64(int32_t hi, int32_t lo) {
    return ((uint64_t)(uint32_t)hi << 32) | (uint64_t)(uint32_t)lo;
}

/* ---------- grouping: key column -> CSR lists of the payload column ------ */

typedef struct {
    omap map;
    int64_t *start;   /* per distinct key, offset into vals; size ndistinct+1 */
    int32_t *vals;    /* payloads grouped by key */
} ogroup;

static int ogroup_build(ogroup *g, const int32_t *key, const int32_t *val, int64_t n) {
    int rc = omap_init(&g->map, n);
    if (rc) return rc;
    int64_t *id = (int64_t *)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
    if (!id) { omap_free(&g->map); return 4; }
    for (int64_t i = 0; i < n; ++i) id[i] = omap_get_or_add(&g->map, key32(key[i]));
    int64_t d = g->map.n;
    g->start = (int64_t *)calloc((size_t)d + 1, sizeof(int64_t));
    g->vals = (int32_t *)malloc((size_t)(n ? n : 1) * sizeof(int32_t));
    if (!g->start || !g->vals) { free(id); free(g->start); free(g->vals); omap_free(&g->map); return 4; }
    for (int64_t i = 0; i < n; ++i) g->start[id[i] + 1]++;
    for (int64_t k = 0; k < d; ++k) g->start[k + 1] += g->start[k];
    int64_t *fill = (int64_t *)malloc((size_t)(d ? d : 1) * sizeof(int64_t));
    if (!fill) { free(id); free(g->start); free(g->vals); omap_free(&g->map); return 4; }
    memcpy(fill, g->start, (size_t)d * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->vals[fill[id[i]]++] = val[i];
    free(fill);
    free(id);
    return 0;
}

static void ogroup_free(ogroup *g) { omap_free(&g->map); free(g->start); free(g->vals); }

/* ---------- row output ---------------------------------------------------- */

static int g_arity;
static int row_cmp(const void *x, const void *y) {
    const int32_t *p = (const int32_t *)x, *q = (const int32_t *)y;
    for (int k = 0; k < g_arity; ++k) {
        if (p[k] < q[k]) return -1;
        if (p[k] > q[k]) return 1;
    }
    return 0;
}

static void sort_rows(int32_t *rows, int64_t n, int arity) {
    g_arity = arity;
    qsort(rows, (size_t)n, sizeof(int32_t) * (size_t)arity, row_cmp);
}

static int check_domain(const int32_t *a, int64_t n, int32_t a_domain) {
    for (int64_t i = 0; i < n; ++i)
        if (a[i] < 0 || a[i] >= a_domain) return 2;
    return 0;
}

/* ---------- linear: R(A,B) S(B,C) T(C,D) --------------------------------- */

int oracle_linear(const int32_t *Ra, const int32_t *Rb, int64_t nR,
                  const int32_t *Sb, const int32_t *Sc, int64_t nS,
                  const int32_t *Tc, const int32_t *Td, int64_t nT,
                  int mode, int32_t a_domain,
                  uint64_t *total, uint64_t *cnt,
                  int32_t *rows, int64_t capacity, int64_t *n_rows) {
    if (nR < 0 || nS < 0 || nT < 0 || !total) return 1;
    if (mode == O_GROUP_BY_A) {
        if (a_domain <= 0 || !cnt) return 1;
        int rc = check_domain(Ra, nR, a_domain);
        if (rc) return rc;
        memset(cnt, 0, (size_t)a_domain * sizeof(uint64_t));
    }
    if (mode == O_MATERIALIZE && (!n_rows || capacity < 0)) return 1;

    ogroup RB, TC;                     /* b -> [a],  c -> [d] */
    int rc = ogroup_build(&RB, Rb, Ra, nR);
    if (rc) return rc;
    rc = ogroup_build(&TC, Tc, Td, nT);
    if (rc) { ogroup_free(&RB); return rc; }

    uint64_t tot = 0;
    int64_t nr = 0;
    for (int64_t s = 0; s < nS; ++s) {
        int64_t i = omap_find(&RB.map, key32(Sb[s]));
        if (i < 0) continue;
        int64_t j = omap_find(&TC.map, key32(Sc[s]));
        if (j < 0) continue;
        uint64_t degR = (uint64_t)(RB.start[i + 1] - RB.start[i]);
        uint64_t degT = (uint64_t)(TC.start[j + 1] - TC.start[j]);
        tot += degR * degT;
        if (mode == O_GROUP_BY_A) {
            for (int64_t p = RB.start[i]; p < RB.start[i + 1]; ++p)
                cnt[RB.vals[p]] += degT;
        } else if (mode == O_MATERIALIZE) {
            for (int64_t p = RB.start[i]; p < RB.start[i + 1]; ++p)
                for (int64_t q = TC.start[j]; q < TC.start[j + 1]; ++q) {
                    if (nr < capacity) {
                        int32_t *r = rows + 4 * nr;
                        r[0] = RB.vals[p]; r[1] = Sb[s]; r[2] = Sc[s]; r[3] = TC.vals[q];
                    }
                    ++nr;
                }
        }
    }
    *total = tot;
    ogroup_free(&RB);
    ogroup_free(&TC);
    if (mode == O_MATERIALIZE) {
        *n_rows = nr;
        if (nr > capacity) return 3;
        sort_rows(rows, nr, 4);
    }
    return 0;
}

/* ---------- linear 4-way: R(A,B) S(B,C) T(C,D) U(D,E) -------------------- */
/*
 * The chain one relation longer (Section 7's "additional levels of
 * hashing"):  Out4 = { (a,b,c,d,e) : (a,b) in R, (b,c) in S, (c,d) in T,
 * (d,e) in U }.  COUNT(*) and COUNT(*) GROUP BY A; for every S tuple (b,c)
 * the matching T tuples (c,d) are walked and each contributes deg_U(d), the
 * number of its U tuples.
 */
int oracle_linear4(const int32_t *Ra, const int32_t *Rb, int64_t nR,
                   const int32_t *Sb, const int32_t *Sc, int64_t nS,
                   const int32_t *Tc, const int32_t *Td, int64_t nT,
                   const int32_t *Ud, const int32_t *Ue, int64_t nU,
                   int mode, int32_t a_domain, uint64_t *total, uint64_t *cnt) {
    if (nR < 0 || nS < 0 || nT < 0 || nU < 0 || !total) return 1;
    if (mode != O_COUNT && mode != O_GROUP_BY_A) return 1;
    if (mode == O_GROUP_BY_A) {
        if (a_domain <= 0 || !cnt) return 1;
        int rc = check_domain(Ra, nR, a_domain);
        if (rc) return rc;
        memset(cnt, 0, (size_t)a_domain * sizeof(uint64_t));
    }
    ogroup RB, TC, UD;                 /* b -> [a],  c -> [d],  d -> [e] */
    int rc = ogroup_build(&RB, Rb, Ra, nR);
    if (rc) return rc;
    rc = ogroup_build(&TC, Tc, Td, nT);
    if (rc) { ogroup_free(&RB); return rc; }
    rc = ogroup_build(&UD, Ud, Ue, nU);
    if (rc) { ogroup_free(&RB); ogroup_free(&TC); return rc; }

    uint64_t tot = 0;
    for (int64_t s = 0; s < nS; ++s) {
        int64_t i = omap_find(&RB.map, key32(Sb[s]));
        if (i < 0) continue;
        int64_t j = omap_find(&TC.map, key32(Sc[s]));
        if (j < 0) continue;
        uint64_t tail = 0;             /* (c,d,e) continuations of this (b,c) */
        for (int64_t q = TC.start[j]; q < TC.start[j + 1]; ++q) {
            int64_t u = omap_find(&UD.map, key32(TC.vals[q]));
            if (u >= 0) tail += (uint64_t)(UD.start[u + 1] - UD.start[u]);
        }
        uint64_t degR = (uint64_t)(RB.start[i + 1] - RB.start[i]);
        tot += degR * tail;
        if (mode == O_GROUP_BY_A)
            for (int64_t p = RB.start[i]; p < RB.start[i + 1]; ++p) cnt[RB.vals[p]] += tail;
    }
    *total = tot;
    ogroup_free(&RB);
    ogroup_free(&TC);
    ogroup_free(&UD);
    return 0;
}

/* ---------- cyclic: R(A,B) S(B,C) T(C,A) --------------------------------- */

int oracle_cyclic(const int32_t *Ra, const int32_t *Rb, int64_t nR,
                  const int32_t *Sb, const int32_t *Sc, int64_t nS,
                  const int32_t *Tc, const int32_t *Ta, int64_t nT,
                  int mode, int32_t a_domain,
                  uint64_t *total, uint64_t *cnt,
                  int32_t *rows, int64_t capacity, int64_t *n_rows) {
    if (nR < 0 || nS < 0 || nT < 0 || !total) return 1;
    if (mode == O_GROUP_BY_A) {
        if (a_domain <= 0 || !cnt) return 1;
        int rc = check_domain(Ra, nR, a_domain);
        if (rc) return rc;
        memset(cnt, 0, (size_t)a_domain * sizeof(uint64_t));
    }
    if (mode == O_MATERIALIZE && (!n_rows || capacity < 0)) return 1;

    ogroup RB;                         /* b -> [a] */
    int rc = ogroup_build(&RB, Rb, Ra, nR);
    if (rc) return rc;
    omap TP;                           /* (c,a) -> dense id, with multiplicity */
    rc = omap_init(&TP, nT);
    if (rc) { ogroup_free(&RB); return rc; }
    uint64_t *mult = (uint64_t *)calloc((size_t)(nT ? nT : 1), sizeof(uint64_t));
    if (!mult) { ogroup_free(&RB); omap_free(&TP); return 4; }
    for (int64_t t = 0; t < nT; ++t) mult[omap_get_or_add(&TP, key64(Tc[t], Ta[t]))]++;

    uint64_t tot = 0;
    int64_t nr = 0;
    for (int64_t s = 0; s < nS; ++s) {
        int64_t i = omap_find(&RB.map, key32(Sb[s]));
        if (i < 0) continue;
        for (int64_t p = RB.start[i]; p < RB.start[i + 1]; ++p) {
            int32_t a = RB.vals[p];
            int64_t k = omap_find(&TP, key64(Sc[s], a));
            if (k < 0) continue;
            uint64_t m = mult[k];
            tot += m;
            if (mode == O_GROUP_BY_A) cnt[a] += m;
            else if (mode == O_MATERIALIZE) {
                for (uint64_t e = 0; e < m; ++e) {
                    if (nr < capacity) {
                        int32_t *r = rows + 3 * nr;
                        r[0] = a; r[1] = Sb[s]; r[2] = Sc[s];
                    }
                    ++nr;
                }
            }
        }
    }
    *total = tot;
    free(mult);
    omap_free(&TP);
    ogroup_free(&RB);
    if (mode == O_MATERIALIZE) {
        *n_rows = nr;
        if (nr > capacity) return 3;
        sort_rows(rows, nr, 3);
    }
    return 0;
}

/* ---------- binary join R(A,B) S(B,C) -> count of I(A,B,C) ---------------
 * |R join S| = sum over b of deg_R(b) * deg_S(b); the cascade's intermediate
 * size (Section 6.3), used to size it and to pin the cascade's first join. */
int oracle_binary_count(const int32_t *Rb, int64_t nR, const int32_t *Sb, int64_t nS,
                        uint64_t *count) {
    if (nR < 0 || nS < 0 || !count) return 1;
    omap m;
    int rc = omap_init(&m, nR);
    if (rc) return rc;
    uint64_t *deg = (uint64_t *)calloc((size_t)(nR ? nR : 1), sizeof(uint64_t));
    if (!deg) { omap_free(&m); return 4; }
    for (int64_t i = 0; i < nR; ++i) deg[omap_get_or_add(&m, key32(Rb[i]))]++;
    uint64_t c = 0;
    for (int64_t s = 0; s < nS; ++s) {
        int64_t k = omap_find(&m, key32(Sb[s]));
        if (k >= 0) c += deg[k];
    }
    *count = c;
    free(deg);
    omap_free(&m);
    return 0;
}
