/*
 * K-truss ORACLE: plain, slow, single-threaded CPU reference used only by the
 * tests, by the package's smoke check and by the benchmark's CPU-baseline leg.
 * It is test infrastructure, not part of the product path, and shares no code
 * with the CUDA library.
 *
 * Paper: M. Blanco, T. M. Low, K. Kim, "Exploration of Fine-Grained Parallelism
 * for Load Balancing Eager K-truss on GPU and CPU", HPEC 2019.
 *
 * Input everywhere: an undirected simple graph as a strictly upper-triangular
 * CSR (row_ptr int32[n+1], col int32[m], columns strictly increasing within a
 * row, col > row), Sec. II-B and Sec. III-D.  Edge e is CSR slot e.
 *
 * Functions
 *   oracle_ktruss              Alg. 1 (bulk peeling) with the eager credit rule
 *                              of Sec. II-B, support counted per edge task as in
 *                              Alg. 3.
 *   oracle_truss_decomposition A second, independent algorithm: sequential
 *                              edge peeling in increasing support order, giving
 *                              every edge's trussness (the largest K whose
 *                              K-truss holds it; definition in Sec. I).
 *   oracle_edge_support        Support of selected edges inside the subgraph a
 *                              mask selects: |N(u) ∩ N(v)| restricted to kept
 *                              edges (the quantity Alg. 1's S[i,j] denotes,
 *                              Sec. II-A), used to check sampled outputs of
 *                              large runs one edge at a time.
 *   oracle_triangles           Triangle count of the subgraph a mask selects,
 *                              by a node iterator with a marker array (used for
 *                              the invariant sum(support) = 3 x triangles).
 *
 * Return codes: 0 success, -1 invalid input, -2 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

/* Checks the input contract of every entry point. */
int oracle_check_csr(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col) {
    if (n < 0 || m < 0 || !row_ptr || (m > 0 && !col)) return OR_EINVAL;
    if (row_ptr[0] != 0 || row_ptr[n] != m) return OR_EINVAL;
    for (int32_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] < row_ptr[i]) return OR_EINVAL;
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if (col[p] <= i || col[p] >= n) return OR_EINVAL;
            if (p > row_ptr[i] && col[p] <= col[p - 1]) return OR_EINVAL;
        }
    }
    return OR_OK;
}

/*
 * Alg. 1 of the paper, computed per edge task (Alg. 3):
 *   repeat:  S <- support of every live edge          (Step 1, computeSupports)
 *            remove every live edge with S < K - 2    (Step 2, pruneEdges)
 *   until a round removes nothing.
 * Step 1 follows the eager update rule of Sec. II-B: the triangle i < kappa < w
 * is found once, by the task of edge (i, kappa), which walks the live part of
 * row i after kappa and the live row kappa together (the two sorted lists of
 * Alg. 3's three update lines); each common column w adds one to S of (i,kappa),
 * (i,w) and (kappa,w).
 *
 * Readings where the paper is silent: the threshold keeps S >= K-2 (Sec. I);
 * all failing edges leave at once (bulk); `rounds` counts executions of Step 1,
 * the loop stopping before Step 1 when no live edge is left and after Step 2
 * when nothing was removed; removed edges report support 0; K < 2 is invalid.
 *
 * Outputs: mask[m] (1 = edge in the K-truss), support[m] (its support inside
 * the K-truss, 0 for removed edges), *rounds, removed_per_round[0..cap) (edges
 * removed by each round, truncated at cap), *triangles (of the final truss),
 * triangles_per_round[0..cap) (triangles of the live graph Step 1 of each
 * round counted; may be NULL).
 */
int oracle_ktruss(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col, int32_t K,
                  uint8_t *mask, int32_t *support, int32_t *rounds, int64_t *removed_per_round,
                  int32_t cap, int64_t *triangles, int64_t *triangles_per_round) {
    int rc = oracle_check_csr(n, m, row_ptr, col);
    if (rc != OR_OK) return rc;
    if (K < 2) return OR_EINVAL;
    uint8_t *live = (uint8_t *)malloc((size_t)(m > 0 ? m : 1));
    int64_t *S = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    int64_t *lstart = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    int64_t *lslot = (int64_t *)malloc((size_t)(m > 0 ? m : 1) * sizeof(int64_t));
    if (!live || !S || !lstart || !lslot) {
        free(live); free(S); free(lstart); free(lslot);
        return OR_ENOMEM;
    }
    memset(live, 1, (size_t)m);
    int64_t m_live = m;
    int32_t r = 0;
    int64_t tri = 0;
    for (;;) {
        if (m_live == 0) break;
        ++r;
        /* live slots of every row, in column order */
        int64_t c = 0;
        for (int32_t i = 0; i < n; ++i) {
            lstart[i] = c;
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p)
                if (live[p]) lslot[c++] = p;
        }
        lstart[n] = c;
        /* Step 1: supports from scratch */
        memset(S, 0, (size_t)m * sizeof(int64_t));
        tri = 0;
        for (int32_t i = 0; i < n; ++i) {
            for (int64_t a = lstart[i]; a < lstart[i + 1]; ++a) {
                int64_t p = lslot[a];
                int32_t kappa = col[p];
                int64_t x = a + 1, xe = lstart[i + 1]; /* live tail of row i */
                int64_t y = lstart[kappa], ye = lstart[kappa + 1]; /* live row kappa */
                while (x < xe && y < ye) {
                    int32_t cx = col[lslot[x]], cy = col[lslot[y]];
                    if (cx == cy) {
                        S[p] += 1;
                        S[lslot[x]] += 1;
                        S[lslot[y]] += 1;
                        ++tri;
                        ++x;
                        ++y;
                    } else if (cx < cy) {
                        ++x;
                    } else {
                        ++y;
                    }
                }
            }
        }
        if (triangles_per_round && r - 1 < cap) triangles_per_round[r - 1] = tri;
        /* Step 2: remove all failing edges at once */
        int64_t removed = 0;
        for (int64_t e = 0; e < m; ++e)
            if (live[e] && S[e] < (int64_t)K - 2) {
                live[e] = 0;
                ++removed;
            }
        if (removed_per_round && r - 1 < cap) removed_per_round[r - 1] = removed;
        m_live -= removed;
        if (removed == 0) break;
        if (m_live == 0) tri = 0;
    }
    for (int64_t e = 0; e < m; ++e) {
        mask[e] = live[e];
        if (support) support[e] = live[e] ? (int32_t)S[e] : 0;
    }
    if (rounds) *rounds = r;
    if (triangles) *triangles = tri;
    free(live); free(S); free(lstart); free(lslot);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Undirected adjacency with edge ids, shared by the two checkers below.     */

typedef struct {
    int32_t n;
    int64_t *off;  /* n+1 */
    int32_t *nbr;  /* 2m, sorted within each vertex */
    int64_t *eid;  /* 2m, CSR slot of the undirected edge */
} sym_adj;

static void sym_free(sym_adj *a) {
    free(a->off); free(a->nbr); free(a->eid);
}

static int sym_build(sym_adj *a, int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col) {
    a->n = n;
    a->off = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    a->nbr = (int32_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int32_t));
    a->eid = (int64_t *)malloc((size_t)(2 * m > 0 ? 2 * m : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
    if (!a->off || !a->nbr || !a->eid || !fill) { sym_free(a); free(fill); return OR_ENOMEM; }
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            a->off[i + 1]++;
            a->off[col[p] + 1]++;
        }
    for (int32_t i = 0; i < n; ++i) a->off[i + 1] += a->off[i];
    memcpy(fill, a->off, ((size_t)n + 1) * sizeof(int64_t));
    /* lower neighbours first (rows j < i, visited in increasing j), then the
     * upper row itself: both in increasing order, so every list is sorted */
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            int32_t j = col[p];
            a->nbr[fill[j]] = i;
            a->eid[fill[j]++] = p;
        }
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            a->nbr[fill[i]] = col[p];
            a->eid[fill[i]++] = p;
        }
    free(fill);
    return OR_OK;
}

/*
 * For each queried edge slot q[k], writes into out[k] the number of vertices w
 * with both (u,w) and (v,w) kept, where (u,v) is edge q[k] and "kept" means
 * keep[slot] != 0 (keep == NULL keeps every edge).  Two sorted neighbour lists
 * are merged, skipping removed edges.
 */
int oracle_edge_support(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                        const uint8_t *keep, int64_t nq, const int64_t *q, int64_t *out) {
    int rc = oracle_check_csr(n, m, row_ptr, col);
    if (rc != OR_OK) return rc;
    sym_adj a;
    if (sym_build(&a, n, m, row_ptr, col) != OR_OK) return OR_ENOMEM;
    /* row of each slot, by binary search on row_ptr */
    for (int64_t k = 0; k < nq; ++k) {
        int64_t e = q[k];
        if (e < 0 || e >= m) { sym_free(&a); return OR_EINVAL; }
        int32_t lo = 0, hi = n - 1;
        while (lo < hi) {
            int32_t mid = lo + (hi - lo + 1) / 2;
            if (row_ptr[mid] <= e) lo = mid; else hi = mid - 1;
        }
        int32_t u = lo, v = col[e];
        int64_t x = a.off[u], xe = a.off[u + 1], y = a.off[v], ye = a.off[v + 1], cnt = 0;
        while (x < xe && y < ye) {
            if (keep && !keep[a.eid[x]]) { ++x; continue; }
            if (keep && !keep[a.eid[y]]) { ++y; continue; }
            if (a.nbr[x] == a.nbr[y]) { ++cnt; ++x; ++y; }
            else if (a.nbr[x] < a.nbr[y]) ++x;
            else ++y;
        }
        out[k] = cnt;
    }
    sym_free(&a);
    return OR_OK;
}

/*
 * Triangles of the subgraph of kept edges (keep == NULL: all edges), by a node
 * iterator: for each vertex u, mark its kept neighbours; for each kept edge
 * (u,v) with u < v and each kept neighbour w > v of v, count w if marked.
 */
int oracle_triangles(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                     const uint8_t *keep, int64_t *triangles) {
    int rc = oracle_check_csr(n, m, row_ptr, col);
    if (rc != OR_OK) return rc;
    sym_adj a;
    if (sym_build(&a, n, m, row_ptr, col) != OR_OK) return OR_ENOMEM;
    uint8_t *mark = (uint8_t *)calloc((size_t)n + 1, 1);
    if (!mark) { sym_free(&a); return OR_ENOMEM; }
    int64_t t = 0;
    for (int32_t u = 0; u < n; ++u) {
        for (int64_t x = a.off[u]; x < a.off[u + 1]; ++x)
            if (!keep || keep[a.eid[x]]) mark[a.nbr[x]] = 1;
        for (int64_t x = a.off[u]; x < a.off[u + 1]; ++x) {
            int32_t v = a.nbr[x];
            if (v <= u || (keep && !keep[a.eid[x]])) continue;
            for (int64_t y = a.off[v]; y < a.off[v + 1]; ++y) {
                int32_t w = a.nbr[y];
                if (w > v && (!keep || keep[a.eid[y]]) && mark[w]) ++t;
            }
        }
        for (int64_t x = a.off[u]; x < a.off[u + 1]; ++x) mark[a.nbr[x]] = 0;
    }
    *triangles = t;
    free(mark);
    sym_free(&a);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Truss decomposition: a second, independent K-truss algorithm.             */

/* position of w in the sorted list nbr[lo, hi), or -1 */
static int64_t find_sorted(const int32_t *nbr, int64_t lo, int64_t hi, int32_t w) {
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (nbr[mid] < w) lo = mid + 1; else hi = mid;
    }
    return (lo < end && nbr[lo] == w) ? lo : -1;
}

/*
 * trussness[e] = the largest K such that edge e belongs to the K-truss (2 for
 * an edge in no triangle).  Sequential peeling in increasing support order,
 * with the edges kept sorted by current support in bins (the bin-sort edge
 * peeling of Wang and Cheng, "Truss decomposition in massive networks",
 * PVLDB 2012):
 *   every edge starts with its triangle count;
 *   take the remaining edge e of least current support s, set k = max(k, s+2),
 *   give e trussness k and delete it;
 *   for every remaining triangle (e, e1, e2) on e, lower the support of e1 and
 *   of e2 by one, except that a support already at or below s stays (such an
 *   edge gets trussness k anyway, as k never decreases);
 * until no edge remains.  The K-truss is then {e : trussness[e] >= K}.
 * The triangles on e = (u, v) are the common neighbours of u and v: the
 * neighbour list of the endpoint with fewer neighbours is walked and each
 * neighbour is looked up in the other list by binary search.
 */
int oracle_truss_decomposition(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                               int32_t *trussness) {
    int rc = oracle_check_csr(n, m, row_ptr, col);
    if (rc != OR_OK) return rc;
    sym_adj a;
    if (sym_build(&a, n, m, row_ptr, col) != OR_OK) return OR_ENOMEM;
    size_t mm = (size_t)(m > 0 ? m : 1);
    int64_t *sup = (int64_t *)calloc(mm, sizeof(int64_t));
    uint8_t *gone = (uint8_t *)calloc(mm, 1);
    int32_t *eu = (int32_t *)malloc(mm * sizeof(int32_t));
    int64_t *order = (int64_t *)malloc(mm * sizeof(int64_t)); /* edges by support */
    int64_t *pos = (int64_t *)malloc(mm * sizeof(int64_t));   /* order[pos[e]] == e */
    int64_t *bin = NULL;
    if (!sup || !gone || !eu || !order || !pos) goto nomem;
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) eu[p] = i;
    /* initial supports: common neighbours by binary search in the longer list */
    int64_t smax = 0;
    for (int64_t e = 0; e < m; ++e) {
        int32_t u = eu[e], v = col[e];
        int32_t s = (a.off[u + 1] - a.off[u] <= a.off[v + 1] - a.off[v]) ? u : v;
        int32_t l = (s == u) ? v : u;
        for (int64_t x = a.off[s]; x < a.off[s + 1]; ++x)
            if (find_sorted(a.nbr, a.off[l], a.off[l + 1], a.nbr[x]) >= 0) sup[e]++;
        if (sup[e] > smax) smax = sup[e];
    }
    /* counting sort of the edges by support; bin[d] = first position of
     * support d among the edges not yet taken */
    bin = (int64_t *)calloc((size_t)smax + 2, sizeof(int64_t));
    if (!bin) goto nomem;
    for (int64_t e = 0; e < m; ++e) bin[sup[e] + 1]++;
    for (int64_t d = 0; d <= smax; ++d) bin[d + 1] += bin[d];
    for (int64_t e = 0; e < m; ++e) {
        pos[e] = bin[sup[e]]++;
        order[pos[e]] = e;
    }
    for (int64_t d = smax; d > 0; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    int64_t k = 2;
    for (int64_t i = 0; i < m; ++i) {
        int64_t e = order[i];
        int64_t s = sup[e];
        if (s + 2 > k) k = s + 2;
        trussness[e] = (int32_t)k;
        gone[e] = 1;
        int32_t u = eu[e], v = col[e];
        int32_t w0 = (a.off[u + 1] - a.off[u] <= a.off[v + 1] - a.off[v]) ? u : v;
        int32_t w1 = (w0 == u) ? v : u;
        for (int64_t x = a.off[w0]; x < a.off[w0 + 1]; ++x) {
            if (gone[a.eid[x]]) continue;
            int64_t y = find_sorted(a.nbr, a.off[w1], a.off[w1 + 1], a.nbr[x]);
            if (y < 0 || gone[a.eid[y]]) continue;
            int64_t f2[2] = {a.eid[x], a.eid[y]};
            for (int t = 0; t < 2; ++t) {
                int64_t f = f2[t], d = sup[f];
                if (d <= s) continue;
                /* move f to the front of bin d, then shrink bin d past it */
                int64_t pf = pos[f], pg = bin[d], g = order[pg];
                order[pf] = g; pos[g] = pf;
                order[pg] = f; pos[f] = pg;
                bin[d]++;
                sup[f] = d - 1;
            }
        }
    }
    free(sup); free(gone); free(eu); free(order); free(pos); free(bin);
    sym_free(&a);
    return OR_OK;
nomem:
    free(sup); free(gone); free(eu); free(order); free(pos); free(bin);
    sym_free(&a);
    return OR_ENOMEM;
}
