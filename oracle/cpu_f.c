/*
 * CPU-F: the paper's fine-grained CPU design, restated in plain C with
 * OpenMP.  Test and benchmark infrastructure only (like the oracle beside it):
 * the benchmark times it on all host cores as the multi-core CPU baseline,
 * and a CPU test checks it against the oracle.  It shares no code with the
 * CUDA library.
 *
 * Paper: M. Blanco, T. M. Low, K. Kim, "Exploration of Fine-Grained Parallelism
 * for Load Balancing Eager K-truss on GPU and CPU", HPEC 2019.
 *
 * What the paper's CPU version does (Sec. III, Sec. III-D, the fine-grained
 * kernel of Sec. III-B):
 *   - one task per stored edge (i, kappa) of the upper-triangular CSR; the task
 *     walks the part of row i after the edge and row kappa with two pointers and,
 *     for every common column, adds one to the supports of the three edges of
 *     the triangle (eager update, Sec. II-B) with atomic additions;
 *   - removed edges are dropped by moving the row's surviving entries left and
 *     ending the row with a zero (column 0 never appears in a strictly
 *     upper-triangular row, so a zero ends every walk);
 *   - rounds repeat until one removes nothing (Alg. 1), all failing edges
 *     leaving at once.
 * Tasks are spread over the threads in dynamic chunks.
 *
 * Outputs and return codes as oracle_ktruss: mask[m], support[m] in input edge
 * order, *rounds; 0 success, -1 invalid input, -2 out of memory.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

int cpuf_ktruss(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col, int32_t K,
                int32_t threads, uint8_t *mask, int32_t *support, int32_t *rounds) {
    if (n < 0 || m < 0 || !row_ptr || (m > 0 && !col) || K < 2) return -1;
    if (row_ptr[0] != 0 || row_ptr[n] != m) return -1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#endif
    size_t mm = (size_t)(m > 0 ? m : 1);
    int32_t *A = (int32_t *)malloc(mm * sizeof(int32_t));    /* live columns, 0 = end of row */
    int32_t *id = (int32_t *)malloc(mm * sizeof(int32_t));   /* input slot of each entry */
    int32_t *row = (int32_t *)malloc(mm * sizeof(int32_t));  /* row of each slot */
    int32_t *S = (int32_t *)malloc(mm * sizeof(int32_t));
    if (!A || !id || !row || !S) {
        free(A); free(id); free(row); free(S);
        return -2;
    }
    for (int32_t i = 0; i < n; ++i)
        for (int64_t p = row_ptr[i]; p < row_ptr[i + 1]; ++p) {
            if (col[p] <= i || col[p] >= n) {
                free(A); free(id); free(row); free(S);
                return -1;
            }
            A[p] = col[p];
            id[p] = (int32_t)p;
            row[p] = i;
        }
    int64_t live = m;
    int32_t r = 0;
    const int32_t thr = K - 2;
    while (live > 0) {
        ++r;
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < m; ++p) S[p] = 0;
        /* supports: one task per stored edge */
#pragma omp parallel for schedule(dynamic, 512)
        for (int64_t p = 0; p < m; ++p) {
            const int32_t kappa = A[p];
            if (kappa == 0) continue; /* past the end of its row */
            const int32_t i = row[p];
            int64_t x = p + 1, xe = row_ptr[i + 1];
            int64_t y = row_ptr[kappa], ye = row_ptr[kappa + 1];
            int32_t own = 0;
            while (x < xe && y < ye) {
                const int32_t a = A[x], b = A[y];
                if (a == 0 || b == 0) break;
                if (a == b) {
                    __atomic_fetch_add(S + x, 1, __ATOMIC_RELAXED);
                    __atomic_fetch_add(S + y, 1, __ATOMIC_RELAXED);
                    ++own;
                    ++x;
                    ++y;
                } else if (a < b) {
                    ++x;
                } else {
                    ++y;
                }
            }
            if (own) __atomic_fetch_add(S + p, own, __ATOMIC_RELAXED);
        }
        /* prune: keep entries with S >= K-2, moved left; zeros after them */
        int64_t removed = 0;
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : removed)
        for (int32_t i = 0; i < n; ++i) {
            int64_t w = row_ptr[i];
            for (int64_t p = row_ptr[i]; p < row_ptr[i + 1] && A[p] != 0; ++p) {
                if (S[p] >= thr) {
                    A[w] = A[p];
                    id[w] = id[p];
                    S[w] = S[p];
                    ++w;
                } else {
                    ++removed;
                }
            }
            for (int64_t p = w; p < row_ptr[i + 1] && A[p] != 0; ++p) A[p] = 0;
        }
        live -= removed;
        if (removed == 0) break;
    }
    memset(mask, 0, (size_t)m);
    if (support) memset(support, 0, (size_t)m * sizeof(int32_t));
    for (int64_t p = 0; p < m; ++p)
        if (A[p] != 0) {
            mask[id[p]] = 1;
            if (support) support[id[p]] = S[p];
        }
    if (rounds) *rounds = r;
    free(A); free(id); free(row); free(S);
    return 0;
}
