// Support step, one thread per live edge (Alg. 3's edge task exactly as the
// paper schedules it, Sec. III-C): the thread of edge (i, kappa) at slot e runs
// a two-pointer merge of row i after e with row kappa, and every common column
// credits the three edges of that triangle (eager rule, Sec. II-B).  This is
// the simple, unbalanced baseline; the balanced kernel lives in
// support_balanced.cu.  The coarse-grained kernel (Alg. 2, one thread per row)
// is here too, to measure the paper's fine/coarse comparison on this GPU.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

// Largest row index i with rp[i] <= e, i.e. the row holding slot e (e < m).
__device__ __forceinline__ int32_t row_of_slot(const int32_t *__restrict__ rp, int32_t n,
                                               int32_t e) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int32_t mid = lo + ((hi - lo + 1) >> 1);
        if (__ldg(rp + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256)
support_edge_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                    int32_t m, int32_t *__restrict__ S, unsigned long long *__restrict__ tri,
                    const int32_t *__restrict__ gid, const uint8_t *__restrict__ skip) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool live = t < m;
    const int32_t e = live ? int32_t(t) : 0;
    int32_t own = 0;
    const int32_t i = live ? row_of_slot(rp, n, e) : 0;
    if (live && !(skip && skip[gid[i]])) {
        const int32_t kappa = __ldg(col + e);
        int32_t x = e + 1;
        const int32_t xe = __ldg(rp + i + 1);
        int32_t y = __ldg(rp + kappa);
        const int32_t ye = __ldg(rp + kappa + 1);
        while (x < xe && y < ye) {
            const int32_t a = __ldg(col + x), b = __ldg(col + y);
            if (a == b) {
                atomicAdd(S + x, 1);
                atomicAdd(S + y, 1);
                ++own;
                ++x;
                ++y;
            } else if (a < b) {
                ++x;
            } else {
                ++y;
            }
        }
        if (own) atomicAdd(S + e, own);
    }
    const int32_t tot = __reduce_add_sync(0xffffffffu, own);
    if ((threadIdx.x & 31) == 0 && tot) atomicAdd(tri, (unsigned long long)tot);
}

// Coarse-grained support step (Alg. 2): one thread per row i applies both
// update rules of the row partition, i.e. for every nonzero kappa of a12 it
// intersects the rest of a12 with row kappa of A22 and credits each triangle
// to (i,kappa), (i,w) and (kappa,w).  All edge tasks of a row run one after
// another in the same thread, which is the load imbalance Sec. III-A describes.
__global__ void __launch_bounds__(256)
support_coarse_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col, int32_t n,
                      int32_t *__restrict__ S, unsigned long long *__restrict__ tri,
                      const int32_t *__restrict__ gid, const uint8_t *__restrict__ skip) {
    const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int32_t i = t < n ? int32_t(t) : 0;
    long long found = 0;
    if (t < n && !(skip && skip[gid[i]])) {
        const int32_t rb = __ldg(rp + i), re = __ldg(rp + i + 1);
        for (int32_t e = rb; e < re; ++e) {
            const int32_t kappa = __ldg(col + e);
            int32_t x = e + 1, y = __ldg(rp + kappa);
            const int32_t ye = __ldg(rp + kappa + 1);
            int32_t own = 0;
            while (x < re && y < ye) {
                const int32_t a = __ldg(col + x), b = __ldg(col + y);
                if (a == b) {
                    atomicAdd(S + x, 1);
                    atomicAdd(S + y, 1);
                    ++own;
                    ++x;
                    ++y;
                } else if (a < b) {
                    ++x;
                } else {
                    ++y;
                }
            }
            if (own) atomicAdd(S + e, own);
            found += own;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) found += __shfl_down_sync(0xffffffffu, found, d);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(tri, (unsigned long long)found);
}

}  // namespace

cudaError_t launch_support_coarse(const Live &g, int32_t *S, RoundCounters *cnt, cudaStream_t s) {
    if (g.m == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = int((int64_t(g.n) + threads - 1) / threads);
    support_coarse_kernel<<<blocks, threads, 0, s>>>(g.rp, g.col, g.n, S, &cnt->triangles, g.gid,
                                                     g.skip);
    return cudaGetLastError();
}

cudaError_t launch_support_edge(const Live &g, int32_t *S, RoundCounters *cnt, cudaStream_t s) {
    if (g.m == 0) return cudaSuccess;
    const int threads = 256;
    const int blocks = int((int64_t(g.m) + threads - 1) / threads);
    support_edge_kernel<<<blocks, threads, 0, s>>>(g.rp, g.col, g.n, g.m, S, &cnt->triangles,
                                                   g.gid, g.skip);
    return cudaGetLastError();
}

}  // namespace kt
