// Input validation of the strictly upper-triangular CSR (Sec. II-B, III-D):
// one warp per row checks its row pointer pair and every column of the row.
#include "ktruss_internal.cuh"

namespace kt {
namespace {

constexpr int32_t kErrRowPtr = 1;    // row_ptr[0] != 0, row_ptr[n] != m, or decreasing
constexpr int32_t kErrRange = 2;     // a column <= its row or >= n
constexpr int32_t kErrOrder = 4;     // columns not strictly increasing in a row
constexpr int32_t kErrBounds = 8;    // row_ptr entry outside [0, m]

__global__ void validate_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                int32_t n, int64_t m, int32_t *err) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int64_t warps = (int64_t(gridDim.x) * blockDim.x) >> 5;
    if (warp == 0 && lane == 0) {
        if (rp[0] != 0 || int64_t(rp[n]) != m) atomicOr(err, kErrRowPtr);
    }
    for (int64_t i = warp; i < n; i += warps) {
        const int32_t b = rp[i], e = rp[i + 1];
        if (b < 0 || int64_t(e) > m || b > int64_t(m) || e < 0) {
            if (lane == 0) atomicOr(err, kErrBounds);
            continue;
        }
        if (e < b) {
            if (lane == 0) atomicOr(err, kErrRowPtr);
            continue;
        }
        int32_t bad = 0;
        for (int32_t p = b + lane; p < e; p += 32) {
            const int32_t c = col[p];
            if (c <= int32_t(i) || c >= n) bad |= kErrRange;
            if (p > b && col[p - 1] >= c) bad |= kErrOrder;
        }
        bad = __reduce_or_sync(0xffffffffu, bad);
        if (bad && lane == 0) atomicOr(err, bad);
    }
}

}  // namespace

cudaError_t launch_validate(const int32_t *rp, const int32_t *col, int32_t n, int64_t m,
                            int32_t *err, cudaStream_t s) {
    const int threads = 256;
    int64_t warps_needed = n > 0 ? n : 1;
    int64_t blocks = (warps_needed * 32 + threads - 1) / threads;
    if (blocks > 152 * 32) blocks = 152 * 32;
    validate_kernel<<<int(blocks), threads, 0, s>>>(rp, col, n, m, err);
    return cudaGetLastError();
}

}  // namespace kt
