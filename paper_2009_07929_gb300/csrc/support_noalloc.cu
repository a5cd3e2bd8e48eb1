// ktruss_support_noalloc: the balanced support step for callers that cannot
// allocate device memory.
//
// Some callers may not call cudaMalloc (or any allocating routine) on their
// path: code that runs inside a memory pool or arena owned by someone else,
// code that must not grow the process's device footprint after start-up, and
// embedded users that budget every byte up front.  For them this entry point
// computes the support of every edge of a graph that stays in the caller's
// device memory, writing into the caller's output, and takes all of its
// working memory from one fixed-size array that lives for as long as the
// library is loaded.
//
// Scratch: g_noalloc_scratch below, kNoAllocScratchBytes (32 MiB), held by
// every GPU that loads the library until the process exits.  It serves graphs
// with at most kNoAllocMaxVertices vertices and kNoAllocMaxEdges edges.
// Every call uses the same array and leaves its contents behind; whatever must
// start at zero is cleared by the call itself.  Calls whose work overlaps on
// the GPU (two streams, two host threads) race on the array and must not be
// issued.
//
// Set-up: the first call on a device, with that device current, looks up the
// device address of the array once (cudaGetSymbolAddress); a host-side name
// of a __device__ array is not a device address.  That first call should come
// before any stream capture.
//
// Every call synchronises its stream and copies the round counters to the
// host before it returns.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "ktruss.h"
#include "ktruss_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int32_t kNoAllocMaxVertices = 1 << 19;
constexpr int64_t kNoAllocMaxEdges = int64_t(1) << 19;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::atomic<void *> g_scratch_addr[kMaxDevices];

// Device address of the scratch array on the current device (set up once per
// device).
cudaError_t scratch_address(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    void *p = g_scratch_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev].store(p, std::memory_order_release);
    }
    *out = p;
    return cudaSuccess;
}

int fail(cudaError_t e) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? KTRUSS_ENOMEM : KTRUSS_ECUDA;
}

}  // namespace

extern "C" int ktruss_support_noalloc(int32_t n, int64_t m, const int32_t *row_ptr,
                                      const int32_t *col, int32_t *support_out,
                                      int64_t *triangles_out, void *cuda_stream) {
    if (n < 0 || m < 0 || !row_ptr || (m > 0 && (!col || !support_out))) return KTRUSS_EINVAL;
    if (n > kNoAllocMaxVertices || m > kNoAllocMaxEdges) return KTRUSS_EINVAL;
    // the round counters sit in the first 256 bytes, the balanced step's
    // scratch after them
    static_assert(sizeof(kt::RoundCounters) <= 256, "round counters exceed their header");
    const size_t need = 256 + kt::balanced_scratch_bytes(n, m);
    if (need > kNoAllocScratchBytes) return KTRUSS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    void *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return fail(e);
    kt::RoundCounters *cnt = static_cast<kt::RoundCounters *>(base);
    kt::BalancedScratch bs;
    bs.base = static_cast<unsigned char *>(base) + 256;
    bs.cap_m = m;
    bs.cap_n = n;
    kt::RoundCounters host{};
    // validate the input before any kernel walks it
    e = cudaMemsetAsync(cnt, 0, sizeof(kt::RoundCounters), s);
    if (e == cudaSuccess) e = kt::launch_validate(row_ptr, col, n, m, &cnt->error, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&host, cnt, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(e);
    if (host.error != 0) return KTRUSS_EINVAL;
    if (m > 0) {
        int launches = 0;
        const kt::Live g{row_ptr, col, nullptr, n, int32_t(m)};
        e = cudaMemsetAsync(support_out, 0, size_t(m) * sizeof(int32_t), s);
        if (e == cudaSuccess) e = kt::launch_support_balanced(g, support_out, cnt, &bs, s, &launches,
                                                              nullptr);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&host, cnt, sizeof(host), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return fail(e);
        // a device-side check of the support kernel gave up (see its give-up
        // words): the supports are incomplete
        if (host.error) return (host.error & kt::kDevErrTimeout) ? KTRUSS_ETIMEOUT : KTRUSS_ECUDA;
    }
    if (triangles_out) *triangles_out = int64_t(host.triangles);
    return KTRUSS_OK;
}
