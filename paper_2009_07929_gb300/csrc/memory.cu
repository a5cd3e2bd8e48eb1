// Device memory cache of libktruss (see cache_get in ktruss_internal.cuh).
#include <mutex>
#include <unordered_map>
#include <vector>

#include "ktruss_internal.cuh"

namespace kt {
namespace {

// Device blocks returned by freed graph handles and finished server requests,
// kept per device (at most kCacheBytes in total) and handed to later requests
// for between half and all of a block, so that a load-run-free cycle or a
// request's life does not pay cudaMalloc and cudaFree each time.  A cudaMalloc
// that fails empties the cache and retries once.  The cache remembers the true
// size of every block it hands out, so that a reused block that is larger
// than its request is counted at its own size when it comes back.
class BlockCache {
  public:
    static constexpr size_t kCacheBytes = size_t(16) << 30;
    cudaError_t get(size_t bytes, void **p) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        {
            std::lock_guard<std::mutex> lock(mu_);
            size_t best = blocks_.size();
            for (size_t i = 0; i < blocks_.size(); ++i) {
                const Block &b = blocks_[i];
                if (b.dev == dev && b.bytes >= bytes && b.bytes / 2 <= bytes &&
                    (best == blocks_.size() || b.bytes < blocks_[best].bytes))
                    best = i;
            }
            if (best < blocks_.size()) {
                *p = blocks_[best].p;
                held_ -= blocks_[best].bytes;
                out_[*p] = blocks_[best].bytes;
                blocks_.erase(blocks_.begin() + long(best));
                return cudaSuccess;
            }
        }
        e = cudaMalloc(p, bytes);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            trim();
            e = cudaMalloc(p, bytes);
        }
        if (e == cudaSuccess) {
            std::lock_guard<std::mutex> lock(mu_);
            out_[*p] = bytes;
        }
        return e;
    }
    // bytes: the size that was asked of get (the block's own size is used
    // when the cache handed the block out)
    void put(void *p, size_t bytes) {
        int dev = 0;
        if (cudaGetDevice(&dev) == cudaSuccess) {
            std::lock_guard<std::mutex> lock(mu_);
            auto it = out_.find(p);
            if (it != out_.end()) {
                bytes = it->second;
                out_.erase(it);
            }
            if (held_ + bytes <= kCacheBytes) {
                blocks_.push_back(Block{dev, bytes, p});
                held_ += bytes;
                return;
            }
        }
        cudaFree(p);
    }
    void trim() {
        std::vector<Block> out;
        {
            std::lock_guard<std::mutex> lock(mu_);
            out.swap(blocks_);
            held_ = 0;
        }
        for (const Block &b : out) cudaFree(b.p);
    }

  private:
    struct Block {
        int dev;
        size_t bytes;
        void *p;
    };
    std::mutex mu_;
    std::vector<Block> blocks_;
    std::unordered_map<void *, size_t> out_;  // blocks handed out: their true size
    size_t held_ = 0;
};

BlockCache &block_cache() {
    static BlockCache *cache = new BlockCache();  // lives as long as the process
    return *cache;
}

}  // namespace

cudaError_t cache_get(size_t bytes, void **p) { return block_cache().get(bytes, p); }
void cache_put(void *p, size_t bytes) { block_cache().put(p, bytes); }
void cache_trim() { block_cache().trim(); }

}  // namespace kt
