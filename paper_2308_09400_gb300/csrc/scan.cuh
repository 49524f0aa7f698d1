// Device-wide exclusive prefix sum (internal).
//
// exclusive_scan(in, out, n): out[i] = sum_{j<i} in[j] for i <= n (out has n+1
// entries, out[n] is the total).  Three launches per level: tile scan (4096
// items per 1024-thread block), recursive scan of the tile totals, and an add
// of the scanned totals.  Deterministic (integer arithmetic).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace gipc {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

// Scratch (in int64 words) needed by exclusive_scan for n items.
inline int64_t scan_scratch_words(int64_t n) {
    int64_t words = 0;
    while (n > kScanTile) {
        n = (n + kScanTile - 1) / kScanTile;
        words += n + 1;
    }
    return words + 1;
}

template <typename TIn>
cudaError_t exclusive_scan(const TIn* in, int64_t* out, int64_t n, int64_t* scratch, cudaStream_t s);

}  // namespace gipc
