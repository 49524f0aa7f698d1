// Context: the device it is bound to and the scratch buffers it owns (internal).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include "common.cuh"

// A growable device buffer owned by a context.
struct gipc_scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
    // Ensure at least `want` bytes; reallocates (contents lost) when growing.
    gipc_status reserve(size_t want) {
        if (want <= bytes) return GIPC_OK;
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
        size_t sz = want + want / 4 + 256;
        if (cudaMalloc(&ptr, sz) != cudaSuccess) {
            cudaGetLastError();
            return gipc::fail(GIPC_ERR_OOM, "device scratch allocation of %zu bytes failed", sz);
        }
        bytes = sz;
        return GIPC_OK;
    }
    void release() {
        if (ptr) cudaFree(ptr);
        ptr = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(ptr); }
};

struct gipc_ctx {
    int device = 0;
    static constexpr int kSlots = 16;
    gipc_scratch slot[kSlots];
    void release_all() {
        for (auto& s : slot) s.release();
    }
};
