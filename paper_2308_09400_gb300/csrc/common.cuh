// Shared host/device helpers of the GIPC library (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gipc.h"

namespace gipc {

// Record a failure message for gipc_last_error() and return `st`.
gipc_status fail(gipc_status st, const char* fmt, ...);
// Map the last launch / runtime error to GIPC_ERR_CUDA with a message.
gipc_status check_launch(const char* what);

// Facts of the current device, looked up once per device (thread-safe): its ordinal, SM count and
// whether it supports cooperative launches.  sms is 0 when no device is usable.
struct DeviceFacts {
    int device = -1;
    int sms = 0;
    bool coop = false;
};
DeviceFacts device_facts();
// CTAs of `threads` threads with `smem` bytes of dynamic shared memory that one SM of the current
// device holds at once for kernel `fn`; raises the kernel's dynamic shared memory limit on that
// device to `smem` first when needed.  Computed once per (kernel, device, threads, smem) under a
// lock; 0 on failure.
int kernel_occupancy(const void* fn, int threads, size_t smem);
// Grid size for `work` items at `per_block` items per CTA, capped at `per_sm` CTAs per SM of the
// current device (at least 1).
unsigned grid_for(int64_t work, int64_t per_block, int per_sm);

constexpr int kMaxStencilVerts = 4;

// Stencil type decoding from the sign pattern (paper Sec. 7.2).  Returns the
// type (0..6) or -1 for a malformed tuple; `v` receives vertex ids in slot order.
__host__ __device__ __forceinline__ int decode_stencil(int32_t i0, int32_t i1, int32_t i2,
                                                       int32_t i3, int32_t v[4]) {
    const int32_t NUL = GIPC_NULL_INDEX;
    if (i0 >= 0 && i1 >= 0) {
        if (i2 < 0 || i3 < 0) return -1;
        v[0] = i0; v[1] = i1; v[2] = i2; v[3] = i3;
        return GIPC_EE;
    }
    if (i0 >= 0) {  // i1 < 0
        if (i1 == NUL || i2 < 0 || i3 < 0) return -1;
        v[0] = i0; v[1] = ~i1; v[2] = i2; v[3] = i3;
        return GIPC_EE_PAR;
    }
    if (i0 == NUL) return -1;
    if (i1 >= 0) {
        if (i2 == NUL) {
            if (i3 != NUL) return -1;
            v[0] = ~i0; v[1] = i1; v[2] = 0; v[3] = 0;
            return GIPC_PP;
        }
        if (i2 < 0) return -1;
        if (i3 == NUL) {
            v[0] = ~i0; v[1] = i1; v[2] = i2; v[3] = 0;
            return GIPC_PE;
        }
        if (i3 < 0) return -1;
        v[0] = ~i0; v[1] = i1; v[2] = i2; v[3] = i3;
        return GIPC_PT;
    }
    if (i1 == NUL || i2 == NUL || i3 == NUL) return -1;
    if (i2 >= 0) {
        if (i3 >= 0) return -1;
        v[0] = ~i0; v[1] = ~i1; v[2] = i2; v[3] = ~i3;
        return GIPC_PE_PAR;
    }
    if (i3 >= 0) return -1;
    v[0] = ~i0; v[1] = ~i1; v[2] = ~i2; v[3] = ~i3;
    return GIPC_PP_PAR;
}

__host__ __device__ __forceinline__ int stencil_verts(int type) {
    return type == GIPC_PE ? 3 : (type == GIPC_PP ? 2 : 4);
}

}  // namespace gipc
