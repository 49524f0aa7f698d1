// Assembly of the Gauss-Newton system into 3x3-block BSR by key sort.
//
// H = M + sum_e P_e^T H_e P_e and g = g_0 + sum_e P_e^T g_e (Alg. 1, the mass
// plus the projected local Hessians; supplement Sec. S6 decomposes the system
// matrix into exactly these local blocks).  The paper never forms H; this
// library does, so the PCG can stream a compact BSR matrix.
//
// Pattern (bit-exact, deterministic):
//   1. count   every element adds s contributions to each of its s rows
//   2. scan    row_start = exclusive prefix of the row counts
//   3. fill    each contribution writes the 64-bit key (col << 32 | cid + 1)
//              into its row bucket (order within a bucket is arbitrary);
//              cid = element_id << 4 | a << 2 | b, the mass key is (i << 32 | 0)
//   4. sort    each row bucket by key: warp-wide bitonic sort in shared memory
//              for rows up to 512 contributions, block-wide up to 8192, and one
//              block sorting in global memory beyond that (rare hub vertices)
//   5. unique  distinct columns per row -> row_nnzb -> rowptr (scan)
//   6. emit    colidx and the first contribution of every block
// Values (deterministic): one thread per block sums its contributions in key
// order, i.e. the mass first, then elements in ascending id (tetrahedra before
// stencils), exactly the order of a sequential reference.  The diagonal block
// of row r also sums the slot gradients of its contributors into g[r].
// Threads take the blocks in falling order of contribution count (a stable
// counting sort of the block ids), so a warp's lanes loop equally long: an
// instruction costs its full issue slots however few lanes are active, which
// matters most for float64 adds (1/64 of the float32 rate).  Each block is
// still summed alone and in key order, so the values do not depend on it.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "context.cuh"
#include "scan.cuh"

namespace gipc {
namespace {

constexpr int kWarpRowMax = 512;
constexpr int kBlockRowMax = 8192;
constexpr int kSortWarps = 4;

enum Slot { S_ROWCNT = 0, S_ROWSTART, S_KEYS, S_NNZB, S_SEG, S_ELEMN3, S_MISC, S_SCAN, S_ROWPTR64, S_ORDER = 61 };

// Blocks are evaluated in order of falling contribution count so that the lanes of a warp run
// loops of equal length: counts are binned into kOrderBins (the last bin holds every count above),
// and each warp of the ordering kernels takes kOrderChunk consecutive blocks.
constexpr int kOrderBins = 32;
constexpr int kOrderChunk = 1024;

struct ElemList {
    const int32_t* idx;
    int64_t count;
    int mode;
    const void* hess;
    const double* lam;
    const double* grad;
};

__device__ __forceinline__ int elem_verts(const int32_t* __restrict__ idx, int64_t count, int64_t e, bool is_tet,
                                          int64_t n, int32_t v[4]) {
    if (is_tet) {
        int32_t s = 4;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            v[j] = idx[j * count + e];
            if (v[j] < 0 || v[j] >= n) s = 0;
        }
        return s;
    }
    const int type = decode_stencil(idx[e], idx[count + e], idx[2 * count + e], idx[3 * count + e], v);
    if (type < 0) return 0;
    const int s = stencil_verts(type);
    for (int j = 0; j < s; ++j)
        if (v[j] >= n) return 0;
    return s;
}

__global__ void init_rows_kernel(int32_t* __restrict__ row_cnt, int64_t n, int with_mass) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) row_cnt[i] = with_mass ? 1 : 0;
}

__global__ void count_kernel(ElemList tets, ElemList sts, int64_t n, int32_t* __restrict__ row_cnt,
                             uint8_t* __restrict__ elem_n3) {
    const int64_t total = tets.count + sts.count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const bool is_tet = e < tets.count;
        const ElemList& L = is_tet ? tets : sts;
        const int64_t el = is_tet ? e : e - tets.count;
        int32_t v[4];
        const int s = elem_verts(L.idx, L.count, el, is_tet, n, v);
        elem_n3[e] = (uint8_t)(3 * s);
        for (int a = 0; a < s; ++a) atomicAdd(row_cnt + v[a], s);
    }
}

__global__ void init_cursor_kernel(const int64_t* __restrict__ row_start, unsigned long long* __restrict__ cursor,
                                   uint64_t* __restrict__ keys, int64_t n, int with_mass) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t st = row_start[i];
    if (with_mass) keys[st] = (uint64_t)i << 32;
    cursor[i] = (unsigned long long)(st + (with_mass ? 1 : 0));
}

__global__ void fill_kernel(ElemList tets, ElemList sts, int64_t n, const uint8_t* __restrict__ elem_n3,
                            unsigned long long* __restrict__ cursor, uint64_t* __restrict__ keys) {
    const int64_t total = tets.count + sts.count;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int s = elem_n3[e] / 3;
        if (s == 0) continue;
        const bool is_tet = e < tets.count;
        const ElemList& L = is_tet ? tets : sts;
        const int64_t el = is_tet ? e : e - tets.count;
        int32_t v[4];
        elem_verts(L.idx, L.count, el, is_tet, n, v);
        for (int a = 0; a < s; ++a) {
            const unsigned long long pos = atomicAdd(cursor + v[a], (unsigned long long)s);
            for (int b = 0; b < s; ++b) {
                const uint32_t cid = (uint32_t)((e << 4) | (a << 2) | b) + 1u;
                keys[pos + b] = ((uint64_t)(uint32_t)v[b] << 32) | cid;
            }
        }
    }
}

__device__ __forceinline__ uint32_t key_col(uint64_t k) { return (uint32_t)(k >> 32); }

// Bitonic sort of P (power of two) keys in shared memory by `nthr` cooperating threads.
template <bool BLOCK>
__device__ __forceinline__ void bitonic_sort(uint64_t* buf, int P, int t0, int nthr) {
    for (int size = 2; size <= P; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = t0; t < (P >> 1); t += nthr) {
                const int i = (t / stride) * 2 * stride + (t % stride);
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const uint64_t a = buf[i], b = buf[j];
                if ((a > b) == up) {
                    buf[i] = b;
                    buf[j] = a;
                }
            }
            if (BLOCK) __syncthreads();
            else __syncwarp();
        }
    }
}

__device__ __forceinline__ int next_pow2(int L) {
    int P = 32;
    while (P < L) P <<= 1;
    return P;
}

// Bitonic sort of the 32 K keys a warp holds in registers (position j 32 + lane in v[j]):
// compare-exchanges between lanes by shuffles, between a lane's own keys in place.  The same
// network as bitonic_sort, without shared memory (whose bandwidth bounded the staged version).
template <int K>
__device__ __forceinline__ void warp_sort_regs(uint64_t (&v)[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int size = 2; size <= 32 * K; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= 32) {
                const int js = stride >> 5;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    if (j & js) continue;
                    const bool up = ((j * 32 + lane) & size) == 0;
                    const uint64_t a = v[j], b = v[j | js];
                    const bool sw = (a > b) == up;
                    v[j] = sw ? b : a;
                    v[j | js] = sw ? a : b;
                }
            } else {
                const bool lower = (lane & stride) == 0;
#pragma unroll
                for (int j = 0; j < K; ++j) {
                    const uint64_t a = v[j], b = __shfl_xor_sync(0xffffffffu, a, stride);
                    const bool up = ((j * 32 + lane) & size) == 0;
                    const uint64_t lo = a < b ? a : b, hi = a < b ? b : a;
                    v[j] = (lower == up) ? lo : hi;   // the pair's lower slot gets the minimum when ascending
                }
            }
        }
    }
}

// One row of L <= 32 K keys at keys[st ..): sort in registers, write back, count distinct columns.
template <int K>
__device__ __forceinline__ int sort_row_regs(uint64_t* __restrict__ keys, int64_t st, int L) {
    const int lane = threadIdx.x & 31;
    uint64_t v[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = j * 32 + lane;
        v[j] = p < L ? keys[st + p] : ~0ull;
    }
    warp_sort_regs<K>(v);
    int heads = 0;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int p = j * 32 + lane;
        const uint64_t up1 = __shfl_up_sync(0xffffffffu, v[j], 1);
        const uint64_t wrap = j > 0 ? __shfl_sync(0xffffffffu, v[j > 0 ? j - 1 : 0], 31) : 0ull;
        const uint64_t prev = lane > 0 ? up1 : wrap;
        if (p < L) {
            keys[st + p] = v[j];
            heads += (p == 0 || key_col(prev) != key_col(v[j])) ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) heads += __shfl_xor_sync(0xffffffffu, heads, o);
    return heads;
}

// Sort each row bucket of at most kWarpRowMax keys with one warp (keys in registers); longer rows
// are queued.
__global__ void __launch_bounds__(32 * kSortWarps)
sort_rows_warp_kernel(const int64_t* __restrict__ row_start, uint64_t* __restrict__ keys, int64_t n,
                      int32_t* __restrict__ row_nnzb, int32_t* __restrict__ long_rows, int32_t* __restrict__ n_long) {
    static_assert(kWarpRowMax == 512, "the register sort dispatch covers rows of up to 512 keys");
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t r = (int64_t)blockIdx.x * kSortWarps + w; r < n; r += (int64_t)gridDim.x * kSortWarps) {
        const int64_t st = row_start[r];
        const int L = (int)(row_start[r + 1] - st);
        if (L > kWarpRowMax) {
            if (lane == 0) long_rows[atomicAdd(n_long, 1)] = (int32_t)r;
            continue;
        }
        const int P = next_pow2(L);
        int heads;
        if (P == 32) heads = sort_row_regs<1>(keys, st, L);
        else if (P == 64) heads = sort_row_regs<2>(keys, st, L);
        else if (P == 128) heads = sort_row_regs<4>(keys, st, L);
        else if (P == 256) heads = sort_row_regs<8>(keys, st, L);
        else heads = sort_row_regs<16>(keys, st, L);
        if (lane == 0) row_nnzb[r] = heads;
    }
}

// Rows longer than kWarpRowMax: one block per row (grid-stride over the queue); rows longer
// than kBlockRowMax are queued again (huge_rows) for the global-memory sort.
__global__ void __launch_bounds__(1024)
sort_rows_block_kernel(const int64_t* __restrict__ row_start, uint64_t* __restrict__ keys,
                       int32_t* __restrict__ row_nnzb, const int32_t* __restrict__ long_rows,
                       const int32_t* __restrict__ n_long, int32_t* __restrict__ huge_rows,
                       int32_t* __restrict__ n_huge) {
    extern __shared__ uint64_t buf[];
    __shared__ int heads_sh;
    const int cnt = *n_long;
    for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int64_t r = long_rows[q];
        const int64_t st = row_start[r];
        const int L = (int)(row_start[r + 1] - st);
        if (L > kBlockRowMax) {
            if (threadIdx.x == 0) huge_rows[atomicAdd(n_huge, 1)] = (int32_t)r;
            continue;
        }
        const int P = next_pow2(L);
        for (int t = threadIdx.x; t < P; t += blockDim.x) buf[t] = t < L ? keys[st + t] : ~0ull;
        if (threadIdx.x == 0) heads_sh = 0;
        __syncthreads();
        bitonic_sort<true>(buf, P, threadIdx.x, blockDim.x);
        int heads = 0;
        for (int t = threadIdx.x; t < L; t += blockDim.x) {
            const uint64_t k = buf[t];
            keys[st + t] = k;
            heads += (t == 0 || key_col(buf[t - 1]) != key_col(k)) ? 1 : 0;
        }
        atomicAdd(&heads_sh, heads);
        __syncthreads();
        if (threadIdx.x == 0) row_nnzb[r] = heads_sh;
        __syncthreads();
    }
}

// Rows longer than kBlockRowMax: one block sorts the row in place in global memory with an
// ascending-only bitonic network (each merge starts with a "flip" compare), which sorts any
// length L: positions >= L act as +infinity and never take part in a swap.
__global__ void __launch_bounds__(1024)
sort_rows_global_kernel(const int64_t* __restrict__ row_start, uint64_t* __restrict__ keys,
                        int32_t* __restrict__ row_nnzb, const int32_t* __restrict__ huge_rows,
                        const int32_t* __restrict__ n_huge) {
    __shared__ int heads_sh;
    const int cnt = *n_huge;
    for (int q = blockIdx.x; q < cnt; q += gridDim.x) {
        const int64_t r = huge_rows[q];
        uint64_t* K = keys + row_start[r];
        const int64_t L = row_start[r + 1] - row_start[r];
        int64_t P = 1;
        while (P < L) P <<= 1;
        for (int64_t k = 2; k <= P; k <<= 1) {
            const int64_t h = k >> 1;
            for (int64_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                const int64_t blk = (i / h) * k, o = i % h;
                const int64_t a = blk + o, b = blk + k - 1 - o;
                if (b < L && K[a] > K[b]) {
                    const uint64_t t = K[a];
                    K[a] = K[b];
                    K[b] = t;
                }
            }
            __syncthreads();
            for (int64_t j = k >> 2; j > 0; j >>= 1) {
                for (int64_t i = threadIdx.x; i < P / 2; i += blockDim.x) {
                    const int64_t a = (i / j) * 2 * j + (i % j), b = a + j;
                    if (b < L && K[a] > K[b]) {
                        const uint64_t t = K[a];
                        K[a] = K[b];
                        K[b] = t;
                    }
                }
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) heads_sh = 0;
        __syncthreads();
        int heads = 0;
        for (int64_t t = threadIdx.x; t < L; t += blockDim.x)
            heads += (t == 0 || key_col(K[t - 1]) != key_col(K[t])) ? 1 : 0;
        atomicAdd(&heads_sh, heads);
        __syncthreads();
        if (threadIdx.x == 0) row_nnzb[r] = heads_sh;
        __syncthreads();
    }
}

__global__ void rowptr32_kernel(const int64_t* __restrict__ rp64, int32_t* __restrict__ rp32, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i <= n) rp32[i] = (int32_t)rp64[i];
}

// One warp per row: column indices and the first contribution (segment start) of every block.
__global__ void emit_kernel(const int64_t* __restrict__ row_start, const uint64_t* __restrict__ keys,
                            const int64_t* __restrict__ rowptr, int64_t n, int32_t* __restrict__ colidx,
                            int64_t* __restrict__ seg) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t r = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < n; r += warps) {
        const int64_t st = row_start[r], L = row_start[r + 1] - st;
        const int64_t out0 = rowptr[r];
        int64_t run = 0;
        for (int64_t base = 0; base < L; base += 32) {
            const int64_t t = base + lane;
            bool h = false;
            uint32_t col = 0;
            if (t < L) {
                col = key_col(keys[st + t]);
                h = t == 0 || key_col(keys[st + t - 1]) != col;
            }
            const unsigned m = __ballot_sync(0xffffffffu, h);
            if (h) {
                const int64_t rank = run + __popc(m & ((1u << lane) - 1u));
                colidx[out0 + rank] = (int32_t)col;
                seg[out0 + rank] = st + t;
            }
            run += __popc(m);
        }
    }
}

__global__ void seg_end_kernel(int64_t* __restrict__ seg, const int64_t* __restrict__ rowptr,
                               const int64_t* __restrict__ row_start, int64_t n) {
    seg[rowptr[n]] = row_start[n];
}

__global__ void grad_init_kernel(const double* __restrict__ g0, double* __restrict__ g, int64_t n3) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3) g[i] = g0 ? g0[i] : 0.0;
}

// Round-to-nearest arithmetic without contraction into FMA, so a block sum is the plain
// sequence of IEEE products and additions in contribution order.
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }

// One thread per block: in-order sum of its contributions (mass first, then elements by id).
// Bin of block b: kOrderBins - 1 for the fewest contributions down to 0 for the most.
__device__ __forceinline__ int order_bin(const int64_t* __restrict__ seg, int64_t b) {
    const int64_t c = seg[b + 1] - seg[b];
    return kOrderBins - 1 - (int)(c < kOrderBins - 1 ? c : kOrderBins - 1);
}

// hist[bin * nchunk + chunk] = blocks of the bin in the chunk (one warp per chunk of kOrderChunk).
__global__ void order_hist_kernel(const int64_t* __restrict__ seg, int64_t nnzb, int64_t nchunk,
                                  int32_t* __restrict__ hist) {
    __shared__ int32_t cnt[8][kOrderBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockIdx.x * 8 + w;
    if (chunk >= nchunk) return;
    cnt[w][lane] = 0;
    __syncwarp();
    const int64_t b0 = chunk * kOrderChunk;
    for (int r = 0; r < kOrderChunk / 32; ++r) {
        const int64_t b = b0 + r * 32 + lane;
        const int bin = b < nnzb ? order_bin(seg, b) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, bin);
        if (bin >= 0 && (same & ((1u << lane) - 1u)) == 0u) cnt[w][bin] += __popc(same);
        __syncwarp();
    }
    hist[(int64_t)lane * nchunk + chunk] = cnt[w][lane];
}

// order[off[bin * nchunk + chunk] + rank] = b: a stable counting sort of all blocks by bin, with
// off the exclusive prefix of hist (bin-major, so every chunk's blocks of a bin follow the
// previous chunk's).
__global__ void order_scatter_kernel(const int64_t* __restrict__ seg, int64_t nnzb, int64_t nchunk,
                                     const int64_t* __restrict__ off, int32_t* __restrict__ order) {
    __shared__ int64_t pos[8][kOrderBins];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t chunk = (int64_t)blockIdx.x * 8 + w;
    if (chunk >= nchunk) return;
    pos[w][lane] = off[(int64_t)lane * nchunk + chunk];
    __syncwarp();
    const int64_t b0 = chunk * kOrderChunk;
    for (int r = 0; r < kOrderChunk / 32; ++r) {
        const int64_t b = b0 + r * 32 + lane;
        const int bin = b < nnzb ? order_bin(seg, b) : -1;
        const unsigned same = __match_any_sync(0xffffffffu, bin);
        const unsigned below = same & ((1u << lane) - 1u);
        if (bin >= 0) order[pos[w][bin] + __popc(below)] = (int32_t)b;
        __syncwarp();
        if (bin >= 0 && below == 0u) pos[w][bin] += __popc(same);
        __syncwarp();
    }
}

template <typename VT>
__global__ void values_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ seg, int64_t nnzb,
                              const int32_t* __restrict__ order, int64_t n, ElemList tets, ElemList sts,
                              const uint8_t* __restrict__ elem_n3, const double* __restrict__ mass,
                              VT* __restrict__ vals, const double* __restrict__ g0, double* __restrict__ gout) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnzb;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = order ? (int64_t)order[t] : t;
        const int64_t s0 = seg[b], s1 = seg[b + 1];
        VT acc[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] = VT(0);
        // a block is diagonal iff its first contribution is the mass or an (a, a) sub-block
        const uint64_t k0 = keys[s0];
        const uint32_t c0 = (uint32_t)k0;
        const bool diag = c0 == 0u || (((c0 - 1u) >> 2) & 3) == ((c0 - 1u) & 3);
        const int64_t row = key_col(k0);
        double ga[3] = {0.0, 0.0, 0.0};
        if (gout && diag && g0) {
#pragma unroll
            for (int i = 0; i < 3; ++i) ga[i] = g0[(int64_t)i * n + row];
        }
        for (int64_t p = s0; p < s1; ++p) {
            const uint64_t key = keys[p];
            const uint32_t cid1 = (uint32_t)key;
            if (cid1 == 0u) {  // mass m_i I_3 on the diagonal
                const VT m = (VT)mass[row];
                acc[0] = add_rn(acc[0], m);
                acc[4] = add_rn(acc[4], m);
                acc[8] = add_rn(acc[8], m);
                continue;
            }
            const uint32_t cid = cid1 - 1u;
            const int64_t e = cid >> 4;
            const int a = (cid >> 2) & 3, bb = cid & 3;
            const bool is_tet = e < tets.count;
            const ElemList& Lst = is_tet ? tets : sts;
            const int64_t el = is_tet ? e : e - tets.count;
            const int64_t cnt = Lst.count;
            if (Lst.mode == GIPC_HESS_DENSE) {
                const int n3 = elem_n3[e];
                const VT* H = static_cast<const VT*>(Lst.hess);
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        acc[3 * i + j] = add_rn(acc[3 * i + j], H[(int64_t)((3 * a + i) * n3 + 3 * bb + j) * cnt + el]);
            } else if (Lst.mode == GIPC_HESS_BLOCKS) {   // the 9 values are contiguous
                const VT* H = static_cast<const VT*>(Lst.hess) + (el * 16 + a * 4 + bb) * 9;
                VT h[9];
#pragma unroll
                for (int q = 0; q < 9; ++q) h[q] = H[q];
#pragma unroll
                for (int q = 0; q < 9; ++q) acc[q] = add_rn(acc[q], h[q]);
            } else {
                const VT* W = static_cast<const VT*>(Lst.hess);
                const VT lam = (VT)Lst.lam[el];
                VT wa[3], wb[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    wa[i] = W[(int64_t)(3 * a + i) * cnt + el];
                    wb[i] = W[(int64_t)(3 * bb + i) * cnt + el];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i)
#pragma unroll
                    for (int j = 0; j < 3; ++j) acc[3 * i + j] = add_rn(acc[3 * i + j], mul_rn(lam, mul_rn(wa[i], wb[j])));
            }
            if (gout && a == bb && Lst.grad) {
#pragma unroll
                for (int i = 0; i < 3; ++i) ga[i] = __dadd_rn(ga[i], Lst.grad[(int64_t)(3 * a + i) * cnt + el]);
            }
        }
#pragma unroll
        for (int q = 0; q < 9; ++q) vals[b * 9 + q] = acc[q];
        if (gout && diag) {
#pragma unroll
            for (int i = 0; i < 3; ++i) gout[(int64_t)i * n + row] = ga[i];
        }
    }
}

// out[r] = base[r] + the slot vectors of the elements containing vertex r, in ascending element
// id (tetrahedra first) -- the order the assembled gradient uses.  The row's keys are sorted by
// (column, contribution id), so the contributions of vertex r to itself form one run.
__global__ void scatter_rows_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ row_start, int64_t n,
                                    ElemList tets, ElemList sts, const double* __restrict__ base,
                                    double* __restrict__ out) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int64_t lo = row_start[r], hi = row_start[r + 1];
    while (lo < hi) {   // first key of column r
        const int64_t m = (lo + hi) >> 1;
        if (key_col(keys[m]) < (uint32_t)r) lo = m + 1;
        else hi = m;
    }
    double acc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) acc[i] = base ? base[(int64_t)i * n + r] : 0.0;
    for (int64_t p = lo; p < row_start[r + 1] && key_col(keys[p]) == (uint32_t)r; ++p) {
        const uint32_t cid1 = (uint32_t)keys[p];
        if (cid1 == 0u) continue;
        const uint32_t cid = cid1 - 1u;
        const int64_t e = cid >> 4;
        const int a = (cid >> 2) & 3;
        const bool is_tet = e < tets.count;
        const ElemList& Lst = is_tet ? tets : sts;
        const int64_t el = is_tet ? e : e - tets.count;
        if (!Lst.grad) continue;
#pragma unroll
        for (int i = 0; i < 3; ++i) acc[i] = __dadd_rn(acc[i], Lst.grad[(int64_t)(3 * a + i) * Lst.count + el]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) out[(int64_t)i * n + r] = acc[i];
}

// Grid for `work` items at `threads` per CTA, capped at `per_sm` CTAs per SM of the current device.
inline unsigned blocks_for(int64_t work, int threads, int per_sm = 32) { return grid_for(work, threads, per_sm); }
// One CTA per SM of the current device (the long-row sorts walk their rows in a grid-stride loop).
inline unsigned one_per_sm() { return (unsigned)std::max(1, device_facts().sms); }

}  // namespace
}  // namespace gipc

extern "C" gipc_status gipc_assemble_bsr(gipc_ctx* ctx, int64_t n, const gipc_elements* stencils_h,
                                         const gipc_elements* tets_h, const double* mass, const double* grad_base,
                                         gipc_bsr* bsr, double* grad_out, void* stream) {
    using namespace gipc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx || !bsr) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: null context or bsr");
    if (n < 0 || n >= INT32_MAX) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: n out of range");
    if (bsr->prec != GIPC_FP64 && bsr->prec != GIPC_MIXED)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: unknown bsr precision");
    if (!bsr->rowptr) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: null rowptr");
    ElemList L[2] = {};
    const gipc_elements* in[2] = {tets_h, stencils_h};
    for (int q = 0; q < 2; ++q) {
        if (!in[q] || in[q]->count == 0) continue;
        const gipc_elements& E = *in[q];
        if (E.count < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: negative element count");
        if (!E.idx || !E.hess) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: null element indices/blocks");
        if (E.hess_mode != GIPC_HESS_DENSE && E.hess_mode != GIPC_HESS_RANK1 && E.hess_mode != GIPC_HESS_BLOCKS)
            return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: unknown Hessian mode");
        if (q == 0 && E.hess_mode == GIPC_HESS_RANK1)
            return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: tetrahedra need dense blocks");
        if (E.hess_mode == GIPC_HESS_RANK1 && !E.lam)
            return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: rank-one blocks need lam");
        L[q] = {E.idx, E.count, E.hess_mode, E.hess, E.lam, E.grad};
    }
    const int64_t ne = L[0].count + L[1].count;
    if (ne >= (int64_t)(1 << 28) - 1) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: too many elements");
    const int with_mass = mass != nullptr;
    bsr->n = n;
    if (n == 0) {
        bsr->nnzb = 0;
        return cudaMemsetAsync(bsr->rowptr, 0, sizeof(int32_t), s) == cudaSuccess ? GIPC_OK
               : fail(GIPC_ERR_CUDA, "gipc_assemble_bsr: memset failed");
    }
    const int64_t cbound = 16 * ne + n;
    gipc_status st;
    if ((st = ctx->slot[S_ROWCNT].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_ROWSTART].reserve(sizeof(int64_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_KEYS].reserve(sizeof(uint64_t) * cbound)) != GIPC_OK) return st;
    if ((st = ctx->slot[S_NNZB].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_ELEMN3].reserve(ne + 1)) != GIPC_OK) return st;
    if ((st = ctx->slot[S_MISC].reserve(sizeof(uint64_t) * n + sizeof(int32_t) * (2 * n + 4))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_SCAN].reserve(sizeof(int64_t) * scan_scratch_words(n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_ROWPTR64].reserve(sizeof(int64_t) * (n + 1))) != GIPC_OK) return st;
    int32_t* row_cnt = ctx->slot[S_ROWCNT].as<int32_t>();
    int64_t* row_start = ctx->slot[S_ROWSTART].as<int64_t>();
    uint64_t* keys = ctx->slot[S_KEYS].as<uint64_t>();
    int32_t* row_nnzb = ctx->slot[S_NNZB].as<int32_t>();
    uint8_t* elem_n3 = ctx->slot[S_ELEMN3].as<uint8_t>();
    unsigned long long* cursor = ctx->slot[S_MISC].as<unsigned long long>();
    int32_t* long_rows = reinterpret_cast<int32_t*>(cursor + n);
    int32_t* n_long = long_rows + n;
    int32_t* n_huge = n_long + 1;
    int32_t* huge_rows = n_huge + 1;
    int64_t* scan_tmp = ctx->slot[S_SCAN].as<int64_t>();
    int64_t* rowptr64 = ctx->slot[S_ROWPTR64].as<int64_t>();

    ctx->prof.start(GIPC_PROF_ASM_PATTERN, s);
    init_rows_kernel<<<blocks_for(n, 256, 1 << 20), 256, 0, s>>>(row_cnt, n, with_mass);
    if (ne > 0) count_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(L[0], L[1], n, row_cnt, elem_n3);
    if (exclusive_scan<int32_t>(row_cnt, row_start, n, scan_tmp, s) != cudaSuccess)
        return check_launch("gipc_assemble_bsr: scan");
    init_cursor_kernel<<<blocks_for(n, 256, 1 << 20), 256, 0, s>>>(row_start, cursor, keys, n, with_mass);
    if (ne > 0) fill_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(L[0], L[1], n, elem_n3, cursor, keys);
    if (cudaMemsetAsync(n_long, 0, 2 * sizeof(int32_t), s) != cudaSuccess)
        return fail(GIPC_ERR_CUDA, "gipc_assemble_bsr: memset failed");
    sort_rows_warp_kernel<<<blocks_for(n, kSortWarps, 64), 32 * kSortWarps, 0, s>>>(
        row_start, keys, n, row_nnzb, long_rows, n_long);
    // raises the kernel's shared memory limit on this device (once per device)
    if (kernel_occupancy((const void*)sort_rows_block_kernel, 1024, kBlockRowMax * sizeof(uint64_t)) <= 0)
        return fail(GIPC_ERR_CUDA, "gipc_assemble_bsr: long-row sort does not fit the device");
    sort_rows_block_kernel<<<one_per_sm(), 1024, kBlockRowMax * sizeof(uint64_t), s>>>(row_start, keys, row_nnzb, long_rows,
                                                                          n_long, huge_rows, n_huge);
    sort_rows_global_kernel<<<one_per_sm(), 1024, 0, s>>>(row_start, keys, row_nnzb, huge_rows, n_huge);
    if (exclusive_scan<int32_t>(row_nnzb, rowptr64, n, scan_tmp, s) != cudaSuccess)
        return check_launch("gipc_assemble_bsr: scan");
    rowptr32_kernel<<<blocks_for(n + 1, 256, 1 << 20), 256, 0, s>>>(rowptr64, bsr->rowptr, n);
    ctx->prof.stop(GIPC_PROF_ASM_PATTERN, s);
    if ((st = check_launch("gipc_assemble_bsr: pattern")) != GIPC_OK) return st;
    int64_t host_vals[2] = {0, 0};
    cudaMemcpyAsync(&host_vals[0], rowptr64 + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return check_launch("gipc_assemble_bsr: sync");
    const int64_t nnzb = host_vals[0];
    if (nnzb >= INT32_MAX) return fail(GIPC_ERR_CAPACITY, "gipc_assemble_bsr: nnzb exceeds int32");
    bsr->nnzb = nnzb;
    if (nnzb > bsr->capacity)
        return fail(GIPC_ERR_CAPACITY, "gipc_assemble_bsr: %lld blocks needed, capacity %lld", (long long)nnzb,
                    (long long)bsr->capacity);
    if (nnzb > 0 && (!bsr->colidx || !bsr->vals)) return fail(GIPC_ERR_INVALID_ARG, "gipc_assemble_bsr: null colidx/vals");
    if ((st = ctx->slot[S_SEG].reserve(sizeof(int64_t) * (nnzb + 1))) != GIPC_OK) return st;
    int64_t* seg = ctx->slot[S_SEG].as<int64_t>();
    // the block order of the values kernel: falling contribution count, stable
    const int64_t nchunk = (nnzb + kOrderChunk - 1) / kOrderChunk;
    const int64_t nbin = (int64_t)kOrderBins * nchunk;
    if ((st = ctx->slot[S_ORDER].reserve(sizeof(int64_t) * (nbin + 1) + sizeof(int32_t) * (nbin + nnzb))) != GIPC_OK)
        return st;
    if ((st = ctx->slot[S_SCAN].reserve(sizeof(int64_t) * scan_scratch_words(std::max(n, nbin) + 1))) != GIPC_OK)
        return st;
    scan_tmp = ctx->slot[S_SCAN].as<int64_t>();
    int64_t* bin_off = ctx->slot[S_ORDER].as<int64_t>();
    int32_t* bin_hist = reinterpret_cast<int32_t*>(bin_off + nbin + 1);
    int32_t* order = bin_hist + nbin;
    ctx->prof.start(GIPC_PROF_ASM_VALUES, s);
    emit_kernel<<<blocks_for(n, 8, 64), 256, 0, s>>>(row_start, keys, rowptr64, n, bsr->colidx, seg);
    seg_end_kernel<<<1, 1, 0, s>>>(seg, rowptr64, row_start, n);
    if (grad_out) grad_init_kernel<<<blocks_for(3 * n, 256, 1 << 30), 256, 0, s>>>(grad_base, grad_out, 3 * n);
    if (nnzb > 0) {
        const unsigned ob = (unsigned)((nchunk + 7) / 8);
        order_hist_kernel<<<ob, 256, 0, s>>>(seg, nnzb, nchunk, bin_hist);
        if (exclusive_scan<int32_t>(bin_hist, bin_off, nbin, scan_tmp, s) != cudaSuccess)
            return check_launch("gipc_assemble_bsr: scan");
        order_scatter_kernel<<<ob, 256, 0, s>>>(seg, nnzb, nchunk, bin_off, order);
        if (bsr->prec == GIPC_FP64)
            values_kernel<double><<<blocks_for(nnzb, 128), 128, 0, s>>>(keys, seg, nnzb, order, n, L[0], L[1], elem_n3,
                                                                      mass, static_cast<double*>(bsr->vals), grad_base,
                                                                      grad_out);
        else
            values_kernel<float><<<blocks_for(nnzb, 128), 128, 0, s>>>(keys, seg, nnzb, order, n, L[0], L[1], elem_n3,
                                                                     mass, static_cast<float*>(bsr->vals), grad_base,
                                                                     grad_out);
    }
    ctx->prof.stop(GIPC_PROF_ASM_VALUES, s);
    return check_launch("gipc_assemble_bsr: values");
}

extern "C" gipc_status gipc_scatter_elements(gipc_ctx* ctx, int64_t n, const gipc_elements* stencils_h,
                                             const gipc_elements* tets_h, const double* base, double* out,
                                             void* stream) {
    using namespace gipc;
    cudaStream_t s = (cudaStream_t)stream;
    if (!ctx || !out) return fail(GIPC_ERR_INVALID_ARG, "gipc_scatter_elements: null context or output");
    if (n <= 0 || n >= INT32_MAX) return fail(GIPC_ERR_INVALID_ARG, "gipc_scatter_elements: n out of range");
    ElemList L[2] = {};
    const gipc_elements* in[2] = {tets_h, stencils_h};
    for (int q = 0; q < 2; ++q) {
        if (!in[q] || in[q]->count == 0) continue;
        const gipc_elements& E = *in[q];
        if (E.count < 0 || !E.idx) return fail(GIPC_ERR_INVALID_ARG, "gipc_scatter_elements: bad element list");
        L[q] = {E.idx, E.count, GIPC_HESS_DENSE, nullptr, nullptr, E.grad};
    }
    const int64_t ne = L[0].count + L[1].count;
    if (ne >= (int64_t)(1 << 28) - 1) return fail(GIPC_ERR_INVALID_ARG, "gipc_scatter_elements: too many elements");
    const int64_t cbound = 16 * ne + n;
    gipc_status st;
    if ((st = ctx->slot[S_ROWCNT].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_ROWSTART].reserve(sizeof(int64_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_KEYS].reserve(sizeof(uint64_t) * cbound)) != GIPC_OK) return st;
    if ((st = ctx->slot[S_NNZB].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_ELEMN3].reserve(ne + 1)) != GIPC_OK) return st;
    if ((st = ctx->slot[S_MISC].reserve(sizeof(uint64_t) * n + sizeof(int32_t) * (2 * n + 4))) != GIPC_OK) return st;
    if ((st = ctx->slot[S_SCAN].reserve(sizeof(int64_t) * scan_scratch_words(n + 1))) != GIPC_OK) return st;
    int32_t* row_cnt = ctx->slot[S_ROWCNT].as<int32_t>();
    int64_t* row_start = ctx->slot[S_ROWSTART].as<int64_t>();
    uint64_t* keys = ctx->slot[S_KEYS].as<uint64_t>();
    int32_t* row_nnzb = ctx->slot[S_NNZB].as<int32_t>();
    uint8_t* elem_n3 = ctx->slot[S_ELEMN3].as<uint8_t>();
    unsigned long long* cursor = ctx->slot[S_MISC].as<unsigned long long>();
    int32_t* long_rows = reinterpret_cast<int32_t*>(cursor + n);
    int32_t* n_long = long_rows + n;
    int32_t* n_huge = n_long + 1;
    int32_t* huge_rows = n_huge + 1;
    int64_t* scan_tmp = ctx->slot[S_SCAN].as<int64_t>();
    init_rows_kernel<<<blocks_for(n, 256, 1 << 20), 256, 0, s>>>(row_cnt, n, 0);
    if (ne > 0) count_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(L[0], L[1], n, row_cnt, elem_n3);
    if (exclusive_scan<int32_t>(row_cnt, row_start, n, scan_tmp, s) != cudaSuccess)
        return check_launch("gipc_scatter_elements: scan");
    init_cursor_kernel<<<blocks_for(n, 256, 1 << 20), 256, 0, s>>>(row_start, cursor, keys, n, 0);
    if (ne > 0) fill_kernel<<<blocks_for(ne, 256), 256, 0, s>>>(L[0], L[1], n, elem_n3, cursor, keys);
    if (cudaMemsetAsync(n_long, 0, 2 * sizeof(int32_t), s) != cudaSuccess)
        return fail(GIPC_ERR_CUDA, "gipc_scatter_elements: memset failed");
    sort_rows_warp_kernel<<<blocks_for(n, kSortWarps, 64), 32 * kSortWarps, 0, s>>>(row_start, keys, n, row_nnzb,
                                                                                       long_rows, n_long);
    if (kernel_occupancy((const void*)sort_rows_block_kernel, 1024, kBlockRowMax * sizeof(uint64_t)) <= 0)
        return fail(GIPC_ERR_CUDA, "gipc_scatter_elements: long-row sort does not fit the device");
    sort_rows_block_kernel<<<one_per_sm(), 1024, kBlockRowMax * sizeof(uint64_t), s>>>(row_start, keys, row_nnzb, long_rows,
                                                                          n_long, huge_rows, n_huge);
    sort_rows_global_kernel<<<one_per_sm(), 1024, 0, s>>>(row_start, keys, row_nnzb, huge_rows, n_huge);
    scatter_rows_kernel<<<blocks_for(n, 256, 1 << 20), 256, 0, s>>>(keys, row_start, n, L[0], L[1], base, out);
    return check_launch("gipc_scatter_elements");
}
