// Modified PCG with a 3x3 block-Jacobi preconditioner on a BSR matrix.
//
// Paper: the Newton system of Alg. 1 is solved by modified-PCG (Sec. 7.2,
// "Parallel solver optimizations", after Baraff and Witkin) with a simple 3x3
// block-diagonal preconditioner (Sec. 7.2, "Preconditioning of the CG solver")
// and stops when delta_new < 1e-4 delta_0 (Sec. 8).  The filter S zeroes
// constrained vertices ("modified" PCG).  Unlike the paper, which multiplies the
// local matrices directly, the matrix here is an assembled BSR.
//
// Per iteration two kernels run, both reading the solver scalars from device
// memory, so the host never waits inside the loop:
//   A  q = S(H c) and the partial dots c.q      -> last CTA: alpha = delta/(c.q)
//   B  x += alpha c; r -= alpha q; s = P^-1 r; partial dots r.s; grid barrier;
//      delta_new, beta, done; c = S(s + beta c)
// B is one cooperative launch; where its tiles do not fit in shared memory it
// runs as an update and a direction kernel.  Dots are reduced deterministically:
// every CTA writes one partial and the partials are summed in index order.  Once
// `done` is set every kernel returns immediately, so surplus launched iterations
// are no-ops.
//
// Product: gipc_pcg copies the matrix once per solve into SELL-32 slices (32
// block rows per slice; within each window of 1024 consecutive rows the rows are
// taken longest first by a stable bucket sort, so a slice's rows are of similar
// length and still neighbours in the mesh; entry-major within a slice), one lane
// per block row.  Each
// warp streams its slices into shared memory with cp.async.bulk and bounded
// mbarrier waits while it multiplies the previous group, and the kernel is
// launched with programmatic stream serialization, so it stages its first slice
// while the previous kernel ends.  The first product H x0 and the allocation-free
// solver use a plain kernel over the BSR rows (three lanes per block row).
//
// Mixed form: float32 blocks and a float32 product (row sums in float32); the
// block-Jacobi factors, s = P^-1 r and the direction are float32 as well, the
// direction's exact float64 image used for the x update and the dots (kept in memory
// by the separate kernels, converted where it is used by the persistent solver, whose
// phases are bound by memory rather than by the FP64 pipe); x, r, alpha, beta and
// the dots stay float64.  On GB300 a float64 operation, or
// a conversion between float64 and float32, issues at 1/64 of the float32 rate,
// so the float32 preconditioner and direction take about half the float64 work
// out of kernel B.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>
#include <cmath>

#include "common.cuh"
#include "context.cuh"
#include "scan.cuh"

namespace gipc {
namespace {

constexpr int kPcgThreads = 256;
constexpr int kRowsPerWarp = 10;  // row-ordered kernel: 3 lanes per row, lanes 30/31 idle
constexpr int kSellC = 32;        // sliced kernel: rows per slice (one lane per row)
constexpr int kVpt = 4;           // vertices per thread in the setup kernel
constexpr int kUpdT = 256;        // update kernel: vertices (= threads) per tile
constexpr int kUpdPerSm = 2;      // update kernel: resident CTAs per SM (persistent grid)
constexpr int kFuseMaxTiles = 8;  // fused update / direction: tiles per CTA kept in shared memory
constexpr int kDirEpt = 4;        // direction kernel: vector entries per thread

enum PcgSlot { P_VEC = 9, P_PINV = 10, P_PART = 11, P_PERM = 12, P_VEC32 = 13, P_SELL = 14, P_SLICE = 15, P_SCENE = 40,
               P_TRACE = 62, P_BATCH = 65 };

constexpr int kLenBuckets = 64;   // rows are ordered by min(blocks in row, 63), longest first
constexpr int kPermChunk = 1024;  // rows per chunk of the stable bucket sort (rows stay in their chunk)

struct PcgScalars {
    double delta_new, delta_old, delta0, alpha, beta, tol, pq;
    int iters, done, max_iter, status;
    int stop_indefinite;   // stop with GIPC_ERR_INDEFINITE on c.q <= 0 (one system, on request)
    unsigned count_a, count_b, count_0;
    unsigned scenes_done;   // batched solves: scenes that have stopped
    unsigned bar_count, bar_gen;   // grid barrier of the fused update / direction kernel
};

// Per-scene state of a batched solve (independent systems on disjoint vertex ranges).
struct SceneScalars {
    double delta0, delta;
    int iters, done, status, pad;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while the previous kernel of the stream finishes; it must wait here before it touches
// anything that kernel writes (a no-op when the launch was an ordinary one).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Lets the next kernel of the stream start launching (its CTAs still wait as above).
__device__ __forceinline__ void pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Block-wide sum (fixed order) -> thread 0.
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (w == 0) {
        t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    __syncthreads();
    return t;
}

// Publish this CTA's partial; returns true in exactly one (the last) CTA, which then sees all partials.
__device__ __forceinline__ bool publish_partial(double* part, double v, unsigned* counter) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        part[blockIdx.x] = v;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        last = prev == gridDim.x - 1;
    }
    __syncthreads();
    return last;
}

// Called by every thread of the last CTA: sums the partials with a fixed thread-to-partial map
// and a fixed tree, so the total is identical run to run (result valid in thread 0).
__device__ __forceinline__ double sum_partials(const double* part, int count) {
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += blockDim.x) s += __ldcg(part + i);
    return block_sum(s);
}

// Double-float numbers for the float-pair product: x = hi + lo with two float32 (|lo| <= half an
// ulp of hi).  Products use Dekker's exact float product (the FMA gives the rounding error of
// hi * hi), sums Knuth's TwoSum; every operation is an explicitly rounded float32 intrinsic, so
// the compiler cannot contract or reorder it.
struct __align__(8) fpair {
    float hi, lo;
    __device__ fpair(float h = 0.0f, float l = 0.0f) : hi(h), lo(l) {}
    __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ fpair two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return fpair(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ fpair fast_two_sum(float a, float b) {   // |a| >= |b| or a == 0
    const float s = __fadd_rn(a, b);
    return fpair(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ fpair operator+(fpair a, fpair b) {
    const fpair s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ fpair split_double(double x) {
    const float h = __double2float_rn(x);
    return fpair(h, __double2float_rn(x - (double)h));
}

// c + a b in each arithmetic (the generic product code calls these)
__device__ __forceinline__ double mac(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float mac(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ fpair mac(fpair a, fpair b, fpair c) {
    const float p = __fmul_rn(a.hi, b.hi);
    const float e = __fmaf_rn(a.hi, b.hi, -p);                                 // a.hi b.hi = p + e exactly
    const float t = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));            // a.lo b.lo (~2^-48) dropped
    const fpair s = two_sum(c.hi, p);
    return fast_two_sum(s.hi, __fadd_rn(c.lo, __fadd_rn(s.lo, t)));
}


// matrix values as the product stores them
__device__ __forceinline__ void store_val(double* d, double v) { *d = v; }
__device__ __forceinline__ void store_val(float* d, float v) { *d = v; }
__device__ __forceinline__ void store_val(fpair* d, double v) { *d = split_double(v); }

// y = (H p)_row,comp for this lane (3 lanes per row, rows taken in the length order of their chunk).
template <typename VT, typename PT>
__device__ __forceinline__ bool spmv_lane(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                          const VT* __restrict__ vals, const PT* __restrict__ p,
                                          const int32_t* __restrict__ perm, int64_t n, int64_t& row, int& comp,
                                          double& out) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (lane >= 3 * kRowsPerWarp) return false;
    const int64_t slot = warp * kRowsPerWarp + lane / 3;
    comp = lane % 3;
    if (slot >= n) return false;
    row = perm[slot];
    const int32_t b0 = rowptr[row], b1 = rowptr[row + 1];
    VT acc0 = VT(0), acc1 = VT(0);
    int32_t b = b0;
    // four blocks per step: the four column loads, then twelve value loads and twelve
    // gathers are all independent, so each lane keeps many memory requests in flight
    for (; b + 4 <= b1; b += 4) {
        int64_t cc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cc[u] = colidx[b + u];
        VT v[12];
        PT pv[12];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const VT* vp = vals + 9 * (int64_t)(b + u) + 3 * comp;
            const PT* pp = p + 3 * cc[u];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                v[3 * u + j] = vp[j];
                pv[3 * u + j] = pp[j];
            }
        }
#pragma unroll
        for (int u = 0; u < 4; u += 2) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                acc0 = fma(v[3 * u + j], (VT)pv[3 * u + j], acc0);
                acc1 = fma(v[3 * u + 3 + j], (VT)pv[3 * u + 3 + j], acc1);
            }
        }
    }
    for (; b < b1; ++b) {
        const int64_t c = colidx[b];
        const VT* vp = vals + 9 * (int64_t)b + 3 * comp;
        const PT* pp = p + 3 * c;
        acc0 = fma(vp[0], (VT)pp[0], acc0);
        acc0 = fma(vp[1], (VT)pp[1], acc0);
        acc0 = fma(vp[2], (VT)pp[2], acc0);
    }
    out = (double)(acc0 + acc1);
    return true;
}

// Stable bucket sort of the rows by length within each chunk of kPermChunk consecutive rows
// (deterministic): per-chunk histograms, a scan in (chunk, bucket) order, then one warp per chunk
// places its rows in order.  Keeping every row in its own chunk keeps the column gathers of a
// slice local (the mixed product gained 4%, the sphere-grid Newton products 4-10%, over one
// global sort; a slice's padding stays small because neighbouring rows have similar lengths).
__device__ __forceinline__ int len_key(const int32_t* __restrict__ rowptr, int64_t r) {
    int len = rowptr[r + 1] - rowptr[r];
    if (len > kLenBuckets - 1) len = kLenBuckets - 1;
    return kLenBuckets - 1 - len;  // longest first
}

__global__ void perm_hist_kernel(const int32_t* __restrict__ rowptr, int64_t n, int32_t* __restrict__ counts,
                                 int64_t chunks) {
    __shared__ int h[kLenBuckets];
    for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const int64_t r0 = (int64_t)blockIdx.x * kPermChunk;
    for (int64_t r = r0 + threadIdx.x; r < n && r < r0 + kPermChunk; r += blockDim.x) atomicAdd(&h[len_key(rowptr, r)], 1);
    __syncthreads();
    for (int i = threadIdx.x; i < kLenBuckets; i += blockDim.x) counts[(int64_t)blockIdx.x * kLenBuckets + i] = h[i];
}

__global__ void perm_scatter_kernel(const int32_t* __restrict__ rowptr, int64_t n, const int64_t* __restrict__ off,
                                    int64_t chunks, int32_t* __restrict__ perm) {
    __shared__ int64_t run[kLenBuckets];
    const int lane = threadIdx.x;
    for (int i = lane; i < kLenBuckets; i += 32) run[i] = off[(int64_t)blockIdx.x * kLenBuckets + i];
    __syncwarp();
    const int64_t r0 = (int64_t)blockIdx.x * kPermChunk;
    for (int t = 0; t < kPermChunk; t += 32) {
        const int64_t r = r0 + t + lane;
        const bool valid = r < n;
        const int key = valid ? len_key(rowptr, r) : kLenBuckets;
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        const int rank = __popc(grp & ((1u << lane) - 1u));
        if (valid) perm[run[key] + rank] = (int32_t)r;
        __syncwarp();
        if (valid && rank == 0) run[key] += __popc(grp);
        __syncwarp();
    }
}

// ---- sliced layout of the matrix for the solver (built once per solve) --------------------
// SELL-32: rows are taken 32 at a time in the chunk-wise length order (one slice per warp, one lane
// per row).  Slice s holds L_s steps (its longest row); step j stores block j of each of its 32
// rows side by side, entry-major: column indices at sell_col[(off_s + j)*32 + i] and entry k of
// the 3x3 block at sell_vals[((off_s + j)*9 + k)*32 + i].  Every value load of a warp then reads
// 32 consecutive words.  Shorter rows are padded with zero blocks (column 0); the kernel never
// reads the padding (each lane walks its own row length).

__global__ void sell_len_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ perm, int64_t n,
                                int64_t nsl, int32_t* __restrict__ slice_len) {
    const int64_t sl = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (sl >= nsl) return;
    int32_t L = 0;
    for (int i = 0; i < kSellC; ++i) {
        const int64_t slot = sl * kSellC + i;
        if (slot < n) {
            const int32_t r = perm[slot];
            const int32_t len = rowptr[r + 1] - rowptr[r];
            L = len > L ? len : L;
        }
    }
    slice_len[sl] = L;
}

template <typename VT, typename VD>
__global__ void sell_fill_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                 const VT* __restrict__ vals, const int32_t* __restrict__ perm, int64_t n, int64_t nsl,
                                 const int64_t* __restrict__ slice_off, int32_t* __restrict__ sell_col,
                                 VD* __restrict__ sell_vals) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nsl * kSellC) return;
    const int64_t sl = t / kSellC;
    const int i = (int)(t - sl * kSellC);
    const int64_t off = slice_off[sl], L = slice_off[sl + 1] - off;
    int32_t b0 = 0, len = 0;
    if (t < n) {
        const int32_t r = perm[t];
        b0 = rowptr[r];
        len = rowptr[r + 1] - b0;
    }
    for (int64_t j = 0; j < L; ++j) {
        const int64_t p = (off + j) * kSellC + i;
        const bool real = j < len;
        sell_col[p] = real ? colidx[b0 + j] : 0;
#pragma unroll
        for (int k = 0; k < 9; ++k)
            store_val(sell_vals + ((off + j) * 9 + k) * kSellC + i, real ? vals[9 * (int64_t)(b0 + j) + k] : VT(0));
    }
}

// ---- q = S(H c) over the SELL-32 layout, slices streamed into shared memory by bulk async copies ----
// Each warp owns NS staging buffers of U steps (U*9*32 values + U*32 column indices, both
// contiguous in the SELL-32 layout) and one mbarrier per buffer.  Lane 0 issues the bulk copies
// of the next groups (cp.async.bulk, completion counted on the buffer's mbarrier) before the warp
// waits for the current one, so HBM streams while the warp gathers the direction and multiplies.  The
// arithmetic order is that of the row-ordered kernel: block j of a row goes to accumulator j % 2
// for j < 4 floor(L / 4) and to accumulator 0 after that, each block adding its three products
// per entry in column order.  Waits are bounded: a wait that runs out records GIPC_ERR_TIMEOUT and
// the solve stops.
__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void async_proxy_fence() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar, uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for `parity` of `bar` for at most ~1 s of SM clock; false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > 2000000000ll) return false;
    return true;
}

// Staging geometry: U steps per group, W warps per CTA, NS buffers per warp.
template <typename VT, int U, int W, int NS>
struct StageLayout {
    static constexpr unsigned kValBytes = U * 9 * kSellC * sizeof(VT);
    static constexpr unsigned kColBytes = U * kSellC * sizeof(int32_t);
    static constexpr unsigned kBuf = kValBytes + kColBytes;   // per buffer (multiple of 128)
    static constexpr unsigned kWarpBytes = NS * kBuf;
    static constexpr unsigned kBlockBytes = W * kWarpBytes + W * NS * 8;
};

// Direction loads of the product.  Within one product launch the direction is read-only, so the
// gathers take the read-only data path; the persistent solver rewrites it every iteration and
// reads it with coherent loads (its grid barriers order the writes before them).
template <bool COHERENT>
__device__ __forceinline__ double ld_dir(const double* p) {
    if constexpr (COHERENT) return *p;
    else return __ldg(p);
}
template <bool COHERENT>
__device__ __forceinline__ float ld_dir(const float* p) {
    if constexpr (COHERENT) return *p;
    else return __ldg(p);
}
template <bool COHERENT>
__device__ __forceinline__ fpair ld_dir(const fpair* p) {
    const float2 v = COHERENT ? *reinterpret_cast<const float2*>(p) : __ldg(reinterpret_cast<const float2*>(p));
    return fpair(v.x, v.y);
}

// The dynamic shared memory of the launch (staging buffers, then the mbarriers).
__device__ __forceinline__ unsigned char* dyn_smem() {
    extern __shared__ __align__(128) unsigned char dsm[];
    return dsm;
}

// Per-warp state of the staging ring.  Buffer b of the warp is refilled by bulk copies that
// complete on mbarrier b; `parity` bit b is the phase parity to wait for next on buffer b and
// `base` the ring position of the current slice's group 0.  `pre_sl` is a slice whose first
// `pre_groups` groups are already in flight (-1: none).  The buffers' addresses are recomputed
// from the warp index where they are used, so the ring costs four registers.
template <typename VT, int U, int W, int NS>
struct StageRing {
    using Lay = StageLayout<VT, U, W, NS>;
    unsigned parity, base;
    int pre_sl, pre_groups;

    __device__ __forceinline__ static unsigned char* wbuf() { return dyn_smem() + (threadIdx.x >> 5) * Lay::kWarpBytes; }
    __device__ __forceinline__ static uint64_t* bars() {
        return reinterpret_cast<uint64_t*>(dyn_smem() + W * Lay::kWarpBytes) + NS * (threadIdx.x >> 5);
    }
    __device__ __forceinline__ void init() {
        if ((threadIdx.x & 31) == 0) {
            for (int b = 0; b < NS; ++b) mbar_init(bars() + b, 1);
            mbar_init_fence();
        }
        __syncwarp();
        parity = 0;
        base = 0;
        pre_sl = -1;
        pre_groups = 0;
    }
    // lane 0: stage group g of a slice (steps [g U, min((g+1) U, Ls)) at step offset off) into
    // buffer b; the matrix stream is marked evict-first in L2, so the solver's vectors stay there
    __device__ __forceinline__ void issue(unsigned b, const VT* sell_vals, const int32_t* sell_col, int64_t off,
                                          int64_t Ls, int64_t g) {
        const int64_t j0 = g * U;
        const int64_t steps = (Ls - j0) < U ? (Ls - j0) : U;
        const unsigned vb = (unsigned)(steps * 9 * kSellC * sizeof(VT)), cb = (unsigned)(steps * kSellC * sizeof(int32_t));
        unsigned char* dst = wbuf() + b * Lay::kBuf;
        uint64_t* bar = bars() + b;
        uint64_t policy;
        asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(policy));
        async_proxy_fence();
        mbar_expect_tx(bar, vb + cb);
        bulk_load(dst, sell_vals + (off + j0) * 9 * kSellC, vb, bar, policy);
        bulk_load(dst + Lay::kValBytes, sell_col + (off + j0) * kSellC, cb, bar, policy);
    }
    // put the leading NS - 1 groups of slice sl in flight (the matrix never changes, so this may
    // run ahead of anything that the product itself waits for)
    __device__ __forceinline__ void preissue(int64_t sl, int64_t nsl, const int64_t* slice_off, const VT* sell_vals,
                                             const int32_t* sell_col) {
        pre_sl = sl < nsl ? (int)sl : -1;
        pre_groups = 0;
        if (pre_sl < 0) return;
        const int64_t off = slice_off[pre_sl], Ls = slice_off[pre_sl + 1] - off;
        pre_groups = (int)std::min<int64_t>(NS - 1, (Ls + U - 1) / U);
        if ((threadIdx.x & 31) == 0)
            for (int g = 0; g < pre_groups; ++g) issue((base + (unsigned)g) % NS, sell_vals, sell_col, off, Ls, g);
    }
    __device__ __forceinline__ bool wait(unsigned b) {   // warp-uniform outcome
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(bars() + b, (parity >> b) & 1));
        parity ^= 1u << b;
        return ok;
    }
    // let the pre-issued copies land (before the CTA may exit)
    __device__ __forceinline__ void drain() {
        for (int g = 0; g < pre_groups; ++g) wait((base + (unsigned)g) % NS);
        pre_sl = -1;
        pre_groups = 0;
        __syncwarp();
    }
    // after a timed-out wait: let every copy that may still be in flight land
    __device__ __forceinline__ void drain_all() {
        for (int b = 0; b < NS; ++b) mbar_wait_bounded(bars() + b, (parity >> b) & 1);
        __syncwarp();
    }
};

// q = S(H c) over this warp's slices; returns this thread's part of c . q.  A warp takes one
// slice per round, in alternating directions (round r: r * warps + wid, then
// r * warps + warps - 1 - wid), so within a chunk's longest-first run long and short slices pair
// up; every thread's set of slices is fixed, so its partial sum is too.  The arithmetic order is
// that of the row-ordered kernel: block j of a row goes to accumulator j % 2 for j < 4 floor(L / 4)
// and to accumulator 0 after that, each block adding its three products per entry in column order.
// Pipeline per warp over the groups g of a slice: the copies of the next NS-1 groups are in flight
// while group g is multiplied; with NS >= 3 the direction entries of group g+1 are also gathered
// before group g is multiplied.
// Slices of a warp: one per round over the whole grid's warps in snake order (above).  The
// warps are numbered CTA-major (STRIDED = false: a CTA's warps take neighbouring slices) or
// warp-major (STRIDED: warp w of CTA b is number w * gridDim.x + b, so every CTA samples the whole
// matrix and the CTAs' totals even out: on the C1 system the busiest CTA carries 1.025 instead of
// 1.046 times the mean, and the 319 warps with a single slice spread over the CTAs).
// DOT_FROM_CG: the row's part of c . q takes c from the gathered float32 direction (exactly the
// float64 image c holds), so the float64 image need not be kept (the mixed persistent solver).
// live(sl) (warp-uniform) tells whether slice sl is multiplied at all; a skipped slice leaves its
// rows of q as they were and contributes nothing to the returned part.
struct EverySlice {
    __device__ __forceinline__ bool operator()(int64_t) const { return true; }
};

template <typename VT, typename PT, int U, int W, int NS, bool COHERENT, bool STRIDED = false,
          bool DOT_FROM_CG = false, typename Live = EverySlice>
__device__ __forceinline__ double spmv_slices(StageRing<VT, U, W, NS>& R, const int32_t* __restrict__ rowptr,
                                              const int64_t* __restrict__ slice_off, const int32_t* __restrict__ sell_col,
                                              const VT* __restrict__ sell_vals, const PT* cg, const double* c,
                                              const int32_t* __restrict__ perm, double* q, const uint8_t* __restrict__ fixed,
                                              int64_t n, int64_t nsl, bool& timed_out, const Live& live = Live()) {
    using Lay = StageLayout<VT, U, W, NS>;
    constexpr bool kPrefetchGather = NS >= 3;
    const int lane = threadIdx.x & 31;
    const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t wid = STRIDED ? (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x
                                : ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double d = 0.0;
    for (int64_t rnd = 0; rnd * warps < nsl && !timed_out; ++rnd) {
        const int64_t sl = rnd * warps + ((rnd & 1) ? warps - 1 - wid : wid);
        if (sl >= nsl) continue;
        if (!live(sl)) {
            if (sl == R.pre_sl) R.drain();   // its leading groups were staged: let them land
            continue;
        }
        const int64_t off = slice_off[sl], Ls = slice_off[sl + 1] - off;
        const int64_t G = (Ls + U - 1) / U;
        const int64_t slot = sl * kSellC + lane;
        const bool real = slot < n;
        const int64_t row = real ? perm[slot] : 0;
        const int64_t L = real ? rowptr[row + 1] - rowptr[row] : 0;
        const int64_t L4 = L & ~int64_t(3);
        VT a0[3] = {VT(0), VT(0), VT(0)}, a1[3] = {VT(0), VT(0), VT(0)};
        PT pc[U][3], pn[U][3];   // gathered direction of the current / next group
        auto gather = [&](unsigned b, int64_t g, PT (&pv)[U][3]) {
            const int32_t* sc = reinterpret_cast<const int32_t*>(R.wbuf() + b * Lay::kBuf + Lay::kValBytes);
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (g * U + u < L) {
                    const int64_t cj = sc[u * kSellC + lane];
#pragma unroll
                    for (int k = 0; k < 3; ++k) pv[u][k] = ld_dir<COHERENT>(cg + 3 * cj + k);
                }
        };
        if (lane == 0 && sl != R.pre_sl)   // (a pre-issued slice's leading groups are already in flight)
            for (int64_t g = 0; g < NS - 1 && g < G; ++g)
                R.issue((R.base + (unsigned)g) % NS, sell_vals, sell_col, off, Ls, g);
        R.pre_sl = -1;
        R.pre_groups = 0;
        if (kPrefetchGather && G > 0) {
            if (!R.wait(R.base % NS)) timed_out = true;
            else gather(R.base % NS, 0, pc);
        }
        for (int64_t g = 0; g < G && !timed_out; ++g) {
            const unsigned b = (R.base + (unsigned)g) % NS;
            // group g+NS-1 goes to the buffer group g-1 used (released at the end of iteration g-1)
            if (g + NS - 1 < G && lane == 0)
                R.issue((R.base + (unsigned)(g + NS - 1)) % NS, sell_vals, sell_col, off, Ls, g + NS - 1);
            if (kPrefetchGather) {
                if (g + 1 < G) {
                    const unsigned bn = (R.base + (unsigned)g + 1) % NS;
                    if (!R.wait(bn)) {
                        timed_out = true;
                        break;
                    }
                    gather(bn, g + 1, pn);
                }
            } else {
                if (!R.wait(b)) {
                    timed_out = true;
                    break;
                }
                gather(b, g, pc);
            }
            const VT* sv = reinterpret_cast<const VT*>(R.wbuf() + b * Lay::kBuf);
            const int64_t j0 = g * U;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t jj = j0 + u;
                if (jj < L) {
                    VT* a = (jj < L4 && (jj & 1)) ? a1 : a0;
#pragma unroll
                    for (int e = 0; e < 3; ++e)
#pragma unroll
                        for (int k = 0; k < 3; ++k)
                            a[e] = mac(sv[(u * 9 + 3 * e + k) * kSellC + lane], (VT)pc[u][k], a[e]);
                }
            }
            if (kPrefetchGather) {
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int k = 0; k < 3; ++k) pc[u][k] = pn[u][k];
            }
            __syncwarp();   // every lane is done with buffer b before it is refilled
        }
        R.base = (R.base + (unsigned)G) % NS;
        if (timed_out) break;
        if (real) {
            const bool fx = fixed && fixed[row];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const double y = fx ? 0.0 : (double)(a0[e] + a1[e]);
                q[3 * row + e] = y;
                if constexpr (DOT_FROM_CG) d += (double)cg[3 * row + e] * y;
                else d += c[3 * row + e] * y;
            }
        }
    }
    return d;
}

// ---- q = S(H c) over the SELL-32 layout, slices streamed into shared memory by bulk async copies ----
// Each warp owns NS staging buffers of U steps (U*9*32 values + U*32 column indices, both
// contiguous in the SELL-32 layout) and one mbarrier per buffer.  Lane 0 issues the bulk copies
// of the next groups (cp.async.bulk, completion counted on the buffer's mbarrier) before the warp
// waits for the current one, so HBM streams while the warp gathers the direction and multiplies.
// Waits are bounded: a wait that runs out records GIPC_ERR_TIMEOUT and the solve stops.
template <typename VT, typename PT, int U, int W, int NS>
__global__ void __launch_bounds__(W * 32)
pcg_spmv_tma_kernel(const int32_t* __restrict__ rowptr, const int64_t* __restrict__ slice_off,
                    const int32_t* __restrict__ sell_col, const VT* __restrict__ sell_vals, const PT* __restrict__ cg,
                    const double* __restrict__ c, const int32_t* __restrict__ perm, double* __restrict__ q,
                    const uint8_t* __restrict__ fixed, int64_t n, int64_t nsl, double* __restrict__ part,
                    PcgScalars* __restrict__ S) {
    StageRing<VT, U, W, NS> R;
    R.init();
    const int lane = threadIdx.x & 31;
    // The matrix does not depend on the previous kernel: the first slice's leading groups are put
    // in flight before waiting for it (under a programmatic dependent launch they overlap its tail).
    R.preissue(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, nsl, slice_off, sell_vals, sell_col);
    pdl_wait();
    if (S->done) {   // uniform: the solve has stopped; let the staged copies land, then leave
        R.drain();
        return;
    }
    bool timed_out = false;
    const double d = spmv_slices<VT, PT, U, W, NS, false>(R, rowptr, slice_off, sell_col, sell_vals, cg, c, perm, q,
                                                          fixed, n, nsl, timed_out);
    if (timed_out) {
        // let copies still in flight land before the CTA can exit, then stop the solve
        R.drain_all();
        if (lane == 0) {
            S->status = GIPC_ERR_TIMEOUT;
            S->done = 1;
        }
    }
    const double bs = block_sum(d);
    if (publish_partial(part, bs, &S->count_a)) {
        const double pq = sum_partials(part, gridDim.x);
        if (threadIdx.x == 0) {
            S->pq = pq;
            S->alpha = S->delta_new / pq;
            S->count_a = 0;
            if (S->stop_indefinite && pq <= 0.0) {   // no descent along c: H not positive definite
                S->status = GIPC_ERR_INDEFINITE;
                S->done = 1;
            }
        }
    }
}

// Staging configurations (U, W, NS) of the FP64 and mixed products, from a sweep on the 4.1M-block
// C1 system (FP64: 84 us vs 86-110 us for the others tried; mixed: 42 us vs 43-56 us).
constexpr int kU64 = 1, kW64 = 16, kNS64 = 2;
constexpr int kU32 = 2, kW32 = 16, kNS32 = 2;
constexpr int kUfp = 2, kWfp = 16, kNSfp = 2;   // float-pair product (8-byte values, FP32-pipe arithmetic)
// The persistent solver's float-pair product stages one step per group, so that two CTAs fit on an SM
// (the grid then owns two vertices per thread of the C1 system, as in the other forms).
constexpr int kUfpLoop = 1;
// Systems that one CTA per SM holds (up to 2 x 512 rows per SM) take the persistent solver with
// wider groups (FP64: 2 steps, mixed: 4), one CTA per SM: their slices are few per warp, so each
// warp's chain of staged groups (and of direction gathers) sets the product's length, and wider
// groups halve it.  On the sphere-grid system (131,906 rows) the solver's time per Newton
// iteration went 2.89 -> 2.34 ms (FP64) and 1.43 -> 1.29 ms (mixed); the C1 system does not fit.
constexpr int kU64Wide = 2, kNS64Wide = 2;
constexpr int kU32Wide = 4, kNS32Wide = 2;

template <typename VT, typename PT, int U, int W, int NS>
void launch_spmv_tma(const int32_t* rowptr, const int64_t* slice_off, const int32_t* sell_col, const VT* sell_vals,
                     const PT* cg, const double* c, const int32_t* perm, double* q, const uint8_t* fixed, int64_t n,
                     int64_t nsl, double* part, PcgScalars* S, cudaStream_t st) {
    using Lay = StageLayout<VT, U, W, NS>;
    // persistent: as many CTAs as are resident at once (shared memory and registers)
    const int sms = std::max(1, device_facts().sms);
    const int per_sm = std::max(1, std::min(16, kernel_occupancy((const void*)pcg_spmv_tma_kernel<VT, PT, U, W, NS>,
                                                                 W * 32, Lay::kBlockBytes)));
    const int64_t want = (nsl + W - 1) / W;   // at most one CTA per W slices
    const unsigned blocks = (unsigned)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)sms * per_sm);
    // programmatic dependent launch: the CTAs may start (and stage matrix slices) while the previous
    // kernel finishes; the kernel waits for it before reading the direction or the scalars
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(W * 32);
    cfg.dynamicSmemBytes = Lay::kBlockBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr_pdl[1];
    attr_pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr_pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr_pdl;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, pcg_spmv_tma_kernel<VT, PT, U, W, NS>, rowptr, slice_off, sell_col, sell_vals, cg, c, perm,
                       q, fixed, n, nsl, part, S);
}

// Staging variants of the batched product tried by the run-time tuner: (U, W, NS) per precision,
// variant 0 the default of the single-system sweep above.  Every variant forms each row in the
// same order, so they differ in time only.
struct SpmvVariant {
    int U, W, NS;
};
constexpr SpmvVariant kVar64[GIPC_SPMV_VARIANTS] = {{kU64, kW64, kNS64}, {1, 8, 2}, {2, 8, 2}, {1, 8, 3}};
constexpr SpmvVariant kVar32[GIPC_SPMV_VARIANTS] = {{kU32, kW32, kNS32}, {1, 16, 2}, {2, 8, 2}, {4, 8, 2}};

template <typename VT, typename PT>
void launch_spmv_variant(int v, const int32_t* rowptr, const int64_t* slice_off, const int32_t* sell_col,
                         const VT* sell_vals, const PT* cg, const double* c, const int32_t* perm, double* q,
                         const uint8_t* fixed, int64_t n, int64_t nsl, double* part, PcgScalars* S, cudaStream_t st) {
    constexpr bool d = std::is_same<VT, double>::value;
    constexpr const SpmvVariant* T = d ? kVar64 : kVar32;
#define GIPC_SPMV_CASE(i)                                                                                            \
    case i:                                                                                                          \
        launch_spmv_tma<VT, PT, T[i].U, T[i].W, T[i].NS>(rowptr, slice_off, sell_col, sell_vals, cg, c, perm, q, fixed, \
                                                         n, nsl, part, S, st);                                       \
        break;
    switch (v) {
        GIPC_SPMV_CASE(1)
        GIPC_SPMV_CASE(2)
        GIPC_SPMV_CASE(3)
        default: GIPC_SPMV_CASE(0)
    }
#undef GIPC_SPMV_CASE
}

// The tuner's entry for a precision and a size class (created on first use).
int spmv_tune_index(gipc_ctx* ctx, bool f64, int64_t nnzb) {
    int cls = 0;
    while (cls < 62 && (int64_t(2) << cls) <= nnzb) ++cls;
    const int prec = f64 ? GIPC_FP64 : GIPC_MIXED;
    for (size_t i = 0; i < ctx->spmv_tunes.size(); ++i)
        if (ctx->spmv_tunes[i].prec == prec && ctx->spmv_tunes[i].size_class == cls) return (int)i;
    gipc_spmv_tune t;
    t.prec = prec;
    t.size_class = cls;
    ctx->spmv_tunes.push_back(t);
    return (int)ctx->spmv_tunes.size() - 1;
}

// The variant of the next chunk: the chosen one, else the one with the fewest timed iterations.
int spmv_tune_pick(const gipc_spmv_tune& t) {
    if (t.chosen >= 0) return t.chosen;
    int v = 0;
    for (int i = 1; i < GIPC_SPMV_VARIANTS; ++i)
        if (t.cnt[i] < t.cnt[v]) v = i;
    return v;
}

// The context's event pair for timing a chunk (created on first use); false if unavailable.
bool spmv_tune_events(gipc_ctx* ctx) {
    for (auto& e : ctx->spmv_ev)
        if (!e && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
            return false;
        }
    return true;
}

// After the synchronisation that ends a timed chunk of m iterations of variant v: add its time,
// and choose once every variant has GIPC_SPMV_TUNE_SAMPLES timed iterations.
void spmv_tune_add(gipc_ctx* ctx, int tune, int v, int m) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->spmv_ev[0], ctx->spmv_ev[1]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    gipc_spmv_tune& t = ctx->spmv_tunes[tune];
    if (t.chosen >= 0) return;
    t.sum_ms[v] += ms;
    t.cnt[v] += m;
    for (int i = 0; i < GIPC_SPMV_VARIANTS; ++i)
        if (t.cnt[i] < GIPC_SPMV_TUNE_SAMPLES) return;
    int best = 0;
    for (int i = 1; i < GIPC_SPMV_VARIANTS; ++i)
        if (t.sum_ms[i] / t.cnt[i] < t.sum_ms[best] / t.cnt[best]) best = i;
    t.chosen = best;
}

// q = S(H c); alpha = delta_new / (c . q)
template <typename VT, typename PT>
__global__ void __launch_bounds__(kPcgThreads)
// direction: c is a search direction (a curvature c.q <= 0 stops the solve); false for the first
// product H x0, whose x0 is any starting point.
pcg_spmv_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx, const VT* __restrict__ vals,
                const PT* __restrict__ cg, const double* __restrict__ c, const int32_t* __restrict__ perm,
                double* __restrict__ q, const uint8_t* __restrict__ fixed, int64_t n, double* __restrict__ part,
                PcgScalars* __restrict__ S, bool direction) {
    if (S->done) return;
    int64_t row;
    int comp;
    double y = 0.0, d = 0.0;
    if (spmv_lane<VT, PT>(rowptr, colidx, vals, cg, perm, n, row, comp, y)) {
        if (fixed && fixed[row]) y = 0.0;
        q[3 * row + comp] = y;
        d = c[3 * row + comp] * y;
    }
    const double bs = block_sum(d);
    if (publish_partial(part, bs, &S->count_a)) {
        const double pq = sum_partials(part, gridDim.x);
        if (threadIdx.x == 0) {
            S->pq = pq;
            S->alpha = S->delta_new / pq;
            S->count_a = 0;
            if (direction && S->stop_indefinite && pq <= 0.0) {   // no descent along c
                S->status = GIPC_ERR_INDEFINITE;
                S->done = 1;
            }
        }
    }
}

// Block-Jacobi preconditioner as a per-vertex LDL^T factorisation of the diagonal block
// H_ii, stored [6][n] (l10, l20, l21, 1/d0, 1/d1, 1/d2 of vertex v at k * n + v).  Applying it by forward and back
// substitution makes r . P^-1 r a sum of squares y_i^2 / d_i, nonnegative by
// construction even when H_ii is very ill-conditioned (an explicit 3x3 inverse is not
// numerically definite there).  A missing or non-positive-definite block falls back to I.
template <typename VT, typename FT>
__global__ void pcg_factor_kernel(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ colidx,
                                  const VT* __restrict__ vals, int64_t n, FT* __restrict__ fac) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    double m[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    int32_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {  // binary search for the diagonal block
        const int32_t mid = (lo + hi) >> 1;
        const int32_t cm = colidx[mid];
        if (cm == r) {
#pragma unroll
            for (int i = 0; i < 9; ++i) m[i] = (double)vals[9 * (int64_t)mid + i];
            break;
        }
        if (cm < r) lo = mid + 1;
        else hi = mid - 1;
    }
    const double d0 = m[0];
    const double l10 = m[3] / d0, l20 = m[6] / d0;
    const double d1 = m[4] - l10 * l10 * d0;
    const double l21 = (m[7] - l20 * l10 * d0) / d1;
    const double d2 = m[8] - l20 * l20 * d0 - l21 * l21 * d1;
    FT* F = fac + r;
    const FT f[6] = {(FT)l10, (FT)l20, (FT)l21, (FT)(1.0 / d0), (FT)(1.0 / d1), (FT)(1.0 / d2)};
    bool ok = d0 > 0.0 && d1 > 0.0 && d2 > 0.0 && isfinite(l10 + l20 + l21 + d2);
#pragma unroll
    for (int k = 0; k < 6; ++k) ok = ok && isfinite((double)f[k]);   // also catches a float32 overflow
    if (!ok) {
        F[0] = F[n] = F[2 * n] = FT(0);
        F[3 * n] = F[4 * n] = F[5 * n] = FT(1);
        return;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k * n] = f[k];
}

__device__ __forceinline__ void load_factor(const double* __restrict__ fac, int64_t n, int64_t v, double F[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k] = fac[k * n + v];
}

// s = P^-1 r for one vertex; returns r . s = sum_i y_i^2 / d_i (>= 0).
__device__ __forceinline__ double precond_apply(const double* __restrict__ F, const double r[3], double s[3]) {
    const double l10 = F[0], l20 = F[1], l21 = F[2];
    const double y0 = r[0];
    const double y1 = r[1] - l10 * y0;
    const double y2 = r[2] - l20 * y0 - l21 * y1;
    const double z0 = y0 * F[3], z1 = y1 * F[4], z2 = y2 * F[5];
    s[2] = z2;
    s[1] = z1 - l21 * z2;
    s[0] = z0 - l10 * s[1] - l20 * z2;
    return y0 * z0 + y1 * z1 + y2 * z2;
}

// The mixed form keeps the factors in float32 ([6][n] floats) and applies them in float32
// arithmetic: the same substitutions, and r . s again a sum of squares y_i^2 / d_i.
__device__ __forceinline__ void load_factor(const float* __restrict__ fac, int64_t n, int64_t v, float F[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) F[k] = fac[k * n + v];
}

__device__ __forceinline__ float precond_apply(const float* __restrict__ F, const float r[3], float s[3]) {
    const float l10 = F[0], l20 = F[1], l21 = F[2];
    const float y0 = r[0];
    const float y1 = r[1] - l10 * y0;
    const float y2 = r[2] - l20 * y0 - l21 * y1;
    const float z0 = y0 * F[3], z1 = y1 * F[4], z2 = y2 * F[5];
    s[2] = z2;
    s[1] = z1 - l21 * z2;
    s[0] = z0 - l10 * s[1] - l20 * z2;
    return y0 * z0 + y1 * z1 + y2 * z2;
}

// The form's factor type: float32 for the mixed form (MIX), float64 otherwise.
template <bool MIX>
using FacT = typename std::conditional<MIX, float, double>::type;

template <bool MIX>
__device__ __forceinline__ void load_factor_t(const double* __restrict__ fac, int64_t n, int64_t v, FacT<MIX> F[6]) {
    load_factor(reinterpret_cast<const FacT<MIX>*>(fac), n, v, F);
}

// s = P^-1 r in the form's arithmetic: the mixed form rounds r to float32 and gives s in float32;
// r . s is returned in float64 either way.
template <bool MIX>
__device__ __forceinline__ double precond_vertex(const FacT<MIX>* F, const double r[3], FacT<MIX> s[3]) {
    if constexpr (MIX) {
        const float rf[3] = {__double2float_rn(r[0]), __double2float_rn(r[1]), __double2float_rn(r[2])};
        return (double)precond_apply(F, rf, s);
    } else {
        return precond_apply(F, r, s);
    }
}

// x += alpha c; r -= alpha q; s = P^-1 r; delta_new = r . s; beta; termination.
// Persistent CTAs walk tiles of kUpdT vertices.  A tile's 3 kUpdT entries of x, c, r, q and s are
// read and written as flat coalesced runs and handed between the flat (axpy) and the per-vertex
// (preconditioner) layouts through shared memory; the factors are [6][n].  The next tile's 18
// loads per thread are issued before the current tile's FP64 work, so the FP64 pipe and HBM
// overlap.  Each thread sums its vertices (one per tile, tiles in order) into its partial.
// The mixed form (MIX) writes s in float32 over the first half of the s buffer.
template <bool MIX>
__global__ void __launch_bounds__(kUpdT, kUpdPerSm)
pcg_update_kernel(double* __restrict__ x, double* __restrict__ r, const double* __restrict__ c,
                  const double* __restrict__ q, double* __restrict__ s, const double* __restrict__ fac,
                  int64_t n, double* __restrict__ part, PcgScalars* __restrict__ S) {
    using ST = FacT<MIX>;
    if (S->done) return;
    __shared__ double rt[3 * kUpdT];
    __shared__ ST st[3 * kUpdT];
    ST* __restrict__ so = reinterpret_cast<ST*>(s);
    const double alpha = S->alpha;
    const int t = threadIdx.x;
    const int64_t ntiles = (n + kUpdT - 1) / kUpdT, ne = 3 * n;
    double xv[3], cv[3], rv[3], qv[3];
    ST F[6];
    auto load = [&](int64_t tl, double* X, double* C, double* R, double* Q, ST* Fv) {
        const int64_t e0 = 3 * kUpdT * tl + t;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t e = e0 + j * kUpdT;
            if (e < ne) {
                X[j] = x[e];
                C[j] = c[e];
                R[j] = r[e];
                Q[j] = q[e];
            }
        }
        const int64_t v = kUpdT * tl + t;
        if (v < n) load_factor_t<MIX>(fac, n, v, Fv);
    };
    double d = 0.0;
    int64_t tl = blockIdx.x;
    if (tl < ntiles) load(tl, xv, cv, rv, qv, F);
    while (tl < ntiles) {   // uniform across the CTA
        const int64_t tn = tl + gridDim.x;
        double xn[3], cn[3], rn[3], qn[3];
        ST Fn[6];
        if (tn < ntiles) load(tn, xn, cn, rn, qn, Fn);
        const int64_t e0 = 3 * kUpdT * tl + t, v = kUpdT * tl + t;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t e = e0 + j * kUpdT;
            if (e < ne) {
                x[e] = xv[j] + alpha * cv[j];
                const double re = rv[j] - alpha * qv[j];
                r[e] = re;
                rt[t + j * kUpdT] = re;
            }
        }
        __syncthreads();
        if (v < n) {
            const double r3[3] = {rt[3 * t], rt[3 * t + 1], rt[3 * t + 2]};
            ST s3[3];
            d += precond_vertex<MIX>(F, r3, s3);
#pragma unroll
            for (int i = 0; i < 3; ++i) st[3 * t + i] = s3[i];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t e = e0 + j * kUpdT;
            if (e < ne) so[e] = st[t + j * kUpdT];
        }
        if (tn < ntiles) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                xv[j] = xn[j];
                cv[j] = cn[j];
                rv[j] = rn[j];
                qv[j] = qn[j];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) F[k] = Fn[k];
        }
        tl = tn;
    }
    const double bs = block_sum(d);
    if (!publish_partial(part, bs, &S->count_b)) return;
    const double dn = sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
        S->delta_old = S->delta_new;
        S->delta_new = dn;
        S->beta = dn / S->delta_old;
        S->iters += 1;
        if (!isfinite(dn) || !isfinite(S->alpha)) {
            S->status = GIPC_ERR_NONFINITE;
            S->done = 1;
        } else if (!(dn > 0.0) || dn < S->tol * S->delta0 || S->iters >= S->max_iter) {
            S->done = 1;
        }
        S->count_b = 0;
    }
}

// Fused update and direction of one solve (one launch per iteration instead of two).
// Phase 1, per tile this CTA owns: x += alpha c; r -= alpha q; s = P^-1 r and this thread's part
// of r.s, as in pcg_update_kernel, but s and c stay in shared memory.  A grid barrier (the grid
// is launched cooperatively, so every CTA is resident) then lets every CTA sum the partials in
// the same fixed order -- identical totals everywhere -- and form beta and the stopping test;
// phase 2 writes c = S(s + beta c) for the same tiles while the solve continues (the mixed form
// forms it in float32 from the kept float32 s and c and writes it with its float64 image).  CTA 0 records the scalars.  The arithmetic is that of the two separate kernels.
// The barrier wait is bounded: past kBarrierCycles it sets GIPC_ERR_TIMEOUT and stops the solve.
constexpr long long kBarrierCycles = 4000000000LL;   // ~2 s at 2 GHz

__device__ __forceinline__ bool grid_barrier(PcgScalars* S) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &S->bar_gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned prev = atomicAdd(&S->bar_count, 1u);
        ok = 1;
        if (prev == gridDim.x - 1) {
            S->bar_count = 0;
            __threadfence();
            atomicExch(&S->bar_gen, g0 + 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > kBarrierCycles) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

template <bool MIX>
__global__ void __launch_bounds__(kUpdT, kUpdPerSm)
pcg_update_direction_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ c,
                            float* __restrict__ c32, fpair* __restrict__ c2, const double* __restrict__ q,
                            const double* __restrict__ fac,
                            const uint8_t* __restrict__ fixed, int64_t n, double* __restrict__ part,
                            PcgScalars* __restrict__ S) {
    pdl_release();   // the next product may begin staging its matrix slices as SMs free up
    if (S->done) return;
    using ST = FacT<MIX>;
    extern __shared__ double keep[];   // per owned tile: s then c in the form's type, flat order, 3 kUpdT each
    ST* const kp = reinterpret_cast<ST*>(keep);
    __shared__ double rt[3 * kUpdT];
    __shared__ ST st[3 * kUpdT];
    // every scalar this launch reads is read here, before the barrier: CTA 0 rewrites them after it
    const double alpha = S->alpha, delta_old = S->delta_new, tol = S->tol, delta0 = S->delta0;
    const int iters = S->iters + 1, max_iter = S->max_iter;
    const int t = threadIdx.x;
    const int64_t ntiles = (n + kUpdT - 1) / kUpdT, ne = 3 * n;
    double xv[3], cv[3], rv[3], qv[3];
    ST kv[3], F[6];   // kv: the mixed form's float32 direction, kept for phase 2
    auto load = [&](int64_t tl, double* X, double* C, double* R, double* Q, ST* K, ST* Fv) {
        const int64_t e0 = 3 * kUpdT * tl + t;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t e = e0 + j * kUpdT;
            if (e < ne) {
                X[j] = x[e];
                C[j] = c[e];
                R[j] = r[e];
                Q[j] = q[e];
                if constexpr (MIX) K[j] = c32[e];
            }
        }
        const int64_t v = kUpdT * tl + t;
        if (v < n) load_factor_t<MIX>(fac, n, v, Fv);
    };
    double d = 0.0;
    int64_t tl = blockIdx.x;
    int slot = 0;
    if (tl < ntiles) load(tl, xv, cv, rv, qv, kv, F);
    while (tl < ntiles) {
        const int64_t tn = tl + gridDim.x;
        double xn[3], cn[3], rn[3], qn[3];
        ST kn[3], Fn[6];
        if (tn < ntiles) load(tn, xn, cn, rn, qn, kn, Fn);
        ST* ks = kp + (int64_t)slot * 6 * kUpdT;
        const int64_t e0 = 3 * kUpdT * tl + t, v = kUpdT * tl + t;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int64_t e = e0 + j * kUpdT;
            if (e < ne) {
                x[e] = xv[j] + alpha * cv[j];
                const double re = rv[j] - alpha * qv[j];
                r[e] = re;
                rt[t + j * kUpdT] = re;
                if constexpr (MIX) ks[3 * kUpdT + t + j * kUpdT] = kv[j];
                else ks[3 * kUpdT + t + j * kUpdT] = cv[j];
            }
        }
        __syncthreads();
        if (v < n) {
            const double r3[3] = {rt[3 * t], rt[3 * t + 1], rt[3 * t + 2]};
            ST s3[3];
            d += precond_vertex<MIX>(F, r3, s3);
#pragma unroll
            for (int i = 0; i < 3; ++i) st[3 * t + i] = s3[i];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 3; ++j) ks[t + j * kUpdT] = st[t + j * kUpdT];
        if (tn < ntiles) {
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                xv[j] = xn[j];
                cv[j] = cn[j];
                rv[j] = rn[j];
                qv[j] = qn[j];
                if constexpr (MIX) kv[j] = kn[j];
            }
#pragma unroll
            for (int k = 0; k < 6; ++k) F[k] = Fn[k];
        }
        tl = tn;
        ++slot;
    }
    const double bs = block_sum(d);
    if (t == 0) part[blockIdx.x] = bs;
    if (!grid_barrier(S)) {
        if (t == 0) {
            S->status = GIPC_ERR_TIMEOUT;
            S->done = 1;
        }
        return;
    }
    __shared__ double dn_sh;
    const double tot = sum_partials(part, gridDim.x);
    if (t == 0) dn_sh = tot;
    __syncthreads();
    const double dn = dn_sh;
    const double beta = dn / delta_old;
    const float beta_f = (float)beta;
    int status = GIPC_OK, done = 0;
    if (!isfinite(dn) || !isfinite(alpha)) {
        status = GIPC_ERR_NONFINITE;
        done = 1;
    } else if (!(dn > 0.0) || dn < tol * delta0 || iters >= max_iter) {
        done = 1;
    }
    if (!done) {
        slot = 0;
        for (int64_t tl2 = blockIdx.x; tl2 < ntiles; tl2 += gridDim.x, ++slot) {
            const ST* ks = kp + (int64_t)slot * 6 * kUpdT;
            const int64_t e0 = 3 * kUpdT * tl2 + t;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int64_t e = e0 + j * kUpdT;
                if (e < ne) {
                    const bool fx = fixed && fixed[e / 3];
                    if constexpr (MIX) {   // the float32 direction and its exact float64 image
                        const float ce = fx ? 0.0f : __fmaf_rn(beta_f, ks[3 * kUpdT + t + j * kUpdT], ks[t + j * kUpdT]);
                        c32[e] = ce;
                        c[e] = (double)ce;
                    } else {
                        const double ce = fx ? 0.0 : ks[t + j * kUpdT] + beta * ks[3 * kUpdT + t + j * kUpdT];
                        c[e] = ce;
                        if (c2) c2[e] = split_double(ce);
                    }
                }
            }
        }
    }
    if (blockIdx.x == 0 && t == 0) {
        S->delta_old = delta_old;
        S->delta_new = dn;
        S->beta = beta;
        S->iters = iters;
        if (S->status != GIPC_ERR_TIMEOUT) {
            S->status = status;
            S->done = done;
        }
    }
}

// ---- persistent solver: every iteration of one solve in one cooperative launch -------------
// The grid is resident for the whole solve.  An iteration is three phases separated by grid
// barriers:
//   A  q = S(H c) over the warp's SELL-32 slices (the product above) and the CTA's part of c . q;
//   B  alpha = delta / (c . q), every CTA summing all the parts in the same fixed order (so every
//      CTA holds the same alpha); r -= alpha q; s = P^-1 r; the CTA's part of r . s; x += alpha c
//      between the CTA's arrival at the barrier and its wait (no other CTA reads x);
//   C  delta_new, beta and the stopping test, identical in every CTA for the same reason;
//      c = S(s + beta c).
// Each thread owns up to kLoopKeep vertices in phases B and C and keeps their s and c in
// registers between the two.  As soon as a warp's product ends it stages the leading groups of
// its first slice of the next product, so the matrix stream restarts while the barriers and the
// vector phases run.  Every element is computed as in the separate product / update / direction
// kernels; only the summation order of the dot products differs.  The direction changes during
// the launch, so its gathers use coherent loads.  Barrier waits are bounded: one that runs out
// records GIPC_ERR_TIMEOUT, and the other CTAs leave at their next barrier the same way.
constexpr int kLoopW = 16;             // warps per CTA (staging as in the separate product)
constexpr int kLoopT = kLoopW * 32;    // threads per CTA
constexpr int kLoopKeep = 2;           // vertices per thread in the vector phases

// Grid barrier on a monotonic arrival counter (zeroed per solve), in two halves: thread 0 of
// every CTA arrives (its fence makes the writes of the CTA that it has synchronised with visible
// first), and the k-th barrier of a launch completes once k * gridDim.x arrivals are counted.
// Work that no other CTA reads may run between the halves.  The wait is false, in every thread of
// the CTA alike, when it runs out (then GIPC_ERR_TIMEOUT is recorded) or when some CTA has
// recorded a timeout (a CTA that gave up never arrives, so the others see its record while they
// wait).
__device__ __forceinline__ void grid_arrive(unsigned* count) {
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(count, 1u);
    }
}
__device__ __forceinline__ bool grid_wait(unsigned* count, unsigned target, int* status) {
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned* vc = count;
        volatile int* vs = status;
        const long long t0 = clock64();
        while (*vc < target) {
            if (*vs == GIPC_ERR_TIMEOUT) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > kBarrierCycles) {
                ok = 0;
                atomicExch(status, GIPC_ERR_TIMEOUT);
                break;
            }
            __nanosleep(20);
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}
__device__ __forceinline__ bool grid_sync(unsigned* count, unsigned target, int* status) {
    __syncthreads();
    grid_arrive(count);
    return grid_wait(count, target, status);
}

// Pairwise sum of N (a power of two) values: log2 N dependent additions instead of N - 1.
template <int N>
__device__ __forceinline__ double tree_sum(double (&v)[N]) {
#pragma unroll
    for (int h = N / 2; h >= 1; h /= 2)
#pragma unroll
        for (int j = 0; j < h; ++j) v[j] += v[j + h];
    return v[0];
}

// FP64 sums with few FP64 warp-instructions.  On this part the FP64 pipe takes 16 cycles per warp
// instruction whatever its active lanes, and scalar work repeated by every thread of the grid is
// paid 32 warps per SM over: so the CTA sums below leave the shuffle tree to one warp, and the
// solver's scalars (alpha, beta, the stopping test) are formed by one lane and shared.
//
// Sum of the CTA's values (blockDim.x <= kLoopT), in a fixed order: every thread stores its value,
// warp 0 adds them pairwise per lane (lane-strided) and reduces across its lanes.  Valid in warp 0.
__device__ __forceinline__ double cta_sum_lean(double v, double* buf) {
    buf[threadIdx.x] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x < 32) {
        double w[kLoopW];
#pragma unroll
        for (int j = 0; j < kLoopW; ++j) {
            const int i = (int)threadIdx.x + 32 * j;
            w[j] = i < (int)blockDim.x ? buf[i] : 0.0;
        }
        s = tree_sum<kLoopW>(w);
        s = warp_sum(s);
    }
    return s;
}

// Sum of every CTA's part (at most 16 x 32 parts) in a fixed order, by warp 0 with all its loads
// in flight at once.  Valid in warp 0.
__device__ __forceinline__ double grid_sum_lean(const double* part) {
    double s = 0.0;
    if (threadIdx.x < 32) {
        double v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int i = (int)threadIdx.x + 32 * j;
            v[j] = i < (int)gridDim.x ? __ldcg(part + i) : 0.0;
        }
        s = tree_sum<16>(v);
        s = warp_sum(s);
    }
    return s;
}

// Phase stamps of the persistent solver (tracing): thread 0 of every CTA folds the globaltimer at
// boundary k of iteration it into the earliest (trace[(it * 9 + k)]) and the latest
// (trace[kTraceMins + it * 9 + k]) stamp over the CTAs.  No-op when trace is null.
constexpr int kTraceMarks = 9;
constexpr int64_t kTraceMins = (int64_t)GIPC_TRACE_MAX_ITERS * kTraceMarks;
__device__ __forceinline__ void phase_mark(unsigned long long* trace, int it, int k) {
    if (trace && threadIdx.x == 0 && it < GIPC_TRACE_MAX_ITERS) {
        unsigned long long now;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now)::"memory");
        atomicMin(trace + it * kTraceMarks + k, now);
        atomicMax(trace + kTraceMins + it * kTraceMarks + k, now);
    }
}

// CTAs per SM the persistent solver is compiled for: two where two staging areas fit in shared
// memory (the register budget then allows 64 per thread), else one.
template <typename VT, int U, int NS>
constexpr int loop_min_blocks() {
    return 2 * (StageLayout<VT, U, kLoopW, NS>::kBlockBytes + 1024) <= 227 * 1024 ? 2 : 1;
}

template <typename VT, typename PT, int U, int NS, bool MIX>
__global__ void __launch_bounds__(kLoopT, loop_min_blocks<VT, U, NS>())
pcg_loop_kernel(const int32_t* __restrict__ rowptr, const int64_t* __restrict__ slice_off,
                const int32_t* __restrict__ sell_col, const VT* __restrict__ sell_vals, const PT* cg, double* x,
                double* r, double* c, float* c32, fpair* c2, double* q, const double* __restrict__ fac,
                const int32_t* __restrict__ perm, const uint8_t* __restrict__ fixed, int64_t n, int64_t nsl,
                double* part_a, double* part_b, PcgScalars* S, int iters, unsigned long long* trace) {
    using ST = FacT<MIX>;
    using CT = typename std::conditional<MIX, float, double>::type;   // the kept direction
    // The solver's scalars, formed by thread 0 and shared with the CTA (every CTA forms the same
    // values from the same parts): delta = r.s, alpha, beta (and beta in float32), the stopping
    // state, and the constants of the stopping test.
    __shared__ double sh_delta, sh_delta_prev, sh_beta, sh_alpha, sh_pq;
    __shared__ float sh_beta_f;
    __shared__ int sh_stop;   // 0: go on; 1: done after the update; 2: done before it (indefinite)
    __shared__ double red[kLoopT];
    if (S->done) return;   // read before any CTA can change it: uniform
    const int t = threadIdx.x;
    if (t == 0) {
        sh_delta = S->delta_new;
        sh_delta_prev = S->delta_old;
        sh_beta = S->beta;
        sh_alpha = S->alpha;
        sh_pq = S->pq;
        sh_beta_f = (float)S->beta;
        sh_stop = 0;
    }
    const double tol = S->tol, delta0 = S->delta0;   // read by thread 0 only (below)
    const int max_iter = S->max_iter, stop_indefinite = S->stop_indefinite;
    int it_total = S->iters, status = GIPC_OK;
    bool abort = false;
    // the warp's slice of round 0 under the warp-major numbering (see spmv_slices)
    const int64_t first_sl = (int64_t)(t >> 5) * gridDim.x + blockIdx.x;
    __syncthreads();   // the scalars above
    StageRing<VT, U, kLoopW, NS> R;
    R.init();
    R.preissue(first_sl, nsl, slice_off, sell_vals, sell_col);
    unsigned nbar = 0;
    auto sync = [&]() { return grid_sync(&S->bar_count, ++nbar * gridDim.x, &S->status); };
    for (int it = 0; it < iters; ++it) {
        // A: q = S(H c), parts of c . q
        if (trace) __syncthreads();
        phase_mark(trace, it, 0);
        bool timed_out = false;
        const double d = spmv_slices<VT, PT, U, kLoopW, NS, true, true, MIX>(R, rowptr, slice_off, sell_col, sell_vals,
                                                                             cg, c, perm, q, fixed, n, nsl, timed_out);
        if (timed_out) {
            R.drain_all();
            if ((t & 31) == 0) atomicExch(&S->status, GIPC_ERR_TIMEOUT);
        } else {
            R.preissue(first_sl, nsl, slice_off, sell_vals, sell_col);
        }
        {
            const double bs = cta_sum_lean(d, red);
            if (t == 0) part_a[blockIdx.x] = bs;
        }
        phase_mark(trace, it, 1);
        if (!sync()) {
            abort = true;
            break;
        }
        phase_mark(trace, it, 2);
        {
            const double pq = grid_sum_lean(part_a);
            if (t == 0) {
                sh_pq = pq;
                sh_alpha = sh_delta / pq;
                if (stop_indefinite && pq <= 0.0) sh_stop = 2;   // no descent along c: H not positive definite
            }
        }
        __syncthreads();
        phase_mark(trace, it, 3);
        if (sh_stop == 2) {
            status = GIPC_ERR_INDEFINITE;
            break;
        }
        const double alpha = sh_alpha;
        // B: r -= alpha q; s = P^-1 r; parts of r . s; then x += alpha c while the barrier fills
        ST sk[kLoopKeep][3];
        CT ck[kLoopKeep][3];
        double d2 = 0.0;
#pragma unroll
        for (int j = 0; j < kLoopKeep; ++j) {
            const int64_t v = ((int64_t)j * gridDim.x + blockIdx.x) * kLoopT + t;
            if (v < n) {
                double qv[3], rv[3];
                ST F[6];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    qv[e] = q[3 * v + e];
                    rv[e] = r[3 * v + e];
                    if constexpr (MIX) ck[j][e] = c32[3 * v + e];
                    else ck[j][e] = c[3 * v + e];
                }
                load_factor_t<MIX>(fac, n, v, F);
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    rv[e] = rv[e] - alpha * qv[e];
                    r[3 * v + e] = rv[e];
                }
                d2 += precond_vertex<MIX>(F, rv, sk[j]);
            }
        }
        {
            // only the part is read by other CTAs: thread 0 arrives as soon as it is written
            const double bs = cta_sum_lean(d2, red);
            if (t == 0) part_b[blockIdx.x] = bs;
            grid_arrive(&S->bar_count);
        }
        phase_mark(trace, it, 4);
#pragma unroll
        for (int j = 0; j < kLoopKeep; ++j) {   // x is read by its owner only
            const int64_t v = ((int64_t)j * gridDim.x + blockIdx.x) * kLoopT + t;
            if (v < n) {
#pragma unroll
                for (int e = 0; e < 3; ++e) x[3 * v + e] = x[3 * v + e] + alpha * (double)ck[j][e];
            }
        }
        __syncthreads();
        if (!grid_wait(&S->bar_count, ++nbar * gridDim.x, &S->status)) {
            abort = true;
            break;
        }
        phase_mark(trace, it, 5);
        it_total += 1;
        {
            const double dn = grid_sum_lean(part_b);
            if (t == 0) {
                const double beta = dn / sh_delta;
                sh_beta = beta;
                sh_beta_f = (float)beta;
                sh_delta_prev = sh_delta;
                sh_delta = dn;
                if (!isfinite(dn) || !isfinite(sh_alpha)) sh_stop = 3;   // non-finite
                else if (!(dn > 0.0) || dn < tol * delta0 || it_total >= max_iter) sh_stop = 1;
            }
        }
        __syncthreads();
        phase_mark(trace, it, 6);
        if (sh_stop) {
            if (sh_stop == 3) status = GIPC_ERR_NONFINITE;
            break;
        }
        // C: c = S(s + beta c)
        const double beta = sh_beta;
        const float beta_f = sh_beta_f;
#pragma unroll
        for (int j = 0; j < kLoopKeep; ++j) {
            const int64_t v = ((int64_t)j * gridDim.x + blockIdx.x) * kLoopT + t;
            if (v < n) {
                const bool fx = fixed && fixed[v];
#pragma unroll
                for (int e = 0; e < 3; ++e) {
                    if constexpr (MIX) {   // the float32 direction (its float64 image is formed where used)
                        c32[3 * v + e] = fx ? 0.0f : __fmaf_rn(beta_f, ck[j][e], sk[j][e]);
                    } else {
                        const double ce = fx ? 0.0 : sk[j][e] + beta * ck[j][e];
                        c[3 * v + e] = ce;
                        if (c2) c2[3 * v + e] = split_double(ce);
                    }
                }
            }
        }
        if (trace) __syncthreads();
        phase_mark(trace, it, 7);
        if (!sync()) {
            abort = true;
            break;
        }
        phase_mark(trace, it, 8);
    }
    R.drain();   // copies staged for a product that will not run
    __syncthreads();
    if (blockIdx.x == 0 && t == 0) {
        S->delta_old = sh_delta_prev;
        S->delta_new = sh_delta;
        S->beta = sh_beta;
        S->alpha = sh_alpha;
        S->pq = sh_pq;
        S->iters = it_total;
        if (!abort && *(volatile int*)&S->status != GIPC_ERR_TIMEOUT) {
            S->status = status;
            S->done = sh_stop != 0;
        } else {
            S->done = 1;
        }
    }
}

// c = S(s + beta c) over the flat [3n] vectors with kDirEpt coalesced entries per thread.  The
// mixed form (MIX) forms it in float32 from the float32 s and c32 and writes c32 and its exact
// float64 image c.
template <bool MIX>
__global__ void __launch_bounds__(kPcgThreads)
pcg_direction_kernel(double* __restrict__ c, float* __restrict__ c32, fpair* __restrict__ c2,
                     const double* __restrict__ s,
                     const uint8_t* __restrict__ fixed, int64_t n, const PcgScalars* __restrict__ S) {
    using ST = FacT<MIX>;
    // runs after the update of the same iteration; `done` may now be set, but c is still refreshed
    // only while the solve continues
    if (S->done) return;
    const double beta = S->beta;
    const ST* __restrict__ si = reinterpret_cast<const ST*>(s);
    const int64_t ne = 3 * n;
    const int64_t e0 = (int64_t)blockIdx.x * (kPcgThreads * kDirEpt) + threadIdx.x;
    ST sv[kDirEpt], cv[kDirEpt];
    bool fx[kDirEpt];
#pragma unroll
    for (int j = 0; j < kDirEpt; ++j) {
        const int64_t e = e0 + j * kPcgThreads;
        fx[j] = false;
        if (e < ne) {
            sv[j] = si[e];
            if constexpr (MIX) cv[j] = c32[e];
            else cv[j] = c[e];
            fx[j] = fixed && fixed[e / 3];
        }
    }
#pragma unroll
    for (int j = 0; j < kDirEpt; ++j) {
        const int64_t e = e0 + j * kPcgThreads;
        if (e < ne) {
            if constexpr (MIX) {
                const float ce = fx[j] ? 0.0f : __fmaf_rn((float)beta, cv[j], sv[j]);
                c32[e] = ce;
                c[e] = (double)ce;
            } else {
                const double ce = fx[j] ? 0.0 : sv[j] + beta * cv[j];
                c[e] = ce;
                if (c2) c2[e] = split_double(ce);
            }
        }
    }
}

__global__ void soa_to_aos_kernel(const double* __restrict__ in, double* __restrict__ out, float* __restrict__ out32,
                                  int64_t n, const uint8_t* __restrict__ fixed) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n) return;
    const int64_t v = e / 3;
    const int comp = (int)(e - 3 * v);
    const double val = (fixed && fixed[v]) ? 0.0 : in[comp * n + v];
    out[e] = val;
    if (out32) out32[e] = (float)val;
}

__global__ void aos_to_soa_kernel(const double* __restrict__ in, double* __restrict__ out, int64_t n) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * n) return;
    const int64_t v = e / 3;
    const int comp = (int)(e - 3 * v);
    out[comp * n + v] = in[e];
}

// Setup: r = S(b - H x0), s = P^-1 r, c = S(s), delta_0 = r.s (H x0 already in q).  The mixed form
// (MIX) keeps s in float32 over the first half of the s buffer and c32 = S(s), c its float64 image.
template <bool MIX>
__global__ void __launch_bounds__(kPcgThreads)
pcg_init_kernel(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
                double* __restrict__ s, double* __restrict__ c, float* __restrict__ c32, fpair* __restrict__ c2,
                const double* __restrict__ pinv,
                const uint8_t* __restrict__ fixed, int64_t n, double* __restrict__ part, PcgScalars* __restrict__ S) {
    using ST = FacT<MIX>;
    ST* __restrict__ so = reinterpret_cast<ST*>(s);
    double d = 0.0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const bool fx = fixed && fixed[v];
        double rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            rv[i] = fx ? 0.0 : b[3 * v + i] - q[3 * v + i];
            r[3 * v + i] = rv[i];
        }
        ST sv[3], F[6];
        load_factor_t<MIX>(pinv, n, v, F);
        d += precond_vertex<MIX>(F, rv, sv);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            so[3 * v + i] = sv[i];
            const ST ce = fx ? ST(0) : sv[i];
            c[3 * v + i] = (double)ce;
            if constexpr (MIX) c32[3 * v + i] = ce;
            else if (c2) c2[3 * v + i] = split_double(ce);
        }
    }
    const double bs = block_sum(d);
    if (!publish_partial(part, bs, &S->count_0)) return;
    const double d0 = sum_partials(part, gridDim.x);
    if (threadIdx.x == 0) {
        S->delta0 = d0;
        S->delta_new = d0;
        S->iters = 0;
        S->status = GIPC_OK;
        S->done = (!(d0 > 0.0) || !isfinite(d0) || S->max_iter <= 0) ? 1 : 0;
        if (!isfinite(d0)) S->status = GIPC_ERR_NONFINITE;
        S->count_0 = 0;
    }
}

__global__ void pcg_set_scalars(PcgScalars* S, double tol, int max_iter, int stop_indefinite) {
    S->tol = tol;
    S->max_iter = max_iter;
    S->done = 0;
    S->iters = 0;
    S->status = GIPC_OK;
    S->count_a = S->count_b = S->count_0 = 0;
    S->scenes_done = 0;
    S->bar_count = S->bar_gen = 0;
    S->stop_indefinite = stop_indefinite;
}

// ---- batched solves: one CTA per scene for everything but the product ---------------------
// Each scene is an independent system on the vertex range [voff[s], voff[s+1]) (the matrix has
// no blocks across ranges).  The product q = S(H c) runs over all rows at once; everything that
// needs a reduction (c.q, r.s) and the updates run with one CTA per scene, so each scene keeps
// its own alpha, beta, delta and stopping test, in the order of the single-system iteration.

__device__ __forceinline__ double block_sum_all(double v) {   // block sum broadcast to every thread
    __shared__ double total;
    const double t = block_sum(v);
    if (threadIdx.x == 0) total = t;
    __syncthreads();
    const double r = total;
    __syncthreads();
    return r;
}

__device__ __forceinline__ void scene_stop(SceneScalars* SS, PcgScalars* S, int nscenes) {
    SS->done = 1;
    if (atomicAdd(&S->scenes_done, 1u) + 1u == (unsigned)nscenes) S->done = 1;
}

template <bool MIX>
__global__ void __launch_bounds__(kPcgThreads)
pcg_scene_init_kernel(const double* __restrict__ b, const double* __restrict__ q, double* __restrict__ r,
                      double* __restrict__ s, double* __restrict__ c, float* __restrict__ c32,
                      const double* __restrict__ pinv, int64_t ldf, const uint8_t* __restrict__ fixed,
                      const int64_t* __restrict__ voff, int nscenes, SceneScalars* __restrict__ SS,
                      PcgScalars* __restrict__ S) {
    using ST = FacT<MIX>;
    ST* __restrict__ so = reinterpret_cast<ST*>(s);
    const int sc = blockIdx.x;
    const int64_t v0 = voff[sc], v1 = voff[sc + 1];
    double d = 0.0;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const bool fx = fixed && fixed[v];
        double rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            rv[i] = fx ? 0.0 : b[3 * v + i] - q[3 * v + i];
            r[3 * v + i] = rv[i];
        }
        ST sv[3], F[6];
        load_factor_t<MIX>(pinv, ldf, v, F);
        d += precond_vertex<MIX>(F, rv, sv);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            so[3 * v + i] = sv[i];
            const ST ce = fx ? ST(0) : sv[i];
            c[3 * v + i] = (double)ce;
            if constexpr (MIX) c32[3 * v + i] = ce;
        }
    }
    const double d0 = block_sum_all(d);
    if (threadIdx.x == 0) {
        SceneScalars& Z = SS[sc];
        Z.delta0 = Z.delta = d0;
        Z.iters = 0;
        Z.done = 0;
        Z.status = isfinite(d0) ? GIPC_OK : GIPC_ERR_NONFINITE;
        if (!(d0 > 0.0) || !isfinite(d0) || S->max_iter <= 0) scene_stop(&Z, S, nscenes);
    }
}

// alpha = delta / (c.q); x += alpha c; r -= alpha q; s = P^-1 r; delta' = r.s; beta; stop test;
// c = S(s + beta c) while the scene continues.
template <bool MIX>
__global__ void __launch_bounds__(kPcgThreads)
pcg_scene_step_kernel(double* __restrict__ x, double* __restrict__ r, double* __restrict__ c, float* __restrict__ c32,
                      const double* __restrict__ q, double* __restrict__ s, const double* __restrict__ pinv,
                      int64_t ldf, const uint8_t* __restrict__ fixed, const int64_t* __restrict__ voff, int nscenes,
                      SceneScalars* __restrict__ SS, PcgScalars* __restrict__ S) {
    const int sc = blockIdx.x;
    if (SS[sc].done) return;
    const int64_t v0 = voff[sc], v1 = voff[sc + 1];
    double pq = 0.0;
    for (int64_t e = 3 * v0 + threadIdx.x; e < 3 * v1; e += blockDim.x) pq += c[e] * q[e];
    pq = block_sum_all(pq);
    const double delta = SS[sc].delta;
    const double alpha = delta / pq;
    using ST = FacT<MIX>;
    ST* __restrict__ so = reinterpret_cast<ST*>(s);
    double d = 0.0;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        double rv[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            x[3 * v + i] += alpha * c[3 * v + i];
            rv[i] = r[3 * v + i] - alpha * q[3 * v + i];
            r[3 * v + i] = rv[i];
        }
        ST sv[3], F[6];
        load_factor_t<MIX>(pinv, ldf, v, F);
        d += precond_vertex<MIX>(F, rv, sv);
#pragma unroll
        for (int i = 0; i < 3; ++i) so[3 * v + i] = sv[i];
    }
    const double dn = block_sum_all(d);
    __shared__ int stop;
    if (threadIdx.x == 0) {
        SceneScalars& Z = SS[sc];
        Z.delta = dn;
        Z.iters += 1;
        stop = 0;
        if (!isfinite(dn) || !isfinite(alpha)) {
            Z.status = GIPC_ERR_NONFINITE;
            stop = 1;
        } else if (!(dn > 0.0) || dn < S->tol * Z.delta0 || Z.iters >= S->max_iter) {
            stop = 1;
        }
        if (stop) scene_stop(&Z, S, nscenes);
    }
    __syncthreads();
    if (stop) return;
    const double beta = dn / delta;
    for (int64_t v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const bool fx = fixed && fixed[v];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if constexpr (MIX) {   // the float32 direction and its exact float64 image
                const float ce = fx ? 0.0f : __fmaf_rn((float)beta, c32[3 * v + i], so[3 * v + i]);
                c32[3 * v + i] = ce;
                c[3 * v + i] = (double)ce;
            } else {
                const double ce = fx ? 0.0 : so[3 * v + i] + beta * c[3 * v + i];
                c[3 * v + i] = ce;
            }
        }
    }
}

// ---- Persistent batched solver: every iteration of nscenes independent solves in one launch ----
// The batch's rows are spread over the CTAs by vertex (CTA b owns the `chunk` vertices from
// b chunk), whatever the scenes' sizes, so the vector phases are balanced; a scene cut by the
// CTAs' ranges has a segment in each.  Per iteration, between bounded grid barriers:
//   A   q = S(H c) over the SELL-32 slices (the product of the single-system solver);
//   B1  per segment, its part of c . q (segment sums in a fixed order, one warp per segment);
//   B2  per scene still running: alpha = delta / (c . q), the scene's parts summed in a fixed
//       order by every CTA that holds part of it (so they all hold the same alpha); x += alpha c,
//       r -= alpha q, s = P^-1 r, and the segments' parts of r . s;
//   C   beta and the stopping test from the r . s parts, the same way; the scene's first CTA
//       records its scalars; c = S(s + beta c).
// Every element is computed as in the per-scene update kernel; only the summation order of the
// two dots differs.  A CTA holds at most kBMaxSeg segments (the host checks before launching).
constexpr int kBKeep = 3;      // vertices per thread
constexpr int kBMaxSeg = 64;   // scene segments per CTA

// Largest s with voff[s] <= v (the scene holding vertex v; empty scenes are skipped).
__device__ __forceinline__ int scene_of(const int64_t* __restrict__ voff, int nscenes, int64_t v) {
    int lo = 0, hi = nscenes - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The most scene segments any CTA of a batched launch would hold.
__global__ void batch_segments_kernel(const int64_t* __restrict__ voff, int nscenes, int64_t n, int64_t chunk,
                                      int grid, int* __restrict__ most) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= grid) return;
    const int64_t a = (int64_t)b * chunk;
    if (a >= n) return;
    const int64_t e = a + chunk < n ? a + chunk : n;
    atomicMax(most, scene_of(voff, nscenes, e - 1) - scene_of(voff, nscenes, a) + 1);
}

// Sums of val over each segment (one warp per segment, lanes strided, then a fixed tree) into
// out[j]; call with every thread of the CTA after val is complete.
__device__ __forceinline__ void segment_sums(const double* val, const int* seg_lo, int nseg, double* out) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int j = w; j < nseg; j += kLoopW) {
        double t = 0.0;
        for (int li = seg_lo[j] + lane; li < seg_lo[j + 1]; li += 32) t += val[li];
        t = warp_sum(t);
        if (lane == 0) out[j] = t;
    }
}

// Total of scene s over the CTAs holding part of it (part[cta + s], CTAs in order), in warp 0 lane 0
// of the calling warp.
__device__ __forceinline__ double scene_total(const double* part, const int64_t* __restrict__ voff, int s,
                                             int64_t chunk) {
    const int64_t v0 = voff[s], v1 = voff[s + 1];
    const int lane = threadIdx.x & 31;
    double t = 0.0;
    if (v1 > v0) {
        const int64_t c0 = v0 / chunk, c1 = (v1 - 1) / chunk;
        for (int64_t cc = c0 + lane; cc <= c1; cc += 32) t += __ldcg(part + cc + s);
    }
    return warp_sum(t);
}

// First and last scene of the rows of every kPermChunk-row chunk (a slice's rows all lie in one chunk).
__global__ void chunk_scenes_kernel(const int64_t* __restrict__ voff, int nscenes, int64_t n, int64_t nchunks,
                                    int2* __restrict__ out) {
    const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= nchunks) return;
    const int64_t a = w * kPermChunk, e = a + kPermChunk < n ? a + kPermChunk : n;
    out[w] = make_int2(scene_of(voff, nscenes, a), scene_of(voff, nscenes, e - 1));
}

// A slice is multiplied while any scene its chunk touches still iterates.  A scene's flag is set
// only between the last two barriers of an iteration and never cleared, so during the product
// every warp of the grid reads the same flags, and a slice found stopped stays stopped.
struct LiveSlice {
    const int2* chunk_sc;
    const SceneScalars* SS;
    __device__ __forceinline__ bool operator()(int64_t sl) const {
        int alive = 0;
        if ((threadIdx.x & 31) == 0) {
            const int2 w = chunk_sc[sl / (kPermChunk / kSellC)];
            for (int s = w.x; s <= w.y && !alive; ++s) alive = !__ldcg(&SS[s].done);
        }
        return __shfl_sync(0xffffffffu, alive, 0) != 0;
    }
};

template <typename VT, typename PT, int U, int NS, bool MIX>
__global__ void __launch_bounds__(kLoopT, loop_min_blocks<VT, U, NS>())
pcg_batch_loop_kernel(const int32_t* __restrict__ rowptr, const int64_t* __restrict__ slice_off,
                      const int32_t* __restrict__ sell_col, const VT* __restrict__ sell_vals, const PT* cg, double* x,
                      double* r, double* c, float* c32, double* q, double* s_buf, const double* __restrict__ fac,
                      const int32_t* __restrict__ perm, const uint8_t* __restrict__ fixed, int64_t n, int64_t nsl,
                      const int64_t* __restrict__ voff, int nscenes, SceneScalars* SS, PcgScalars* S, double* part_a,
                      double* part_b, int iters, int64_t chunk, const int2* __restrict__ chunk_sc) {
    using ST = FacT<MIX>;
    ST* const so = reinterpret_cast<ST*>(s_buf);
    __shared__ double val[kBKeep * kLoopT];
    __shared__ int seg_lo[kBMaxSeg + 1];
    __shared__ double seg_sum[kBMaxSeg], seg_alpha[kBMaxSeg], seg_beta[kBMaxSeg], seg_delta[kBMaxSeg];
    __shared__ int seg_go[kBMaxSeg], seg_cont[kBMaxSeg], seg_iters[kBMaxSeg];
    if (S->done) return;   // read before any CTA can change it: uniform
    const int t = threadIdx.x, lane = t & 31, wq = t >> 5;
    const int64_t a = (int64_t)blockIdx.x * chunk;
    const int64_t e = a + chunk < n ? a + chunk : n;
    const bool owns = a < n;
    const int s0 = owns ? scene_of(voff, nscenes, a) : 0;
    const int nseg = owns ? scene_of(voff, nscenes, e - 1) - s0 + 1 : 0;
    for (int j = t; j <= nseg; j += kLoopT) {
        const int64_t lo = j < nseg ? voff[s0 + j] : e;
        seg_lo[j] = (int)((lo > a ? lo : a) - a);
    }
    __syncthreads();
    int myseg[kBKeep];
#pragma unroll
    for (int k = 0; k < kBKeep; ++k) {
        const int li = t + k * kLoopT;
        int j = 0;
        while (j + 1 < nseg && seg_lo[j + 1] <= li) ++j;
        myseg[k] = j;
    }
    const double tol = S->tol;
    const int max_iter = S->max_iter;
    const int64_t first_sl = (int64_t)(t >> 5) * gridDim.x + blockIdx.x;
    const LiveSlice live{chunk_sc, SS};
    StageRing<VT, U, kLoopW, NS> R;
    R.init();
    if (first_sl < nsl && live(first_sl)) R.preissue(first_sl, nsl, slice_off, sell_vals, sell_col);
    unsigned nbar = 0;
    auto sync = [&]() { return grid_sync(&S->bar_count, ++nbar * gridDim.x, &S->status); };
    bool abort = false;
    for (int it = 0; it < iters; ++it) {
        // A: q = S(H c) over the slices of the scenes still iterating
        bool timed_out = false;
        spmv_slices<VT, PT, U, kLoopW, NS, true, true, false, LiveSlice>(R, rowptr, slice_off, sell_col, sell_vals, cg,
                                                                          c, perm, q, fixed, n, nsl, timed_out, live);
        if (timed_out) {
            R.drain_all();
            if (lane == 0) atomicExch(&S->status, GIPC_ERR_TIMEOUT);
        } else if (first_sl < nsl && live(first_sl)) {
            R.preissue(first_sl, nsl, slice_off, sell_vals, sell_col);
        }
        for (int j = t; j < nseg; j += kLoopT) seg_go[j] = !__ldcg(&SS[s0 + j].done);
        if (!sync()) {
            abort = true;
            break;
        }
        // B1: the segments' parts of c . q (zero for stopped scenes, whose rows of q are stale)
#pragma unroll
        for (int k = 0; k < kBKeep; ++k) {
            const int li = t + k * kLoopT;
            const int64_t v = a + li;
            if (v < e)
                val[li] = seg_go[myseg[k]]
                              ? (c[3 * v] * q[3 * v] + c[3 * v + 1] * q[3 * v + 1]) + c[3 * v + 2] * q[3 * v + 2]
                              : 0.0;
        }
        __syncthreads();
        segment_sums(val, seg_lo, nseg, seg_sum);
        __syncthreads();
        for (int j = t; j < nseg; j += kLoopT) part_a[blockIdx.x + s0 + j] = seg_sum[j];
        if (!sync()) {
            abort = true;
            break;
        }
        // B2: alpha per scene; x, r, s; the segments' parts of r . s
        for (int j = wq; j < nseg; j += kLoopW) {
            const int sc = s0 + j;
            const double pq = scene_total(part_a, voff, sc, chunk);
            if (lane == 0) {
                const SceneScalars Z = SS[sc];
                seg_go[j] = !Z.done;
                seg_delta[j] = Z.delta;
                seg_iters[j] = Z.iters;
                seg_alpha[j] = Z.delta / pq;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBKeep; ++k) {
            const int li = t + k * kLoopT;
            const int64_t v = a + li;
            if (v >= e) continue;
            double d = 0.0;
            if (seg_go[myseg[k]]) {
                const double alpha = seg_alpha[myseg[k]];
                double rv[3];
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    x[3 * v + i] += alpha * c[3 * v + i];
                    rv[i] = r[3 * v + i] - alpha * q[3 * v + i];
                    r[3 * v + i] = rv[i];
                }
                ST sv[3], F[6];
                load_factor_t<MIX>(fac, n, v, F);
                d = precond_vertex<MIX>(F, rv, sv);
#pragma unroll
                for (int i = 0; i < 3; ++i) so[3 * v + i] = sv[i];
            }
            val[li] = d;
        }
        __syncthreads();
        segment_sums(val, seg_lo, nseg, seg_sum);
        __syncthreads();
        for (int j = t; j < nseg; j += kLoopT) part_b[blockIdx.x + s0 + j] = seg_sum[j];
        if (!sync()) {
            abort = true;
            break;
        }
        // C: beta and the stopping test per scene; the scene's first CTA records them; direction
        for (int j = wq; j < nseg; j += kLoopW) {
            const int sc = s0 + j;
            const double dn = scene_total(part_b, voff, sc, chunk);
            if (lane == 0) {
                int cont = 0;
                if (seg_go[j]) {
                    const int its = seg_iters[j] + 1;
                    const double alpha = seg_alpha[j];
                    SceneScalars& Z = SS[sc];
                    int stop = 0, nonfinite = 0;
                    if (!isfinite(dn) || !isfinite(alpha)) stop = nonfinite = 1;
                    else if (!(dn > 0.0) || dn < tol * Z.delta0 || its >= max_iter) stop = 1;
                    if (voff[sc] / chunk == (int64_t)blockIdx.x) {   // the scene's first CTA
                        Z.delta = dn;
                        Z.iters = its;
                        if (nonfinite) Z.status = GIPC_ERR_NONFINITE;
                        if (stop) scene_stop(&Z, S, nscenes);
                    }
                    cont = !stop;
                    seg_beta[j] = dn / seg_delta[j];
                }
                seg_cont[j] = cont;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kBKeep; ++k) {
            const int li = t + k * kLoopT;
            const int64_t v = a + li;
            if (v >= e || !seg_cont[myseg[k]]) continue;
            const double beta = seg_beta[myseg[k]];
            const bool fx = fixed && fixed[v];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                if constexpr (MIX) {   // the float32 direction and its exact float64 image
                    const float ce = fx ? 0.0f : __fmaf_rn((float)beta, c32[3 * v + i], so[3 * v + i]);
                    c32[3 * v + i] = ce;
                    c[3 * v + i] = (double)ce;
                } else {
                    const double ce = fx ? 0.0 : so[3 * v + i] + beta * c[3 * v + i];
                    c[3 * v + i] = ce;
                }
            }
        }
        if (!sync()) {
            abort = true;
            break;
        }
        if (*(volatile int*)&S->done) break;   // every scene has stopped (read by all after the barrier)
    }
    R.drain();
    (void)abort;
}

inline unsigned spmv_blocks(int64_t n) {
    const int64_t warps = (n + kRowsPerWarp - 1) / kRowsPerWarp;
    return (unsigned)((warps * 32 + kPcgThreads - 1) / kPcgThreads);
}

inline unsigned upd_blocks(int64_t n) { return grid_for(n, kUpdT, kUpdPerSm); }

inline unsigned dir_blocks(int64_t n) {
    const int64_t per = (int64_t)kPcgThreads * kDirEpt;
    return (unsigned)(n > 0 ? (3 * n + per - 1) / per : 1);
}

// Launch shape of the fused update / direction kernel, or ok = false when it does not apply (the
// owned tiles would not fit in shared memory, or the grid would not be resident all at once).
struct FusePlan {
    bool ok = false;
    unsigned grid = 0;
    size_t smem = 0;
};

template <bool MIX>
inline FusePlan plan_fused(int64_t n) {
    FusePlan p;
    const DeviceFacts df = device_facts();
    if (df.sms <= 0 || !df.coop) return p;
    const int64_t ntiles = (n + kUpdT - 1) / kUpdT;
    if (ntiles < 1) return p;
    const int64_t grid = std::min<int64_t>(ntiles, (int64_t)df.sms * kUpdPerSm);
    const int64_t tpc = (ntiles + grid - 1) / grid;
    if (tpc > kFuseMaxTiles) return p;
    const size_t smem = (size_t)tpc * 6 * kUpdT * sizeof(double);
    // the limit is raised once to the largest tile count, so every smaller launch fits under it
    if (kernel_occupancy((const void*)pcg_update_direction_kernel<MIX>, kUpdT,
                         kFuseMaxTiles * 6 * kUpdT * sizeof(double)) <= 0)
        return p;
    const int per_sm = kernel_occupancy((const void*)pcg_update_direction_kernel<MIX>, kUpdT, smem);
    if ((int64_t)per_sm * df.sms < grid) return p;
    p.ok = true;
    p.grid = (unsigned)grid;
    p.smem = smem;
    return p;
}

// Launch shape of the persistent solver, or ok = false when it does not apply (no cooperative
// launch, or more vertices than the co-resident grid owns at kLoopKeep per thread).  The grid is
// no larger than the product and the vector phases need, so small systems also synchronise
// fewer CTAs.
struct LoopPlan {
    bool ok = false;
    unsigned grid = 0;
    size_t smem = 0;
};

template <typename VT, typename PT, int U, int NS, bool MIX>
inline LoopPlan plan_loop(int64_t n, int64_t nsl) {
    LoopPlan p;
    const DeviceFacts df = device_facts();
    if (df.sms <= 0 || !df.coop || n <= 0) return p;
    const size_t smem = StageLayout<VT, U, kLoopW, NS>::kBlockBytes;
    const int per_sm = kernel_occupancy((const void*)pcg_loop_kernel<VT, PT, U, NS, MIX>, kLoopT, smem);
    if (per_sm <= 0) return p;
    const int64_t cap = (int64_t)df.sms * per_sm;
    const int64_t want = std::max<int64_t>((nsl + kLoopW - 1) / kLoopW, (n + (int64_t)kLoopKeep * kLoopT - 1) / ((int64_t)kLoopKeep * kLoopT));
    const int64_t grid = std::max<int64_t>(1, std::min(cap, want));
    if (grid * kLoopKeep * kLoopT < n) return p;
    p.ok = true;
    p.grid = (unsigned)grid;
    p.smem = smem;
    return p;
}

struct BatchPlan {
    bool ok = false;
    unsigned grid = 0;
    size_t smem = 0;
    int64_t chunk = 0;
};

template <typename VT, typename PT, int U, int NS, bool MIX>
inline BatchPlan plan_batch(int64_t n, int64_t nsl) {
    BatchPlan p;
    const DeviceFacts df = device_facts();
    if (df.sms <= 0 || !df.coop || n <= 0) return p;
    const size_t smem = StageLayout<VT, U, kLoopW, NS>::kBlockBytes;
    const int per_sm = kernel_occupancy((const void*)pcg_batch_loop_kernel<VT, PT, U, NS, MIX>, kLoopT, smem);
    if (per_sm <= 0) return p;
    const int64_t cap = (int64_t)df.sms * per_sm, per_cta = (int64_t)kBKeep * kLoopT;
    const int64_t want = std::max<int64_t>((nsl + kLoopW - 1) / kLoopW, (n + per_cta - 1) / per_cta);
    const int64_t grid = std::max<int64_t>(1, std::min(cap, want));
    const int64_t chunk = (n + grid - 1) / grid;
    if (chunk > per_cta) return p;
    p.ok = true;
    p.grid = (unsigned)grid;
    p.smem = smem;
    p.chunk = chunk;
    return p;
}

inline unsigned vec_blocks(int64_t n) { return grid_for(n, (int64_t)kPcgThreads * kVpt, 8); }

}  // namespace
}  // namespace gipc

namespace gipc {
// One solve, or (voff != NULL) nscenes independent solves on the vertex ranges voff (device,
// [nscenes+1]) with per-scene scalars; scene_iters_h / scene_status_h (host, [nscenes]) report
// each scene's iterations and status.  voff_h (optional): the same ranges in host memory, so the
// batched launch is planned without reading them back.
gipc_status pcg_impl(gipc_ctx* ctx, const gipc_bsr* A, const double* rhs, double* x, const uint8_t* fixed,
                     const gipc_pcg_params* prm, int* iters_out_h, double* rel_out_h, cudaStream_t st,
                     const int64_t* voff, int nscenes, int* scene_iters_h, int* scene_status_h,
                     const int64_t* voff_h) {
    if (!ctx || !A || !prm) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: null context, matrix or parameters");
    const int64_t n = A->n;
    if (n < 0 || A->nnzb < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: negative sizes");
    if (A->prec != GIPC_FP64 && A->prec != GIPC_MIXED) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: bad precision");
    if (!(prm->rel_tol >= 0.0) || prm->max_iter < 0 || prm->check_every < 0)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: need rel_tol >= 0, max_iter >= 0, check_every >= 0");
    if (prm->product != GIPC_PRODUCT_NATIVE && prm->product != GIPC_PRODUCT_FLOAT_PAIR)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: unknown product arithmetic %d", prm->product);
    if (n == 0) {
        if (iters_out_h) *iters_out_h = 0;
        if (rel_out_h) *rel_out_h = 0.0;
        return GIPC_OK;
    }
    if (!rhs || !x || !A->rowptr || (A->nnzb > 0 && (!A->colidx || !A->vals)))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg: null vector or matrix pointer");
    gipc_status s;
    const int64_t nvec = 3 * n;
    const unsigned vb = vec_blocks(n), sb = spmv_blocks(n), ub = upd_blocks(n), db = dir_blocks(n);
    const bool f64 = A->prec == GIPC_FP64;
    const bool fp = f64 && !voff && prm->product == GIPC_PRODUCT_FLOAT_PAIR;
    const int64_t nsl = (n + kSellC - 1) / kSellC;
    // one persistent launch for all iterations of a single system where the grid holds it
    LoopPlan loop;
    bool wide = false;   // the one-CTA-per-SM persistent solver (kU64Wide / kU32Wide)
    if (!voff) {
        if (fp) {
            loop = plan_loop<fpair, fpair, kUfpLoop, kNSfp, false>(n, nsl);
        } else if (f64) {
            loop = plan_loop<double, double, kU64Wide, kNS64Wide, false>(n, nsl);
            wide = loop.ok;
            if (!wide) loop = plan_loop<double, double, kU64, kNS64, false>(n, nsl);
        } else {
            loop = plan_loop<float, float, kU32Wide, kNS32Wide, true>(n, nsl);
            wide = loop.ok;
            if (!wide) loop = plan_loop<float, float, kU32, kNS32, true>(n, nsl);
        }
    }
    const FusePlan fuse = (voff || loop.ok) ? FusePlan{} : (f64 ? plan_fused<false>(n) : plan_fused<true>(n));
    const unsigned maxb = std::max(std::max(std::max(sb, vb), ub), std::max(fuse.grid, 2 * loop.grid));
    if ((s = ctx->slot[P_VEC].reserve(sizeof(double) * 6 * nvec)) != GIPC_OK) return s;
    if ((s = ctx->slot[P_PINV].reserve(sizeof(double) * 6 * n)) != GIPC_OK) return s;
    if ((s = ctx->slot[P_PART].reserve(sizeof(double) * (maxb + 8) + sizeof(PcgScalars) + 64)) != GIPC_OK) return s;
    double* V = ctx->slot[P_VEC].as<double>();
    double *b = V, *xv = V + nvec, *r = V + 2 * nvec, *sv = V + 3 * nvec, *c = V + 4 * nvec, *q = V + 5 * nvec;
    double* pinv = ctx->slot[P_PINV].as<double>();
    PcgScalars* S = reinterpret_cast<PcgScalars*>(ctx->slot[P_PART].as<char>());
    double* part = reinterpret_cast<double*>(ctx->slot[P_PART].as<char>() + ((sizeof(PcgScalars) + 63) / 64) * 64);

    const unsigned eb = (unsigned)((nvec + 255) / 256);
    const int max_iter = prm->max_iter;
    // row order by length within 1024-row chunks (stable, deterministic)
    const int64_t chunks = (n + kPermChunk - 1) / kPermChunk;
    const int64_t ncnt = (int64_t)kLenBuckets * chunks;
    if ((s = ctx->slot[P_PERM].reserve(sizeof(int32_t) * (n + ncnt) + sizeof(int64_t) * (ncnt + 1 + scan_scratch_words(ncnt)) + 64)) != GIPC_OK) return s;
    int32_t* perm = ctx->slot[P_PERM].as<int32_t>();
    int32_t* counts = perm + n;
    int64_t* offs = reinterpret_cast<int64_t*>(ctx->slot[P_PERM].as<char>() + ((sizeof(int32_t) * (n + ncnt) + 15) / 16) * 16);
    int64_t* scan_tmp = offs + ncnt + 1;
    float* c32 = nullptr;
    fpair* c2 = nullptr;   // float-pair copy of the direction (float-pair product)
    if (!f64) {
        if ((s = ctx->slot[P_VEC32].reserve(sizeof(float) * 2 * nvec)) != GIPC_OK) return s;
    } else if (fp) {
        if ((s = ctx->slot[P_VEC32].reserve(sizeof(fpair) * nvec)) != GIPC_OK) return s;
        c2 = ctx->slot[P_VEC32].as<fpair>();
    }
    float* x32 = f64 ? nullptr : ctx->slot[P_VEC32].as<float>();
    if (!f64) c32 = x32 + nvec;
    perm_hist_kernel<<<(unsigned)chunks, 256, 0, st>>>(A->rowptr, n, counts, chunks);
    if (exclusive_scan<int32_t>(counts, offs, ncnt, scan_tmp, st) != cudaSuccess) return check_launch("gipc_pcg: scan");
    perm_scatter_kernel<<<(unsigned)chunks, 32, 0, st>>>(A->rowptr, n, offs, chunks, perm);
    // sliced layout: slice lengths, their offsets, then the copy
    if ((s = ctx->slot[P_SLICE].reserve(sizeof(int32_t) * (nsl + 1) + sizeof(int64_t) * (nsl + 2 + scan_scratch_words(nsl)) + 64)) != GIPC_OK) return s;
    int32_t* slice_len = ctx->slot[P_SLICE].as<int32_t>();
    int64_t* slice_off = reinterpret_cast<int64_t*>(ctx->slot[P_SLICE].as<char>() + ((sizeof(int32_t) * (nsl + 1) + 15) / 16) * 16);
    int64_t* slice_scan = slice_off + nsl + 2;
    sell_len_kernel<<<(unsigned)((nsl + 255) / 256), 256, 0, st>>>(A->rowptr, perm, n, nsl, slice_len);
    if (exclusive_scan<int32_t>(slice_len, slice_off, nsl, slice_scan, st) != cudaSuccess) return check_launch("gipc_pcg: scan");
    int64_t steps = 0;
    cudaMemcpyAsync(&steps, slice_off + nsl, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg: slice sync");
    const size_t vsz = f64 ? sizeof(double) : sizeof(float);
    const int64_t cells = steps * kSellC;
    if ((s = ctx->slot[P_SELL].reserve(sizeof(int32_t) * cells + 256 + vsz * 9 * cells)) != GIPC_OK) return s;
    int32_t* sell_col = ctx->slot[P_SELL].as<int32_t>();
    void* sell_vals = ctx->slot[P_SELL].as<char>() + ((sizeof(int32_t) * cells + 255) / 256) * 256;
    const unsigned fb = (unsigned)((nsl * kSellC + 255) / 256);
    if (fp) sell_fill_kernel<double, fpair><<<fb, 256, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, perm, n, nsl, slice_off, sell_col, (fpair*)sell_vals);
    else if (f64) sell_fill_kernel<double, double><<<fb, 256, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, perm, n, nsl, slice_off, sell_col, (double*)sell_vals);
    else sell_fill_kernel<float, float><<<fb, 256, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, perm, n, nsl, slice_off, sell_col, (float*)sell_vals);
    pcg_set_scalars<<<1, 1, 0, st>>>(S, prm->rel_tol, max_iter,
                                     (!voff && (prm->flags & GIPC_PCG_STOP_ON_INDEFINITE)) ? 1 : 0);
    soa_to_aos_kernel<<<eb, 256, 0, st>>>(rhs, b, nullptr, n, fixed);
    soa_to_aos_kernel<<<eb, 256, 0, st>>>(x, xv, x32, n, fixed);
    if (f64) pcg_factor_kernel<double, double><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, n, pinv);
    else pcg_factor_kernel<float, float><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, n, reinterpret_cast<float*>(pinv));
    // q = S(H x0), reusing the spmv kernel with a scratch dot (alpha is overwritten at iteration 1)
    if (f64) pcg_spmv_kernel<double, double><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, xv, xv, perm, q, fixed, n, part, S, false);
    else pcg_spmv_kernel<float, float><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, x32, xv, perm, q, fixed, n, part, S, false);
    SceneScalars* SS = nullptr;
    if (voff) {
        if ((s = ctx->slot[P_SCENE].reserve(sizeof(SceneScalars) * (nscenes + 1))) != GIPC_OK) return s;
        SS = ctx->slot[P_SCENE].as<SceneScalars>();
        if (f64) pcg_scene_init_kernel<false><<<nscenes, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, pinv, n, fixed, voff, nscenes, SS, S);
        else pcg_scene_init_kernel<true><<<nscenes, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, pinv, n, fixed, voff, nscenes, SS, S);
    } else {
        if (f64) pcg_init_kernel<false><<<vb, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, c2, pinv, fixed, n, part, S);
        else pcg_init_kernel<true><<<vb, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, c2, pinv, fixed, n, part, S);
    }
    if ((s = check_launch("gipc_pcg: setup")) != GIPC_OK) return s;

    PcgScalars hs{};
    int launched = 0;
    if (loop.ok && max_iter > 0) {
        // every iteration in one cooperative launch; the stopping test runs on the device
        double* part_b = part + loop.grid;
        int64_t n_arg = n, nsl_arg = nsl;
        int iters_arg = max_iter;
        const uint8_t* fixed_arg = fixed;
        const int32_t* rp = A->rowptr;
        const void* fn;
        const void* cg;
        if (fp) {
            fn = (const void*)pcg_loop_kernel<fpair, fpair, kUfpLoop, kNSfp, false>;
            cg = c2;
        } else if (f64) {
            fn = wide ? (const void*)pcg_loop_kernel<double, double, kU64Wide, kNS64Wide, false>
                      : (const void*)pcg_loop_kernel<double, double, kU64, kNS64, false>;
            cg = c;
        } else {
            fn = wide ? (const void*)pcg_loop_kernel<float, float, kU32Wide, kNS32Wide, true>
                      : (const void*)pcg_loop_kernel<float, float, kU32, kNS32, true>;
            cg = c32;
        }
        unsigned long long* trace = nullptr;
        if (ctx->solver_trace) {   // earliest stamps start at the largest value, latest at zero
            const size_t half = sizeof(unsigned long long) * (size_t)kTraceMins;
            if ((s = ctx->slot[P_TRACE].reserve(2 * half)) != GIPC_OK) return s;
            trace = ctx->slot[P_TRACE].as<unsigned long long>();
            if (cudaMemsetAsync(trace, 0xff, half, st) != cudaSuccess ||
                cudaMemsetAsync(trace + kTraceMins, 0, half, st) != cudaSuccess)
                return check_launch("gipc_pcg: trace reset");
        }
        void* args[] = {&rp, &slice_off, &sell_col, &sell_vals, &cg, &xv, &r, &c, &c32, &c2, &q, &pinv, &perm,
                        &fixed_arg, &n_arg, &nsl_arg, &part, &part_b, &S, &iters_arg, &trace};
        ctx->prof.start(GIPC_PROF_PCG_LOOP, st);
        if (cudaLaunchCooperativeKernel(fn, dim3(loop.grid), dim3(kLoopT), args, loop.smem, st) != cudaSuccess)
            return check_launch("gipc_pcg: persistent solver");
        ctx->prof.stop(GIPC_PROF_PCG_LOOP, st);
        if ((s = check_launch("gipc_pcg: persistent solver")) != GIPC_OK) return s;
        launched = max_iter;
    }
    if (voff && !fp && max_iter > 0 && ctx->batch_loop) {
        // every iteration of the batch in one cooperative launch, where the grid holds it and no CTA
        // would cut more than kBMaxSeg scenes
        const BatchPlan bp = f64 ? plan_batch<double, double, kU64, kNS64, false>(n, nsl)
                                 : plan_batch<float, float, kU32, kNS32, true>(n, nsl);
        if (bp.ok) {
            const int64_t nchunks = (n + kPermChunk - 1) / kPermChunk;
            if ((s = ctx->slot[P_BATCH].reserve(sizeof(double) * 2 * ((size_t)bp.grid + nscenes + 1) + 16 +
                                                sizeof(int2) * (size_t)nchunks)) != GIPC_OK)
                return s;
            double* part_a = ctx->slot[P_BATCH].as<double>();
            double* part_b = part_a + bp.grid + nscenes + 1;
            int* most = reinterpret_cast<int*>(part_b + bp.grid + nscenes + 1);
            int2* chunk_sc = reinterpret_cast<int2*>(most + 4);
            chunk_scenes_kernel<<<(unsigned)((nchunks + 255) / 256), 256, 0, st>>>(voff, nscenes, n, nchunks, chunk_sc);
            int most_h = 0;
            if (voff_h) {   // the most scene segments a CTA would hold, from the host copy of the ranges
                auto scene_of_h = [&](int64_t v) {   // as scene_of
                    int lo = 0, hi = nscenes - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (voff_h[mid] <= v) lo = mid;
                        else hi = mid - 1;
                    }
                    return lo;
                };
                for (int64_t b = 0; b < (int64_t)bp.grid && b * bp.chunk < n; ++b) {
                    const int64_t a = b * bp.chunk, e = std::min<int64_t>(a + bp.chunk, n);
                    most_h = std::max(most_h, scene_of_h(e - 1) - scene_of_h(a) + 1);
                }
            } else {
                cudaMemsetAsync(most, 0, sizeof(int), st);
                batch_segments_kernel<<<(bp.grid + 255) / 256, 256, 0, st>>>(voff, nscenes, n, bp.chunk, (int)bp.grid,
                                                                             most);
                cudaMemcpyAsync(&most_h, most, sizeof(int), cudaMemcpyDeviceToHost, st);
                if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg: batch plan");
            }
            if (most_h <= kBMaxSeg) {
                int64_t n_arg = n, nsl_arg = nsl, chunk_arg = bp.chunk;
                int ns_arg = nscenes, iters_arg = max_iter;
                const uint8_t* fixed_arg = fixed;
                const int32_t* rp = A->rowptr;
                const void* fn = f64 ? (const void*)pcg_batch_loop_kernel<double, double, kU64, kNS64, false>
                                     : (const void*)pcg_batch_loop_kernel<float, float, kU32, kNS32, true>;
                const void* cg = f64 ? (const void*)c : (const void*)c32;
                void* args[] = {&rp, &slice_off, &sell_col, &sell_vals, &cg, &xv, &r, &c, &c32, &q, &sv, &pinv, &perm,
                                &fixed_arg, &n_arg, &nsl_arg, &voff, &ns_arg, &SS, &S, &part_a, &part_b, &iters_arg,
                                &chunk_arg, &chunk_sc};
                ctx->prof.start(GIPC_PROF_PCG_LOOP, st);
                if (cudaLaunchCooperativeKernel(fn, dim3(bp.grid), dim3(kLoopT), args, bp.smem, st) != cudaSuccess)
                    return check_launch("gipc_pcg: persistent batch solver");
                ctx->prof.stop(GIPC_PROF_PCG_LOOP, st);
                if ((s = check_launch("gipc_pcg: persistent batch solver")) != GIPC_OK) return s;
                launched = max_iter;
            }
        }
    }
    const int chunk = prm->check_every > 0 ? prm->check_every : (prm->rel_tol > 0.0 ? 16 : max_iter + 1);
    // batched systems: the product's staging variant is chosen at run time (the scenes' dots are
    // summed by the scene kernel, so the variant changes no result); single systems keep variant 0
    // Variants are timed over whole chunks of iterations (product and scene step, with the overlap
    // of consecutive launches), and only chunks after which the solve still runs count.
    const int tune = (voff && !fp && ctx->spmv_autotune && launched < max_iter) ? spmv_tune_index(ctx, f64, A->nnzb) : -1;
    while (launched < max_iter) {
        const int m = (max_iter - launched) < chunk ? (max_iter - launched) : chunk;
        const int var = tune >= 0 ? spmv_tune_pick(ctx->spmv_tunes[tune]) : 0;
        const bool timed = tune >= 0 && ctx->spmv_tunes[tune].chosen < 0 && launched + m < max_iter &&
                           spmv_tune_events(ctx) && cudaEventRecord(ctx->spmv_ev[0], st) == cudaSuccess;
        for (int it = 0; it < m; ++it) {
            ctx->prof.start(GIPC_PROF_PCG_SPMV, st);
            if (fp)
                launch_spmv_tma<fpair, fpair, kUfp, kWfp, kNSfp>(A->rowptr, slice_off, sell_col, (const fpair*)sell_vals,
                                                                 c2, c, perm, q, fixed, n, nsl, part, S, st);
            else if (f64)
                launch_spmv_variant<double, double>(var, A->rowptr, slice_off, sell_col, (const double*)sell_vals, c, c,
                                                    perm, q, fixed, n, nsl, part, S, st);
            else
                launch_spmv_variant<float, float>(var, A->rowptr, slice_off, sell_col, (const float*)sell_vals, c32, c,
                                                  perm, q, fixed, n, nsl, part, S, st);
            ctx->prof.stop(GIPC_PROF_PCG_SPMV, st);
            if (voff) {
                ctx->prof.start(GIPC_PROF_PCG_UPDATE, st);
                if (f64)
                    pcg_scene_step_kernel<false><<<nscenes, kPcgThreads, 0, st>>>(xv, r, c, c32, q, sv, pinv, n, fixed,
                                                                                  voff, nscenes, SS, S);
                else
                    pcg_scene_step_kernel<true><<<nscenes, kPcgThreads, 0, st>>>(xv, r, c, c32, q, sv, pinv, n, fixed,
                                                                                 voff, nscenes, SS, S);
                ctx->prof.stop(GIPC_PROF_PCG_UPDATE, st);
                continue;
            }
            ctx->prof.start(GIPC_PROF_PCG_UPDATE, st);
            if (fuse.ok) {
                int64_t n_arg = n;
                const uint8_t* fixed_arg = fixed;
                void* args[] = {&xv, &r, &c, &c32, &c2, &q, &pinv, &fixed_arg, &n_arg, &part, &S};
                const void* fused_fn = f64 ? (const void*)pcg_update_direction_kernel<false>
                                           : (const void*)pcg_update_direction_kernel<true>;
                if (cudaLaunchCooperativeKernel(fused_fn, dim3(fuse.grid), dim3(kUpdT), args,
                                                fuse.smem, st) != cudaSuccess)
                    return check_launch("gipc_pcg: fused update");
                ctx->prof.stop(GIPC_PROF_PCG_UPDATE, st);
                continue;
            }
            if (f64) pcg_update_kernel<false><<<ub, kUpdT, 0, st>>>(xv, r, c, q, sv, pinv, n, part, S);
            else pcg_update_kernel<true><<<ub, kUpdT, 0, st>>>(xv, r, c, q, sv, pinv, n, part, S);
            ctx->prof.stop(GIPC_PROF_PCG_UPDATE, st);
            ctx->prof.start(GIPC_PROF_PCG_DIRECTION, st);
            if (f64) pcg_direction_kernel<false><<<db, kPcgThreads, 0, st>>>(c, c32, c2, sv, fixed, n, S);
            else pcg_direction_kernel<true><<<db, kPcgThreads, 0, st>>>(c, c32, c2, sv, fixed, n, S);
            ctx->prof.stop(GIPC_PROF_PCG_DIRECTION, st);
        }
        launched += m;
        if (timed) cudaEventRecord(ctx->spmv_ev[1], st);
        if ((s = check_launch("gipc_pcg: iteration")) != GIPC_OK) return s;
        if (launched < max_iter) {
            cudaMemcpyAsync(&hs, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg: sync");
            if (timed && !hs.done) spmv_tune_add(ctx, tune, var, m);
            if (hs.done) break;
        }
    }
    aos_to_soa_kernel<<<eb, 256, 0, st>>>(xv, x, n);
    cudaMemcpyAsync(&hs, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st);
    if (voff) {
        std::vector<SceneScalars> hz((size_t)nscenes);
        cudaMemcpyAsync(hz.data(), SS, sizeof(SceneScalars) * nscenes, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg: final sync");
        if (hs.status == GIPC_ERR_TIMEOUT)
            return fail(GIPC_ERR_TIMEOUT, "gipc_pcg: a grid barrier of the persistent batch solver timed out");
        int most = 0;
        bool nonfinite = false, short_of_tol = false;
        for (int k = 0; k < nscenes; ++k) {
            if (scene_iters_h) scene_iters_h[k] = hz[k].iters;
            most = std::max(most, hz[k].iters);
            const bool nf = hz[k].status == GIPC_ERR_NONFINITE;
            const bool nc = prm->rel_tol > 0.0 && hz[k].delta0 > 0.0 && hz[k].delta >= prm->rel_tol * hz[k].delta0 &&
                            hz[k].delta > 0.0;
            if (scene_status_h) scene_status_h[k] = nf ? GIPC_ERR_NONFINITE : (nc ? GIPC_ERR_NOT_CONVERGED : GIPC_OK);
            nonfinite |= nf;
            short_of_tol |= nc;
        }
        if (iters_out_h) *iters_out_h = most;
        if (rel_out_h) *rel_out_h = 0.0;
        if (nonfinite) return fail(GIPC_ERR_NONFINITE, "gipc_pcg: non-finite residual in a scene");
        if (short_of_tol) return fail(GIPC_ERR_NOT_CONVERGED, "gipc_pcg: a scene did not reach the tolerance");
        return GIPC_OK;
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg: final sync");
    if (iters_out_h) *iters_out_h = hs.iters;
    if (rel_out_h) *rel_out_h = hs.delta0 > 0.0 ? hs.delta_new / hs.delta0 : 0.0;
    if (loop.ok && ctx->solver_trace) ctx->solver_trace_iters = hs.iters;
    if (hs.status == GIPC_ERR_NONFINITE) return fail(GIPC_ERR_NONFINITE, "gipc_pcg: non-finite residual");
    if (hs.status == GIPC_ERR_INDEFINITE)
        return fail(GIPC_ERR_INDEFINITE, "gipc_pcg: c . H c <= 0 after %d iterations (H not positive definite)", hs.iters);
    if (prm->rel_tol > 0.0 && hs.delta0 > 0.0 && hs.delta_new >= prm->rel_tol * hs.delta0 && hs.delta_new > 0.0)
        return fail(GIPC_ERR_NOT_CONVERGED, "gipc_pcg: %d iterations without reaching the tolerance", hs.iters);
    return GIPC_OK;
}
}  // namespace gipc

extern "C" gipc_status gipc_pcg(gipc_ctx* ctx, const gipc_bsr* A, const double* rhs, double* x,
                                const uint8_t* fixed, const gipc_pcg_params* prm, int* iters_out_h,
                                double* rel_out_h, void* stream) {
    return gipc::pcg_impl(ctx, A, rhs, x, fixed, prm, iters_out_h, rel_out_h, (cudaStream_t)stream, nullptr, 1, nullptr,
                          nullptr, nullptr);
}

extern "C" gipc_status gipc_pcg_batch_persistent(gipc_ctx* ctx, int enable) {
    using namespace gipc;
    if (!ctx) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_batch_persistent: null context");
    ctx->batch_loop = enable != 0;
    return GIPC_OK;
}

extern "C" gipc_status gipc_spmv_autotune(gipc_ctx* ctx, int enable) {
    using namespace gipc;
    if (!ctx) return fail(GIPC_ERR_INVALID_ARG, "gipc_spmv_autotune: null context");
    ctx->spmv_autotune = enable != 0;
    return GIPC_OK;
}

extern "C" gipc_status gipc_spmv_tunings(gipc_ctx* ctx, gipc_spmv_tuning* out_h, int cap, int* count_h) {
    using namespace gipc;
    if (!ctx || !count_h || (cap > 0 && !out_h)) return fail(GIPC_ERR_INVALID_ARG, "gipc_spmv_tunings: null argument");
    const int m = std::min(cap, (int)ctx->spmv_tunes.size());
    for (int k = 0; k < m; ++k) {
        const gipc_spmv_tune& t = ctx->spmv_tunes[k];
        const SpmvVariant* V = t.prec == GIPC_FP64 ? kVar64 : kVar32;
        gipc_spmv_tuning& o = out_h[k];
        o.precision = t.prec;
        o.size_class = t.size_class;
        o.chosen = t.chosen;
        for (int i = 0; i < GIPC_SPMV_VARIANTS; ++i) {
            o.U[i] = V[i].U;
            o.W[i] = V[i].W;
            o.NS[i] = V[i].NS;
            o.samples[i] = t.cnt[i];
            o.mean_us[i] = t.cnt[i] > 0 ? 1e3 * t.sum_ms[i] / t.cnt[i] : 0.0;
        }
    }
    *count_h = (int)ctx->spmv_tunes.size();
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_solver_trace(gipc_ctx* ctx, int enable) {
    if (!ctx) return gipc::fail(GIPC_ERR_INVALID_ARG, "gipc_profile_solver_trace: null context");
    ctx->solver_trace = enable != 0;
    ctx->solver_trace_iters = 0;
    return GIPC_OK;
}

extern "C" gipc_status gipc_profile_solver_phases(gipc_ctx* ctx, double* phase_us_h, int* iters_h) {
    using namespace gipc;
    if (!ctx || !phase_us_h) return fail(GIPC_ERR_INVALID_ARG, "gipc_profile_solver_phases: null argument");
    const int iters = std::min(ctx->solver_trace_iters, (int)GIPC_TRACE_MAX_ITERS);
    if (iters < 4 || !ctx->slot[P_TRACE].ptr)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_profile_solver_phases: no traced solve of four or more iterations");
    std::vector<unsigned long long> h(2 * (size_t)kTraceMins);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(h.data(), ctx->slot[P_TRACE].ptr, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost) !=
            cudaSuccess)
        return check_launch("gipc_profile_solver_phases");
    auto mn = [&](int it, int k) { return (double)h[(size_t)it * kTraceMarks + k]; };
    auto mx = [&](int it, int k) { return (double)h[(size_t)kTraceMins + (size_t)it * kTraceMarks + k]; };
    // phase p runs from boundary a (first CTA, or last CTA for a barrier) to boundary b (last CTA, or
    // first CTA for a barrier); iterations 2 .. iters-2 (each has a successor)
    std::vector<double> v;
    for (int p = 0; p < GIPC_PHASE_COUNT; ++p) {
        v.clear();
        for (int it = 2; it < iters - 1; ++it) {
            double len;
            switch (p) {
                case GIPC_PHASE_PRODUCT: len = mx(it, 1) - mn(it, 0); break;
                case GIPC_PHASE_BARRIER_A: len = mn(it, 2) - mx(it, 1); break;
                case GIPC_PHASE_TOTAL_A: len = mx(it, 3) - mn(it, 2); break;
                case GIPC_PHASE_VECTOR: len = mx(it, 4) - mn(it, 3); break;
                case GIPC_PHASE_BARRIER_B: len = mn(it, 5) - mx(it, 4); break;
                case GIPC_PHASE_TOTAL_B: len = mx(it, 6) - mn(it, 5); break;
                case GIPC_PHASE_DIRECTION: len = mx(it, 7) - mn(it, 6); break;
                case GIPC_PHASE_BARRIER_C: len = mn(it, 8) - mx(it, 7); break;
                default: len = mn(it + 1, 0) - mn(it, 0); break;
            }
            v.push_back(len * 1e-3);   // ns -> us
        }
        std::sort(v.begin(), v.end());
        const size_t m = v.size();
        phase_us_h[p] = m % 2 ? v[m / 2] : 0.5 * (v[m / 2 - 1] + v[m / 2]);
    }
    if (iters_h) *iters_h = iters - 3;
    return GIPC_OK;
}

// ------------------------------------------------------------------------------------------
// Allocation-free variant of the solver (gipc_pcg_noalloc).
//
// Some callers may not allocate device memory: a host framework that owns every byte of
// device memory through its own pool and forbids cudaMalloc, or a latency-critical loop in
// which a cudaMalloc / cudaFree (which can synchronise the device) would stall work queued on
// other streams.  This variant runs the same algorithm as gipc_pcg with the row-ordered product
// over the BSR arrays (no sliced copy of the matrix, no fused or persistent kernels), and its
// working vectors live in one fixed-size array in device global memory defined below, so it
// needs neither a context nor any allocation.  The caller still passes the matrix, right-hand
// side and solution buffers.
#include <mutex>

namespace gipc {
namespace {

constexpr int64_t kNoAllocMaxN = GIPC_PCG_NOALLOC_MAX_N;
constexpr size_t na_align(size_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t kNaChunks = (kNoAllocMaxN + kPermChunk - 1) / kPermChunk;
constexpr int64_t kNaCounts = (int64_t)kLenBuckets * kNaChunks;
// The partials hold one value per CTA of the largest grid that writes them for n <= kNoAllocMaxN:
// the row-ordered product, the update and the vector (setup) kernels.  The two grid-capped ones
// (update, vector) never exceed their uncapped size, which is what is counted here.
constexpr int64_t na_div_up(int64_t a, int64_t b) { return (a + b - 1) / b; }
constexpr int64_t kNaSpmvBlocks = na_div_up(na_div_up(kNoAllocMaxN, kRowsPerWarp) * 32, kPcgThreads);
constexpr int64_t kNaUpdBlocks = na_div_up(kNoAllocMaxN, kUpdT);
constexpr int64_t kNaVecBlocks = na_div_up(kNoAllocMaxN, (int64_t)kPcgThreads * kVpt);
constexpr int kNaMaxBlocks = (int)std::max(std::max(kNaSpmvBlocks, kNaUpdBlocks), kNaVecBlocks);
// region sizes (bytes), each 256-byte aligned
constexpr size_t kNaVec = na_align(sizeof(double) * 18 * kNoAllocMaxN);        // b, x, r, s, c, q
constexpr size_t kNaFac = na_align(sizeof(double) * 6 * kNoAllocMaxN);         // LDL^T factors
constexpr size_t kNaVec32 = na_align(sizeof(float) * 6 * kNoAllocMaxN);        // float32 x0 and c
constexpr size_t kNaPerm = na_align(sizeof(int32_t) * (kNoAllocMaxN + kNaCounts));
constexpr size_t kNaOffs = na_align(sizeof(int64_t) * (kNaCounts + 1 + 64));   // offsets + scan scratch
constexpr size_t kNaPart = na_align(256 + sizeof(double) * kNaMaxBlocks);      // scalars + partials
constexpr size_t kNoAllocBytes = kNaVec + kNaFac + kNaVec32 + kNaPerm + kNaOffs + kNaPart;
static_assert(kNaCounts <= kScanTile, "row-length histogram must fit one scan tile");
static_assert(sizeof(PcgScalars) <= 256, "solver scalars must fit their slot");

}  // namespace
}  // namespace gipc

// The fixed scratch: every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char g_pcg_noalloc_scratch[gipc::kNoAllocBytes];

namespace gipc {
namespace {

std::mutex g_na_mutex;
constexpr int kNaMaxDevices = 256;
void* g_na_addr[kNaMaxDevices] = {};

// Device address of the fixed scratch on the current device.  In host code the array's name
// is only a host-side stand-in, so the address comes from cudaGetSymbolAddress, once per
// device, with that device current.
gipc_status noalloc_scratch(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices)
        return fail(GIPC_ERR_CUDA, "gipc_pcg_noalloc: no usable current device");
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_pcg_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(GIPC_ERR_CUDA, "gipc_pcg_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        g_na_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_na_addr[dev]);
    return GIPC_OK;
}

}  // namespace
}  // namespace gipc

extern "C" gipc_status gipc_pcg_noalloc(const gipc_bsr* A, const double* rhs, double* x, const uint8_t* fixed,
                                        const gipc_pcg_params* prm, int* iters_out_h, double* rel_out_h,
                                        void* stream) {
    using namespace gipc;
    cudaStream_t st = (cudaStream_t)stream;
    if (!A || !prm) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: null matrix or parameters");
    const int64_t n = A->n;
    if (n < 0 || A->nnzb < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: negative sizes");
    if (n > kNoAllocMaxN)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: n = %lld exceeds the fixed scratch limit of %lld vertices",
                    (long long)n, (long long)kNoAllocMaxN);
    if (A->prec != GIPC_FP64 && A->prec != GIPC_MIXED)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: bad precision");
    if (!(prm->rel_tol >= 0.0) || prm->max_iter < 0 || prm->check_every < 0)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: need rel_tol >= 0, max_iter >= 0, check_every >= 0");
    // (the float-pair product is accepted and runs as the native one here)
    if (prm->product != GIPC_PRODUCT_NATIVE && prm->product != GIPC_PRODUCT_FLOAT_PAIR)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: unknown product arithmetic %d", prm->product);
    if (n == 0) {
        if (iters_out_h) *iters_out_h = 0;
        if (rel_out_h) *rel_out_h = 0.0;
        return GIPC_OK;
    }
    if (!rhs || !x || !A->rowptr || (A->nnzb > 0 && (!A->colidx || !A->vals)))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: null vector or matrix pointer");
    unsigned char* base = nullptr;
    gipc_status s = noalloc_scratch(&base);
    if (s != GIPC_OK) return s;

    const int64_t nvec = 3 * n;
    const unsigned vb = vec_blocks(n), sb = spmv_blocks(n), ub = upd_blocks(n), db = dir_blocks(n);
    if (std::max(std::max(vb, sb), ub) > (unsigned)kNaMaxBlocks)   // cannot happen for n <= kNoAllocMaxN
        return fail(GIPC_ERR_INVALID_ARG, "gipc_pcg_noalloc: grid exceeds the fixed partials");
    double* V = reinterpret_cast<double*>(base);
    double *b = V, *xv = V + nvec, *r = V + 2 * nvec, *sv = V + 3 * nvec, *c = V + 4 * nvec, *q = V + 5 * nvec;
    double* pinv = reinterpret_cast<double*>(base + kNaVec);
    const bool f64 = A->prec == GIPC_FP64;
    float* x32 = f64 ? nullptr : reinterpret_cast<float*>(base + kNaVec + kNaFac);
    float* c32 = f64 ? nullptr : x32 + nvec;
    int32_t* perm = reinterpret_cast<int32_t*>(base + kNaVec + kNaFac + kNaVec32);
    const int64_t chunks = (n + kPermChunk - 1) / kPermChunk;
    const int64_t ncnt = (int64_t)kLenBuckets * chunks;
    int32_t* counts = perm + n;
    int64_t* offs = reinterpret_cast<int64_t*>(base + kNaVec + kNaFac + kNaVec32 + kNaPerm);
    int64_t* scan_tmp = offs + ncnt + 1;
    unsigned char* pbase = base + kNaVec + kNaFac + kNaVec32 + kNaPerm + kNaOffs;
    PcgScalars* S = reinterpret_cast<PcgScalars*>(pbase);
    double* part = reinterpret_cast<double*>(pbase + 256);

    const unsigned eb = (unsigned)((nvec + 255) / 256);
    const int max_iter = prm->max_iter;
    perm_hist_kernel<<<(unsigned)chunks, 256, 0, st>>>(A->rowptr, n, counts, chunks);
    if (exclusive_scan<int32_t>(counts, offs, ncnt, scan_tmp, st) != cudaSuccess)
        return check_launch("gipc_pcg_noalloc: scan");
    perm_scatter_kernel<<<(unsigned)chunks, 32, 0, st>>>(A->rowptr, n, offs, chunks, perm);
    // the solver scalars (iteration count, done flag, reduction counters) start from zero on
    // every call: pcg_set_scalars clears them; all other scratch is written before it is read
    pcg_set_scalars<<<1, 1, 0, st>>>(S, prm->rel_tol, max_iter, (prm->flags & GIPC_PCG_STOP_ON_INDEFINITE) ? 1 : 0);
    soa_to_aos_kernel<<<eb, 256, 0, st>>>(rhs, b, nullptr, n, fixed);
    soa_to_aos_kernel<<<eb, 256, 0, st>>>(x, xv, x32, n, fixed);
    if (f64) pcg_factor_kernel<double, double><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, n, pinv);
    else pcg_factor_kernel<float, float><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, n, reinterpret_cast<float*>(pinv));
    if (f64) pcg_spmv_kernel<double, double><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, xv, xv, perm, q, fixed, n, part, S, false);
    else pcg_spmv_kernel<float, float><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, x32, xv, perm, q, fixed, n, part, S, false);
    if (f64) pcg_init_kernel<false><<<vb, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, nullptr, pinv, fixed, n, part, S);
    else pcg_init_kernel<true><<<vb, kPcgThreads, 0, st>>>(b, q, r, sv, c, c32, nullptr, pinv, fixed, n, part, S);
    if ((s = check_launch("gipc_pcg_noalloc: setup")) != GIPC_OK) return s;

    const int chunk = prm->check_every > 0 ? prm->check_every : (prm->rel_tol > 0.0 ? 16 : max_iter + 1);
    PcgScalars hs{};
    int launched = 0;
    while (launched < max_iter) {
        const int m = (max_iter - launched) < chunk ? (max_iter - launched) : chunk;
        for (int it = 0; it < m; ++it) {
            if (f64) pcg_spmv_kernel<double, double><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const double*)A->vals, c, c, perm, q, fixed, n, part, S, true);
            else pcg_spmv_kernel<float, float><<<sb, kPcgThreads, 0, st>>>(A->rowptr, A->colidx, (const float*)A->vals, c32, c, perm, q, fixed, n, part, S, true);
            if (f64) {
                pcg_update_kernel<false><<<ub, kUpdT, 0, st>>>(xv, r, c, q, sv, pinv, n, part, S);
                pcg_direction_kernel<false><<<db, kPcgThreads, 0, st>>>(c, c32, nullptr, sv, fixed, n, S);
            } else {
                pcg_update_kernel<true><<<ub, kUpdT, 0, st>>>(xv, r, c, q, sv, pinv, n, part, S);
                pcg_direction_kernel<true><<<db, kPcgThreads, 0, st>>>(c, c32, nullptr, sv, fixed, n, S);
            }
        }
        launched += m;
        if ((s = check_launch("gipc_pcg_noalloc: iteration")) != GIPC_OK) return s;
        if (launched < max_iter) {
            cudaMemcpyAsync(&hs, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg_noalloc: sync");
            if (hs.done) break;
        }
    }
    aos_to_soa_kernel<<<eb, 256, 0, st>>>(xv, x, n);
    cudaMemcpyAsync(&hs, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_pcg_noalloc: final sync");
    if (iters_out_h) *iters_out_h = hs.iters;
    if (rel_out_h) *rel_out_h = hs.delta0 > 0.0 ? hs.delta_new / hs.delta0 : 0.0;
    if (hs.status == GIPC_ERR_NONFINITE) return fail(GIPC_ERR_NONFINITE, "gipc_pcg_noalloc: non-finite residual");
    if (hs.status == GIPC_ERR_INDEFINITE)
        return fail(GIPC_ERR_INDEFINITE, "gipc_pcg_noalloc: c . H c <= 0 after %d iterations (H not positive definite)",
                    hs.iters);
    if (prm->rel_tol > 0.0 && hs.delta0 > 0.0 && hs.delta_new >= prm->rel_tol * hs.delta0 && hs.delta_new > 0.0)
        return fail(GIPC_ERR_NOT_CONVERGED, "gipc_pcg_noalloc: %d iterations without reaching the tolerance", hs.iters);
    return GIPC_OK;
}
