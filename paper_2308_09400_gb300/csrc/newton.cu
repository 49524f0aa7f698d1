// One implicit time step by projected Newton with CCD-filtered backtracking line search
// (Alg. 1 on the incremental potential of Sec. 3.1, Eq. 1-2).
//
// The host drives the loop; every arithmetic step runs in the library's kernels: contact
// detection and CCD (contact.cu), tetrahedron and stencil evaluation, BSR assembly, the
// modified PCG, and the small vector kernels and deterministic reductions below.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "context.cuh"

namespace gipc {

gipc_status find_contacts_impl(gipc_ctx* ctx, const double* x, const double* rest_x, int64_t n, const gipc_surface& srf,
                               double dhat, int32_t* stencils, double* eps_x, int64_t cap, int64_t* count,
                               bool compact, const int32_t* vscene, int64_t* npt_out, cudaStream_t st, int nscenes,
                               bool cached);
gipc_status ccd_impl(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const gipc_surface& srf, double slack,
                     double* alpha_h, cudaStream_t st, const int32_t* vscene, int nscenes, double* amin_dev,
                     bool cached);
gipc_status stencil_type_order(const int32_t* stencils, int64_t k, int32_t* order, unsigned* counts, cudaStream_t s);
gipc_status eval_tets_live(const double* x, int64_t n, const int32_t* tets, int64_t T, const double* Dm_inv,
                           const double* vol, const gipc_elastic_params* prm, int prec, int hess_mode, double* energy,
                           double* grad, void* hess, const int32_t* vscene, const int32_t* live, cudaStream_t stream);
gipc_status eval_stencils_ordered(const double* x, int64_t n, const int32_t* stencils, int64_t k,
                                  const double* eps_x, const gipc_barrier_params* prm, int prec, int mode,
                                  double* energy, double* grad, void* hess, double* lam, uint8_t* flags,
                                  const int32_t* order, cudaStream_t s);
gipc_status pcg_impl(gipc_ctx* ctx, const gipc_bsr* A, const double* rhs, double* x, const uint8_t* fixed,
                     const gipc_pcg_params* prm, int* iters_out_h, double* rel_out_h, cudaStream_t st,
                     const int64_t* voff, int nscenes, int* scene_iters_h, int* scene_status_h,
                     const int64_t* voff_h);

namespace {

enum NewtonSlot { N_VEC = 20, N_ST0 = 21, N_ST1 = 22, N_SEVAL = 23, N_TEVAL = 24, N_ENER = 25, N_ROW = 26,
                  N_COL = 27, N_VAL = 28, N_RED = 29 };
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 512;   // partial sums per reduction (fixed: results do not depend on the device)

inline unsigned nb(int64_t w, int t) { return (unsigned)std::max<int64_t>(1, (w + t - 1) / t); }

// xt = x0 + dt v0 + dt^2 g on free vertices, x0 on fixed ones
__global__ void inertia_target_kernel(const double* __restrict__ x0, const double* __restrict__ v0,
                                      const uint8_t* __restrict__ fixed, int64_t n, double dt, double dt2g0,
                                      double dt2g1, double dt2g2, double* __restrict__ xt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool fx = fixed && fixed[i];
    const double g[3] = {dt2g0, dt2g1, dt2g2};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double p = x0[q * n + i];
        xt[q * n + i] = fx ? p : __dadd_rn(__dadd_rn(p, __dmul_rn(dt, v0[q * n + i])), g[q]);
    }
}

// gbase = m (x - xt);  rhs is set to zero for the solver's initial guess elsewhere
__global__ void grad_base_kernel(const double* __restrict__ x, const double* __restrict__ xt,
                                 const double* __restrict__ m, int64_t n, double* __restrict__ gb) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    gb[j] = __dmul_rn(m[j % n], __dsub_rn(x[j], xt[j]));
}

__global__ void negate_kernel(const double* __restrict__ a, int64_t m, double* __restrict__ b) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) b[j] = -a[j];
}

// x = xp + alpha d
__global__ void axpy_kernel(const double* __restrict__ xp, const double* __restrict__ d, double alpha, int64_t m,
                            double* __restrict__ x) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) x[j] = __dadd_rn(xp[j], __dmul_rn(alpha, d[j]));
}

// v = (x - x0) / dt
__global__ void velocity_kernel(const double* __restrict__ x, const double* __restrict__ x0, double dt, int64_t m,
                                double* __restrict__ v) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) v[j] = __ddiv_rn(__dsub_rn(x[j], x0[j]), dt);
}

__device__ __forceinline__ double block_reduce(double v, bool is_max) {
    __shared__ double sh[kRedThreads / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? fmax(v, u) : __dadd_rn(v, u);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < kRedThreads / 32 ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double u = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_max ? fmax(v, u) : __dadd_rn(v, u);
        }
    }
    return v;
}

// term kinds of the reductions
enum RedKind { R_ARRAY = 0, R_INERTIA = 1, R_MAXABS = 2 };

// Partial sums over fixed chunks: block b reduces [b*chunk, (b+1)*chunk) in a fixed pattern.
__global__ void __launch_bounds__(kRedThreads)
partial_reduce_kernel(int kind, const double* __restrict__ a, const double* __restrict__ b,
                      const double* __restrict__ m, int64_t n, int64_t count, int64_t chunk,
                      double* __restrict__ partial) {
    const int64_t lo = (int64_t)blockIdx.x * chunk;
    const int64_t hi = std::min(count, lo + chunk);
    double acc = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kRedThreads) {
        double t;
        if (kind == R_ARRAY) {
            t = a[i];
            acc = __dadd_rn(acc, t);
        } else if (kind == R_INERTIA) {
            const double dx = __dsub_rn(a[i], b[i]), dy = __dsub_rn(a[n + i], b[n + i]),
                         dz = __dsub_rn(a[2 * n + i], b[2 * n + i]);
            t = __dmul_rn(m[i], __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
            acc = __dadd_rn(acc, t);
        } else {
            acc = fmax(acc, fabs(a[i]));
        }
    }
    acc = block_reduce(acc, kind == R_MAXABS);
    if (threadIdx.x == 0) partial[blockIdx.x] = acc;
}

__global__ void __launch_bounds__(kRedThreads)
final_reduce_kernel(const double* __restrict__ partial, int np, bool is_max, double* __restrict__ out) {
    double acc = 0.0;
    for (int i = threadIdx.x; i < np; i += kRedThreads) acc = is_max ? fmax(acc, partial[i]) : __dadd_rn(acc, partial[i]);
    acc = block_reduce(acc, is_max);
    if (threadIdx.x == 0) *out = acc;
}

// Enqueue a reduction of `count` terms into *out (device).
void reduce(int kind, const double* a, const double* b, const double* m, int64_t n, int64_t count, double* partial,
            double* out, cudaStream_t st) {
    if (count <= 0) {
        cudaMemsetAsync(out, 0, sizeof(double), st);
        return;
    }
    const int64_t chunk = std::max<int64_t>(kRedThreads, (count + kRedBlocks - 1) / kRedBlocks);
    const int np = (int)((count + chunk - 1) / chunk);
    partial_reduce_kernel<<<np, kRedThreads, 0, st>>>(kind, a, b, m, n, count, chunk, partial);
    final_reduce_kernel<<<1, kRedThreads, 0, st>>>(partial, np, kind == R_MAXABS, out);
}

struct ContactSet {
    int slot;
    int64_t cap = 0, k = 0;
    int32_t* st = nullptr;
    double* eps = nullptr;
    int32_t* order = nullptr;   // the stencils grouped by type (stencil_type_order), for their evaluation
    unsigned* tcnt = nullptr;   // its 16 counters
};

// The contact set's storage in its slot: eps [cap], stencils [4][cap], the type order [cap] and its
// counters.  contact_storage grows it to `cap` stencils; contact_view takes what the slot holds.
constexpr size_t kContactBytes = 5 * sizeof(int32_t) + sizeof(double), kContactExtra = 16 * sizeof(unsigned) + 16;
void contact_pointers(gipc_ctx* ctx, ContactSet& cs, int64_t cap) {
    cs.cap = cap;
    cs.eps = ctx->slot[cs.slot].as<double>();
    cs.st = reinterpret_cast<int32_t*>(cs.eps + cap);
    cs.order = cs.st + 4 * cap;
    cs.tcnt = reinterpret_cast<unsigned*>(cs.order + cap);
}
gipc_status contact_storage(gipc_ctx* ctx, ContactSet& cs, int64_t cap) {
    const gipc_status r = ctx->slot[cs.slot].reserve((size_t)cap * kContactBytes + kContactExtra);
    if (r != GIPC_OK) return r;
    contact_pointers(ctx, cs, cap);
    return GIPC_OK;
}
void contact_view(gipc_ctx* ctx, ContactSet& cs) {
    const size_t b = ctx->slot[cs.slot].bytes;
    contact_pointers(ctx, cs, b > kContactExtra ? (int64_t)((b - kContactExtra) / kContactBytes) : 0);
}

struct Step {
    gipc_ctx* ctx;
    const gipc_scene& sc;
    const gipc_step_params& prm;
    cudaStream_t st;
    int64_t n;
    double *x0, *xt, *xp, *d, *g, *rhs, *gb;
    double *partial, *res;
    ContactSet set[2];

    Step(gipc_ctx* c, const gipc_scene& s, const gipc_step_params& p, cudaStream_t q)
        : ctx(c), sc(s), prm(p), st(q), n(s.n) {
        set[0].slot = N_ST0;
        set[1].slot = N_ST1;
    }

    gipc_status contacts(const double* x, ContactSet& cs) {
        for (int attempt = 0; attempt < 2; ++attempt) {
            int64_t cnt = 0;
            const gipc_status s = find_contacts_impl(ctx, x, sc.rest_x, n, sc.surface, prm.barrier.dhat, cs.st, cs.eps,
                                                     cs.cap, &cnt, true, nullptr, nullptr, st, 1, true);
            if (s == GIPC_OK) {
                cs.k = cnt;
                return stencil_type_order(cs.st, cs.k, cs.order, cs.tcnt, st);
            }
            if (s != GIPC_ERR_CAPACITY) return s;
            const gipc_status r = contact_storage(ctx, cs, cnt + cnt / 4 + 1024);
            if (r != GIPC_OK) return r;
        }
        return fail(GIPC_ERR_CUDA, "gipc_newton_step: contact count changed between passes");
    }

    // I(x) and the contacts at x
    gipc_status potential(const double* x, ContactSet& cs, double* I) {
        gipc_status s;
        if ((s = contacts(x, cs)) != GIPC_OK) return s;
        const int64_t T = sc.T, k = cs.k;
        gipc_prof_span span(ctx->prof, GIPC_PROF_ENERGY, st);
        if ((s = ctx->slot[N_ENER].reserve(sizeof(double) * (T + k + 2))) != GIPC_OK) return s;
        double* te = ctx->slot[N_ENER].as<double>();
        double* se = te + T;
        gipc_elastic_params ep = prm.elastic;
        ep.scale = prm.dt * prm.dt;
        if ((s = gipc_eval_tets(x, n, sc.tets, T, sc.Dm_inv, sc.vol, &ep, GIPC_FP64, GIPC_HESS_DENSE, te, nullptr, nullptr, st)) != GIPC_OK)
            return s;
        if (k > 0 && (s = eval_stencils_ordered(x, n, cs.st, k, cs.eps, &prm.barrier, GIPC_FP64, GIPC_HESS_DENSE, se, nullptr,
                                                nullptr, nullptr, nullptr, cs.order, st)) != GIPC_OK)
            return s;
        reduce(R_INERTIA, x, xt, sc.mass, n, n, partial, res + 0, st);
        reduce(R_ARRAY, te, nullptr, nullptr, 0, T, partial + kRedBlocks, res + 1, st);
        reduce(R_ARRAY, se, nullptr, nullptr, 0, k, partial + 2 * kRedBlocks, res + 2, st);
        double h[3];
        cudaMemcpyAsync(h, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step: energy");
        *I = (0.5 * h[0] + h[1]) + h[2];
        if (!std::isfinite(*I)) return fail(GIPC_ERR_NONFINITE, "gipc_newton_step: non-finite energy");
        return GIPC_OK;
    }

    gipc_status run(double* x, double* v, gipc_step_stats* stats) {
        const int64_t m3 = 3 * n;
        gipc_status s;
        // the broad-phase candidates are reused only within this step (the caller may change the
        // scene between steps)
        ctx->ccache.valid = false;
        if ((s = ctx->slot[N_VEC].reserve(sizeof(double) * 7 * m3)) != GIPC_OK) return s;
        if ((s = ctx->slot[N_RED].reserve(sizeof(double) * (4 * kRedBlocks + 8))) != GIPC_OK) return s;
        x0 = ctx->slot[N_VEC].as<double>();
        xt = x0 + m3;
        xp = xt + m3;
        d = xp + m3;
        g = d + m3;
        rhs = g + m3;
        gb = rhs + m3;
        partial = ctx->slot[N_RED].as<double>();
        res = partial + 4 * kRedBlocks;
        for (auto& cs : set) contact_view(ctx, cs);
        const double dt = prm.dt;
        cudaMemcpyAsync(x0, x, sizeof(double) * m3, cudaMemcpyDeviceToDevice, st);
        inertia_target_kernel<<<nb(n, 256), 256, 0, st>>>(x0, v, sc.fixed, n, dt, (dt * dt) * prm.gravity[0],
                                                           (dt * dt) * prm.gravity[1], (dt * dt) * prm.gravity[2], xt);
        int cur = 0;
        double I_prev = 0.0;
        if ((s = potential(x, set[cur], &I_prev)) != GIPC_OK) return s;
        gipc_step_stats S{};
        const int T = (int)sc.T;
        const bool mixed = prm.prec == GIPC_MIXED;
        const size_t hb = mixed ? sizeof(float) : sizeof(double);
        for (int it = 0; it < prm.max_newton; ++it) {
            ContactSet& A = set[cur];
            const int64_t k = A.k;
            // element gradients and projected Hessians
            ctx->prof.start(GIPC_PROF_ELEMENTS, st);
            if ((s = ctx->slot[N_TEVAL].reserve(sizeof(double) * 12 * T + hb * 144 * T + 16)) != GIPC_OK) return s;
            double* tg = ctx->slot[N_TEVAL].as<double>();
            void* th = tg + 12 * (int64_t)T;
            gipc_elastic_params ep = prm.elastic;
            ep.scale = dt * dt;
            if ((s = gipc_eval_tets(x, n, sc.tets, T, sc.Dm_inv, sc.vol, &ep, prm.prec, GIPC_HESS_DENSE, nullptr, tg, th, st)) != GIPC_OK)
                return s;
            const bool rank1 = prm.hess_mode == GIPC_HESS_RANK1;
            const int64_t hper = rank1 ? 12 : 144;
            if ((s = ctx->slot[N_SEVAL].reserve(sizeof(double) * 13 * std::max<int64_t>(k, 1) + hb * hper * k + 16)) != GIPC_OK)
                return s;
            double* sg = ctx->slot[N_SEVAL].as<double>();
            double* sl = sg + 12 * k;
            void* sh = sl + std::max<int64_t>(k, 1);
            if (k > 0 &&
                (s = eval_stencils_ordered(x, n, A.st, k, A.eps, &prm.barrier, prm.prec, prm.hess_mode, nullptr, sg, sh,
                                           rank1 ? sl : nullptr, nullptr, A.order, st)) != GIPC_OK)
                return s;
            ctx->prof.stop(GIPC_PROF_ELEMENTS, st);
            grad_base_kernel<<<nb(m3, 256), 256, 0, st>>>(x, xt, sc.mass, n, gb);
            // H = M + sum P^T H_e P, g = M(x - xt) + sum P^T g_e
            gipc_elements te{sc.tets, T, GIPC_HESS_DENSE, th, nullptr, tg};
            gipc_elements se{A.st, k, prm.hess_mode, sh, rank1 ? sl : nullptr, sg};
            if ((s = ctx->slot[N_ROW].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return s;
            gipc_bsr H{};
            H.prec = prm.prec;
            H.rowptr = ctx->slot[N_ROW].as<int32_t>();
            for (int attempt = 0; attempt < 2; ++attempt) {
                H.capacity = std::min<int64_t>((int64_t)(ctx->slot[N_COL].bytes / sizeof(int32_t)),
                                               (int64_t)(ctx->slot[N_VAL].bytes / (9 * hb)));
                H.colidx = ctx->slot[N_COL].as<int32_t>();
                H.vals = ctx->slot[N_VAL].ptr;
                s = gipc_assemble_bsr(ctx, n, k > 0 ? &se : nullptr, &te, sc.mass, gb, &H, g, st);
                if (s != GIPC_ERR_CAPACITY || H.nnzb <= H.capacity) break;
                const int64_t cap = H.nnzb + H.nnzb / 8 + 1024;
                if ((s = ctx->slot[N_COL].reserve(sizeof(int32_t) * cap)) != GIPC_OK) return s;
                if ((s = ctx->slot[N_VAL].reserve(9 * hb * cap)) != GIPC_OK) return s;
                s = GIPC_ERR_CAPACITY;
            }
            if (s != GIPC_OK) return s;
            // d = argmin of the quadratic model (modified PCG, fixed vertices filtered)
            negate_kernel<<<nb(m3, 256), 256, 0, st>>>(g, m3, rhs);
            cudaMemsetAsync(d, 0, sizeof(double) * m3, st);
            gipc_pcg_params pp{prm.pcg_tol, prm.max_pcg, 0};
            int pit = 0;
            s = gipc_pcg(ctx, &H, rhs, d, sc.fixed, &pp, &pit, nullptr, st);
            if (s != GIPC_OK && s != GIPC_ERR_NOT_CONVERGED) return s;
            S.pcg_iters += pit;
            // step filter and backtracking
            double alpha = 1.0;
            if ((s = ccd_impl(ctx, x, d, n, sc.surface, 0.1, &alpha, st, nullptr, 1, nullptr, true)) != GIPC_OK) return s;
            cudaMemcpyAsync(xp, x, sizeof(double) * m3, cudaMemcpyDeviceToDevice, st);
            const int nxt = 1 - cur;
            double I_new = I_prev;
            for (int ls = 0; ls < std::max(prm.max_ls, 1); ++ls) {
                axpy_kernel<<<nb(m3, 256), 256, 0, st>>>(xp, d, alpha, m3, x);
                if ((s = potential(x, set[nxt], &I_new)) != GIPC_OK) return s;
                ++S.ls_trials;
                if (I_new <= I_prev) break;
                alpha *= 0.5;
            }
            cur = nxt;
            I_prev = I_new;
            ++S.newton_iters;
            S.last_alpha = alpha;
            reduce(R_MAXABS, d, nullptr, nullptr, 0, m3, partial + 3 * kRedBlocks, res + 3, st);
            double dmax = 0.0;
            cudaMemcpyAsync(&dmax, res + 3, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step: step norm");
            if (dmax / (sc.l * dt) <= prm.eps_d) {
                S.converged = 1;
                break;
            }
        }
        velocity_kernel<<<nb(m3, 256), 256, 0, st>>>(x, x0, dt, m3, v);
        S.contacts = set[cur].k;
        S.energy = I_prev;
        if (stats) *stats = S;
        return check_launch("gipc_newton_step");
    }
};


// ============================================================================ batched scenes
// Many independent scenes in one set of launches per phase: the scenes are concatenated (vertex
// ranges voff), contacts never pair across scenes (the broad phase hashes the scene into its
// cells), the matrix is block diagonal, the PCG keeps per-scene scalars, and every scalar of the
// Newton loop (energies, CCD step, line-search step, stopping test) is per scene.

enum BatchSlot { B_VS = 48 };

// scene of vertex v for every v (scene k owns [voff[k], voff[k+1]))
__global__ void vertex_scene_kernel(const int64_t* __restrict__ voff, int nscenes, int64_t n, int32_t* __restrict__ vs) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    int lo = 0, hi = nscenes - 1;
    while (lo < hi) {   // last k with voff[k] <= v
        const int mid = (lo + hi + 1) >> 1;
        if (voff[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    vs[v] = lo;
}

// Layout check: every element inside one scene; element lists non-decreasing in scene.
__global__ void batch_layout_kernel(const int32_t* __restrict__ ids, int nv, int64_t m, int64_t n,
                                    const int32_t* __restrict__ vs, int32_t* __restrict__ bad) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int32_t s0 = -1;
    for (int a = 0; a < nv; ++a) {
        const int32_t v = ids[a * m + t];
        if (v < 0 || v >= n) {
            atomicOr(bad, 1);
            return;
        }
        if (s0 < 0) s0 = vs[v];
        else if (vs[v] != s0) atomicOr(bad, 2);
    }
    if (t + 1 < m) {
        const int32_t v1 = ids[t + 1];
        if (v1 >= 0 && v1 < n && vs[v1] < s0) atomicOr(bad, 4);
    }
}

// Range [lo, hi) of scene sc in a list of m items whose scene (of the first vertex) is
// non-decreasing; stencils decode a sign-encoded first slot.
template <bool STENCIL>
__device__ __forceinline__ void scene_range(const int32_t* __restrict__ first, int64_t lo0, int64_t hi0,
                                            const int32_t* __restrict__ vs, int sc, int64_t& lo, int64_t& hi) {
    auto key = [&](int64_t i) {
        const int32_t v = first[i];
        return vs[STENCIL ? (v >= 0 ? v : ~v) : v];
    };
    int64_t a = lo0, b = hi0;   // first index with key >= sc
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (key(m) < sc) a = m + 1;
        else b = m;
    }
    lo = a;
    b = hi0;                    // first index with key > sc
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (key(m) <= sc) a = m + 1;
        else b = m;
    }
    hi = a;
}

__device__ __forceinline__ double bsum_all(double v) {   // fixed-order block sum, broadcast
    __shared__ double sh[32];
    __shared__ double total;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) total = t;
    }
    __syncthreads();
    const double r = total;
    __syncthreads();
    return r;
}

// Per-scene incremental potential: 1/2 sum m |x - xt|^2 over the scene's vertices + its tets'
// energies + its stencils' energies (point-triangle block [0, npt), then edge-edge block).
// One CTA per scene, each sum in a fixed order.
__global__ void __launch_bounds__(256)
scene_energy_kernel(const double* __restrict__ x, const double* __restrict__ xt, const double* __restrict__ mass,
                    int64_t n, const int64_t* __restrict__ voff, const int32_t* __restrict__ tets, int64_t T,
                    const double* __restrict__ te, const int32_t* __restrict__ st, int64_t k, int64_t npt,
                    const double* __restrict__ se, const int32_t* __restrict__ vs, double* __restrict__ I,
                    int64_t* __restrict__ contacts, const int32_t* __restrict__ live) {
    const int sc = blockIdx.x;
    int64_t l1, h1, l2, h2;
    scene_range<true>(st, 0, npt, vs, sc, l1, h1);
    scene_range<true>(st, npt, k, vs, sc, l2, h2);
    if (threadIdx.x == 0 && contacts) contacts[sc] = (h1 - l1) + (h2 - l2);
    if (live && !live[sc]) return;   // (uniform in the block) I[sc] keeps its value
    double a = 0.0;
    for (int64_t i = voff[sc] + threadIdx.x; i < voff[sc + 1]; i += blockDim.x) {
        const double dx = __dsub_rn(x[i], xt[i]), dy = __dsub_rn(x[n + i], xt[n + i]), dz = __dsub_rn(x[2 * n + i], xt[2 * n + i]);
        a = __dadd_rn(a, __dmul_rn(mass[i], __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz))));
    }
    const double inertia = bsum_all(a);
    int64_t lo, hi;
    scene_range<false>(tets, 0, T, vs, sc, lo, hi);
    a = 0.0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) a = __dadd_rn(a, te[i]);
    const double elastic = bsum_all(a);
    a = 0.0;
    for (int64_t i = l1 + threadIdx.x; i < h1; i += blockDim.x) a = __dadd_rn(a, se[i]);
    for (int64_t i = l2 + threadIdx.x; i < h2; i += blockDim.x) a = __dadd_rn(a, se[i]);
    const double barrier = bsum_all(a);
    if (threadIdx.x == 0) I[sc] = __dadd_rn(__dadd_rn(__dmul_rn(0.5, inertia), elastic), barrier);
}

// Per-scene max |d| over the scene's vertices.
__global__ void __launch_bounds__(256)
scene_maxabs_kernel(const double* __restrict__ d, int64_t n, const int64_t* __restrict__ voff, double* __restrict__ out) {
    const int sc = blockIdx.x;
    double a = 0.0;
    for (int64_t i = voff[sc] + threadIdx.x; i < voff[sc + 1]; i += blockDim.x)
        a = fmax(a, fmax(fabs(d[i]), fmax(fabs(d[n + i]), fabs(d[2 * n + i]))));
    __shared__ double sh[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, sh[w]);
        out[sc] = m;
    }
}

// x = xp + alpha[scene] d
__global__ void axpy_scene_kernel(const double* __restrict__ xp, const double* __restrict__ d,
                                  const double* __restrict__ alpha, const int32_t* __restrict__ vs, int64_t n,
                                  double* __restrict__ x) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    x[j] = __dadd_rn(xp[j], __dmul_rn(alpha[vs[j % n]], d[j]));
}

// solver filter: fixed vertices and every vertex of a scene that has stopped
__global__ void scene_mask_kernel(const uint8_t* __restrict__ fixed, const int32_t* __restrict__ vs,
                                  const int32_t* __restrict__ active, int64_t n, uint8_t* __restrict__ mask) {
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    mask[v] = (fixed && fixed[v]) || !active[vs[v]] ? 1 : 0;
}

// ---- packing: the batch is rebuilt (gathered) to hold only the scenes still iterating ------
// Element ranges of every scene in a list ordered by scene (one thread per scene).
__global__ void scene_elem_ranges_kernel(const int32_t* __restrict__ first, int64_t m, const int32_t* __restrict__ vs,
                                         int ns, int64_t* __restrict__ lo, int64_t* __restrict__ hi) {
    const int sc = blockIdx.x * blockDim.x + threadIdx.x;
    if (sc >= ns) return;
    int64_t l, h;
    scene_range<false>(first, 0, m, vs, sc, l, h);
    lo[sc] = l;
    hi[sc] = h;
}

__device__ __forceinline__ int packed_scene(const int64_t* __restrict__ off, int nsp, int64_t i) {
    int lo = 0, hi = nsp - 1;   // last k with off[k] <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Packed vertex v' of packed scene s' comes from original vertex src[s'] + (v' - pvoff[s']).
__global__ void pack_vertices_kernel(int64_t np, const int64_t* __restrict__ pvoff, int nsp,
                                     const int64_t* __restrict__ src, int64_t n, const double* __restrict__ x,
                                     const double* __restrict__ xt, const double* __restrict__ rest,
                                     const double* __restrict__ mass, const uint8_t* __restrict__ fixed,
                                     double* __restrict__ xw, double* __restrict__ xtw, double* __restrict__ restw,
                                     double* __restrict__ massw, uint8_t* __restrict__ fixedw, int64_t* __restrict__ orig,
                                     int32_t* __restrict__ vsw) {
    const int64_t vp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vp >= np) return;
    const int sp = packed_scene(pvoff, nsp, vp);
    const int64_t v = src[sp] + (vp - pvoff[sp]);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        xw[c * np + vp] = x[c * n + v];
        xtw[c * np + vp] = xt[c * n + v];
        restw[c * np + vp] = rest[c * n + v];
    }
    massw[vp] = mass[v];
    fixedw[vp] = fixed ? fixed[v] : 0;
    orig[vp] = v;
    vsw[vp] = sp;
}

// Packed element e' of packed scene s' is original element esrc[s'] + (e' - peoff[s']); its
// vertex ids shift by vshift[s'].  Optional per-element payload: Dm^-1 (9) and volume.
__global__ void pack_elements_kernel(int64_t mp, const int64_t* __restrict__ peoff, int nsp,
                                     const int64_t* __restrict__ esrc, const int64_t* __restrict__ vshift, int nv,
                                     const int32_t* __restrict__ ids, int64_t m, int32_t* __restrict__ idsw,
                                     const double* __restrict__ dm, const double* __restrict__ vol,
                                     double* __restrict__ dmw, double* __restrict__ volw) {
    const int64_t ep = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ep >= mp) return;
    const int sp = packed_scene(peoff, nsp, ep);
    const int64_t e = esrc[sp] + (ep - peoff[sp]);
    for (int a = 0; a < nv; ++a) idsw[a * mp + ep] = (int32_t)(ids[a * m + e] + vshift[sp]);
    if (dm) {
#pragma unroll
        for (int k = 0; k < 9; ++k) dmw[k * mp + ep] = dm[k * m + e];
        volw[ep] = vol[e];
    }
}

__global__ void unpack_x_kernel(int64_t np, const int64_t* __restrict__ orig, const double* __restrict__ xw, int64_t n,
                                double* __restrict__ x) {
    const int64_t vp = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (vp >= np) return;
#pragma unroll
    for (int c = 0; c < 3; ++c) x[c * n + orig[vp]] = xw[c * np + vp];
}

enum PackSlot { W_V = 41, W_E = 42, W_S = 43, W_I = 44, W_M = 47 };

struct BatchStep {
    gipc_ctx* ctx;
    const gipc_scene& full;          // the caller's batch
    const gipc_step_params& prm;
    cudaStream_t st;
    const int ns_full;
    const int64_t* voff_full_h;
    const double* l_full_h;
    // current (possibly packed) batch
    gipc_scene sc{};
    int64_t n = 0;
    int ns = 0;
    std::vector<int> map;            // packed scene -> original scene
    std::vector<int64_t> voff_h;
    std::vector<double> l_h;
    int64_t* voff = nullptr;         // device [ns+1]
    int32_t* vs = nullptr;           // device [n]
    const int64_t* orig = nullptr;   // device [n] original vertex id, NULL when not packed
    double *x = nullptr, *xt = nullptr;
    // full-size vectors
    double *x0 = nullptr, *xt_full = nullptr, *xp = nullptr, *d = nullptr, *g = nullptr, *rhs = nullptr, *gb = nullptr;
    double *sI = nullptr, *sA = nullptr, *sD = nullptr;
    int64_t* sC = nullptr;
    int32_t* sAct = nullptr;      // device [ns] scenes still iterating
    int32_t* sSearch = nullptr;   // device [ns] scenes still searching along their step
    uint8_t* mask = nullptr;
    ContactSet set[2];
    // element ranges of every original scene (host) for packing
    std::vector<int64_t> tlo, thi, rlo, rhi, elo, ehi, plo, phi;
    std::vector<double> I_h, Inew_h, alpha_h, dmax_h;
    std::vector<int64_t> cont_h;
    std::vector<int32_t> active_h;
    int64_t npt_cur = 0, npt_nxt = 0;

    BatchStep(gipc_ctx* c, const gipc_scene& s, const gipc_step_params& p, cudaStream_t q, int nsc, const int64_t* vo,
              const double* l)
        : ctx(c), full(s), prm(p), st(q), ns_full(nsc), voff_full_h(vo), l_full_h(l) {
        set[0].slot = N_ST0;
        set[1].slot = N_ST1;
    }

    void sizes_per_scene() {
        I_h.assign(ns, 0.0);
        Inew_h.assign(ns, 0.0);
        alpha_h.assign(ns, 1.0);
        dmax_h.assign(ns, 0.0);
        cont_h.assign(ns, 0);
    }

    gipc_status scene_scalars() {
        gipc_status s;
        if ((s = ctx->slot[W_S].reserve(sizeof(double) * 3 * ns + sizeof(int64_t) * (2 * ns + 2) +
                                        sizeof(int32_t) * (2 * ns + 6) + 64)) != GIPC_OK)
            return s;
        sI = ctx->slot[W_S].as<double>();
        sA = sI + ns;
        sD = sA + ns;
        sC = reinterpret_cast<int64_t*>(sD + ns);
        voff = sC + ns;
        sAct = reinterpret_cast<int32_t*>(voff + ns + 2);
        sSearch = sAct + ns + 2;   // (sAct[ns] is the layout check's flag)
        return GIPC_OK;
    }

    gipc_status contacts_b(const double* xc, ContactSet& cs, int64_t* npt) {
        for (int attempt = 0; attempt < 2; ++attempt) {
            int64_t cnt = 0;
            const gipc_status s = find_contacts_impl(ctx, xc, sc.rest_x, n, sc.surface, prm.barrier.dhat, cs.st, cs.eps,
                                                     cs.cap, &cnt, true, vs, npt, st, ns, true);
            if (s == GIPC_OK) {
                cs.k = cnt;
                return stencil_type_order(cs.st, cs.k, cs.order, cs.tcnt, st);
            }
            if (s != GIPC_ERR_CAPACITY) return s;
            const gipc_status r = contact_storage(ctx, cs, cnt + cnt / 4 + 1024);
            if (r != GIPC_OK) return r;
        }
        return fail(GIPC_ERR_CUDA, "gipc_newton_step_batch: contact count changed between passes");
    }

    // per-scene I(x) into I_out (host) and the contacts at x; with `live` (device, per scene) the
    // energies of the other scenes are neither evaluated nor changed (their contacts still are)
    gipc_status potential_b(const double* xc, ContactSet& cs, int64_t* npt, std::vector<double>& I_out,
                            const int32_t* live = nullptr) {
        gipc_status s;
        if ((s = contacts_b(xc, cs, npt)) != GIPC_OK) return s;
        const int64_t T = sc.T, k = cs.k;
        gipc_prof_span span(ctx->prof, GIPC_PROF_ENERGY, st);
        if ((s = ctx->slot[N_ENER].reserve(sizeof(double) * (T + k + 2))) != GIPC_OK) return s;
        double* te = ctx->slot[N_ENER].as<double>();
        double* se = te + T;
        gipc_elastic_params ep = prm.elastic;
        ep.scale = prm.dt * prm.dt;
        if ((s = eval_tets_live(xc, n, sc.tets, T, sc.Dm_inv, sc.vol, &ep, GIPC_FP64, GIPC_HESS_DENSE, te, nullptr, nullptr,
                                vs, live, st)) != GIPC_OK)
            return s;
        if (k > 0 && (s = eval_stencils_ordered(xc, n, cs.st, k, cs.eps, &prm.barrier, GIPC_FP64, GIPC_HESS_DENSE, se, nullptr,
                                                nullptr, nullptr, nullptr, cs.order, st)) != GIPC_OK)
            return s;
        scene_energy_kernel<<<ns, 256, 0, st>>>(xc, xt, sc.mass, n, voff, sc.tets, T, te, cs.st, k, *npt, se, vs, sI, sC,
                                                live);
        cudaMemcpyAsync(I_out.data(), sI, sizeof(double) * ns, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(cont_h.data(), sC, sizeof(int64_t) * ns, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step_batch: energy");
        for (int k2 = 0; k2 < ns; ++k2)
            if (!std::isfinite(I_out[k2]))
                return fail(GIPC_ERR_NONFINITE, "gipc_newton_step_batch: non-finite energy in scene %d", map[k2]);
        return GIPC_OK;
    }

    // element ranges of every original scene in the four lists (one synchronisation)
    gipc_status full_ranges(const int32_t* vs_full) {
        gipc_status s;
        if ((s = ctx->slot[W_I].reserve(sizeof(int64_t) * 8 * (ns_full + 1))) != GIPC_OK) return s;
        int64_t* R = ctx->slot[W_I].as<int64_t>();
        const int32_t* lists[4] = {full.tets, full.surface.tris, full.surface.edges, full.surface.verts};
        const int64_t counts[4] = {full.T, full.surface.ntri, full.surface.nedge, full.surface.nvert};
        for (int q = 0; q < 4; ++q)
            scene_elem_ranges_kernel<<<nb(ns_full, 128), 128, 0, st>>>(lists[q], counts[q], vs_full, ns_full,
                                                                       R + 2 * q * ns_full, R + (2 * q + 1) * ns_full);
        std::vector<int64_t> h(8 * (size_t)ns_full);
        cudaMemcpyAsync(h.data(), R, sizeof(int64_t) * 8 * ns_full, cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step_batch: ranges");
        auto cp = [&](std::vector<int64_t>& o, int k) { o.assign(h.begin() + k * ns_full, h.begin() + (k + 1) * ns_full); };
        cp(tlo, 0);
        cp(thi, 1);
        cp(rlo, 2);
        cp(rhi, 3);
        cp(elo, 4);
        cp(ehi, 5);
        cp(plo, 6);
        cp(phi, 7);
        return GIPC_OK;
    }

    // Rebuild the working batch from the caller's arrays with the original scenes `keep`.
    gipc_status pack(const std::vector<int>& keep, double* x_full) {
        gipc_status s;
        ctx->ccache.valid = false;   // the packed lists reuse the same buffers with other scenes
        const int nsp = (int)keep.size();
        std::vector<int64_t> pvoff(nsp + 1, 0), src(nsp), vshift(nsp);
        std::vector<int64_t> poff[4], psrc[4];
        const std::vector<int64_t>* los[4] = {&tlo, &rlo, &elo, &plo};
        const std::vector<int64_t>* his[4] = {&thi, &rhi, &ehi, &phi};
        for (int q = 0; q < 4; ++q) {
            poff[q].assign(nsp + 1, 0);
            psrc[q].assign(nsp, 0);
        }
        for (int k = 0; k < nsp; ++k) {
            const int o = keep[k];
            src[k] = voff_full_h[o];
            pvoff[k + 1] = pvoff[k] + (voff_full_h[o + 1] - voff_full_h[o]);
            vshift[k] = pvoff[k] - voff_full_h[o];
            for (int q = 0; q < 4; ++q) {
                psrc[q][k] = (*los[q])[o];
                poff[q][k + 1] = poff[q][k] + ((*his[q])[o] - (*los[q])[o]);
            }
        }
        const int64_t np = pvoff[nsp];
        const int64_t mT = poff[0][nsp], mR = poff[1][nsp], mE = poff[2][nsp], mP = poff[3][nsp];
        // small index arrays: pvoff, src, vshift, then (poff, psrc) for the four lists
        const size_t idx_words = (size_t)(nsp + 1) + 2 * nsp + 4 * (2 * nsp + 1);
        if ((s = ctx->slot[W_M].reserve(sizeof(int64_t) * (idx_words + 8))) != GIPC_OK) return s;
        int64_t* M = ctx->slot[W_M].as<int64_t>();
        std::vector<int64_t> hm;
        hm.reserve(idx_words);
        hm.insert(hm.end(), pvoff.begin(), pvoff.end());
        hm.insert(hm.end(), src.begin(), src.end());
        hm.insert(hm.end(), vshift.begin(), vshift.end());
        for (int q = 0; q < 4; ++q) {
            hm.insert(hm.end(), poff[q].begin(), poff[q].end());
            hm.insert(hm.end(), psrc[q].begin(), psrc[q].end());
        }
        cudaMemcpyAsync(M, hm.data(), sizeof(int64_t) * hm.size(), cudaMemcpyHostToDevice, st);
        const int64_t* d_pvoff = M;
        const int64_t* d_src = M + nsp + 1;
        const int64_t* d_vshift = d_src + nsp;
        const int64_t* d_poff[4];
        const int64_t* d_psrc[4];
        const int64_t* cur = d_vshift + nsp;
        for (int q = 0; q < 4; ++q) {
            d_poff[q] = cur;
            d_psrc[q] = cur + nsp + 1;
            cur += 2 * nsp + 1;
        }
        // vertex data: x, xt, rest (3 each), mass, original id, scene id, fixed, solver mask
        const size_t vbytes = sizeof(double) * 10 * np + sizeof(int64_t) * np + sizeof(int32_t) * np + 2 * np + 64;
        if ((s = ctx->slot[W_V].reserve(vbytes)) != GIPC_OK) return s;
        double* V = ctx->slot[W_V].as<double>();
        double* xw = V;
        double* xtw = V + 3 * np;
        double* restw = V + 6 * np;
        double* massw = V + 9 * np;
        int64_t* origw = reinterpret_cast<int64_t*>(V + 10 * np);
        int32_t* vsw = reinterpret_cast<int32_t*>(origw + np);
        uint8_t* fixedw = reinterpret_cast<uint8_t*>(vsw + np);
        uint8_t* maskw = fixedw + np;
        pack_vertices_kernel<<<nb(np, 256), 256, 0, st>>>(np, d_pvoff, nsp, d_src, full.n, x_full, xt_full, full.rest_x,
                                                          full.mass, full.fixed, xw, xtw, restw, massw, fixedw, origw, vsw);
        // elements: tets (+ Dm^-1, volume), triangles, edges, surface vertices
        const size_t ebytes = sizeof(int32_t) * (4 * mT + 3 * mR + 2 * mE + mP) + sizeof(double) * 10 * mT + 256;
        if ((s = ctx->slot[W_E].reserve(ebytes)) != GIPC_OK) return s;
        double* E = ctx->slot[W_E].as<double>();
        double* dmw = E;
        double* volw = E + 9 * mT;
        int32_t* tw = reinterpret_cast<int32_t*>(volw + mT);
        int32_t* rw = tw + 4 * mT;
        int32_t* ew = rw + 3 * mR;
        int32_t* pw = ew + 2 * mE;
        const int32_t* lists[4] = {full.tets, full.surface.tris, full.surface.edges, full.surface.verts};
        const int64_t counts[4] = {full.T, full.surface.ntri, full.surface.nedge, full.surface.nvert};
        int32_t* outs[4] = {tw, rw, ew, pw};
        const int64_t pm[4] = {mT, mR, mE, mP};
        const int nvs[4] = {4, 3, 2, 1};
        for (int q = 0; q < 4; ++q)
            if (pm[q] > 0)
                pack_elements_kernel<<<nb(pm[q], 256), 256, 0, st>>>(
                    pm[q], d_poff[q], nsp, d_psrc[q], d_vshift, nvs[q], lists[q], counts[q], outs[q],
                    q == 0 ? full.Dm_inv : nullptr, q == 0 ? full.vol : nullptr, q == 0 ? dmw : nullptr,
                    q == 0 ? volw : nullptr);
        // the working batch
        ns = nsp;
        n = np;
        map = keep;
        voff_h = pvoff;
        l_h.assign(nsp, 0.0);
        for (int k = 0; k < nsp; ++k) l_h[k] = l_full_h[keep[k]];
        sc = full;
        sc.n = np;
        sc.rest_x = restw;
        sc.tets = tw;
        sc.T = mT;
        sc.Dm_inv = dmw;
        sc.vol = volw;
        sc.mass = massw;
        sc.fixed = fixedw;
        sc.surface = gipc_surface{rw, mR, ew, mE, pw, mP};
        x = xw;
        xt = xtw;
        orig = origw;
        vs = vsw;
        mask = maskw;
        if ((s = scene_scalars()) != GIPC_OK) return s;
        cudaMemcpyAsync(voff, voff_h.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, st);
        sizes_per_scene();
        return check_launch("gipc_newton_step_batch: pack");
    }

    void unpack(double* x_full) {
        if (orig) unpack_x_kernel<<<nb(n, 256), 256, 0, st>>>(n, orig, x, full.n, x_full);
    }

    gipc_status run_batch(double* x_full, double* v, gipc_step_stats* stats) {
        const int64_t nf = full.n, m3f = 3 * nf;
        gipc_status s;
        ctx->ccache.valid = false;   // candidates are reused only within this step
        if ((s = ctx->slot[N_VEC].reserve(sizeof(double) * 7 * m3f)) != GIPC_OK) return s;
        if ((s = ctx->slot[B_VS].reserve(sizeof(int32_t) * (nf + 1) + nf + 64)) != GIPC_OK) return s;
        x0 = ctx->slot[N_VEC].as<double>();
        xt_full = x0 + m3f;
        xp = xt_full + m3f;
        d = xp + m3f;
        g = d + m3f;
        rhs = g + m3f;
        gb = rhs + m3f;
        for (auto& cs : set) contact_view(ctx, cs);
        // the unpacked working batch is the caller's
        ns = ns_full;
        n = nf;
        sc = full;
        map.resize(ns);
        for (int k = 0; k < ns; ++k) map[k] = k;
        voff_h.assign(voff_full_h, voff_full_h + ns + 1);
        l_h.assign(l_full_h, l_full_h + ns);
        vs = ctx->slot[B_VS].as<int32_t>();
        mask = reinterpret_cast<uint8_t*>(vs + nf + 1);
        orig = nullptr;
        x = x_full;
        xt = xt_full;
        if ((s = scene_scalars()) != GIPC_OK) return s;
        sizes_per_scene();
        std::vector<int32_t> act_full(ns_full, 1);
        // scene of every vertex, and the layout the per-scene sums rely on
        cudaMemcpyAsync(voff, voff_h.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, st);
        vertex_scene_kernel<<<nb(n, 256), 256, 0, st>>>(voff, ns, n, vs);
        int32_t* bad = sAct + ns;
        cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
        if (sc.T > 0) batch_layout_kernel<<<nb(sc.T, 256), 256, 0, st>>>(sc.tets, 4, sc.T, n, vs, bad);
        const gipc_surface& sf = sc.surface;
        if (sf.ntri > 0) batch_layout_kernel<<<nb(sf.ntri, 256), 256, 0, st>>>(sf.tris, 3, sf.ntri, n, vs, bad);
        if (sf.nedge > 0) batch_layout_kernel<<<nb(sf.nedge, 256), 256, 0, st>>>(sf.edges, 2, sf.nedge, n, vs, bad);
        if (sf.nvert > 0) batch_layout_kernel<<<nb(sf.nvert, 256), 256, 0, st>>>(sf.verts, 1, sf.nvert, n, vs, bad);
        int32_t bad_h = 0;
        cudaMemcpyAsync(&bad_h, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step_batch: layout");
        if (bad_h)
            return fail(GIPC_ERR_INVALID_ARG,
                        "gipc_newton_step_batch: an element spans two scenes, an id is out of range, or a list is not "
                        "ordered by scene (code %d)",
                        bad_h);
        if ((s = full_ranges(vs)) != GIPC_OK) return s;
        const double dt = prm.dt;
        cudaMemcpyAsync(x0, x_full, sizeof(double) * m3f, cudaMemcpyDeviceToDevice, st);
        inertia_target_kernel<<<nb(nf, 256), 256, 0, st>>>(x0, v, full.fixed, nf, dt, (dt * dt) * prm.gravity[0],
                                                            (dt * dt) * prm.gravity[1], (dt * dt) * prm.gravity[2], xt_full);
        int cur = 0;
        if ((s = potential_b(x, set[cur], &npt_cur, I_h)) != GIPC_OK) return s;
        std::vector<gipc_step_stats> S((size_t)ns_full);
        std::vector<double> I_full(ns_full, 0.0);
        std::vector<int64_t> cont_full(ns_full, 0);
        std::vector<int> piters(ns_full, 0), pstat(ns_full, 0);
        std::vector<int32_t> accepted(ns_full, 0);
        active_h.assign(ns, 1);
        const bool mixed = prm.prec == GIPC_MIXED;
        const size_t hb = mixed ? sizeof(float) : sizeof(double);
        for (int it = 0; it < prm.max_newton; ++it) {
            int n_active = 0;
            for (int k = 0; k < ns; ++k) n_active += active_h[k] != 0;
            if (n_active == 0) break;
            if (2 * n_active <= ns) {
                // half the packed scenes have stopped: keep their results, repack the others
                for (int k = 0; k < ns; ++k) {
                    I_full[map[k]] = I_h[k];
                    cont_full[map[k]] = cont_h[k];
                }
                unpack(x_full);
                std::vector<int> keep;
                for (int k = 0; k < ns; ++k)
                    if (active_h[k]) keep.push_back(map[k]);
                if ((s = pack(keep, x_full)) != GIPC_OK) return s;
                active_h.assign(ns, 1);
                if ((s = potential_b(x, set[cur], &npt_cur, I_h)) != GIPC_OK) return s;
            }
            ContactSet& A = set[cur];
            const int64_t k = A.k;
            const int64_t m3 = 3 * n;
            const int T = (int)sc.T;
            // the scenes still iterating: the others' elements give zero gradient and Hessian (their
            // directions are filtered out below), so they are not evaluated
            cudaMemcpyAsync(sAct, active_h.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st);
            ctx->prof.start(GIPC_PROF_ELEMENTS, st);
            if ((s = ctx->slot[N_TEVAL].reserve(sizeof(double) * 12 * T + hb * 144 * T + 16)) != GIPC_OK) return s;
            double* tg = ctx->slot[N_TEVAL].as<double>();
            void* th = tg + 12 * (int64_t)T;
            gipc_elastic_params ep = prm.elastic;
            ep.scale = dt * dt;
            if ((s = eval_tets_live(x, n, sc.tets, T, sc.Dm_inv, sc.vol, &ep, prm.prec, GIPC_HESS_DENSE, nullptr, tg, th, vs,
                                    sAct, st)) != GIPC_OK)
                return s;
            const bool rank1 = prm.hess_mode == GIPC_HESS_RANK1;
            const int64_t hper = rank1 ? 12 : 144;
            if ((s = ctx->slot[N_SEVAL].reserve(sizeof(double) * 13 * std::max<int64_t>(k, 1) + hb * hper * k + 16)) != GIPC_OK)
                return s;
            double* sg = ctx->slot[N_SEVAL].as<double>();
            double* sl = sg + 12 * k;
            void* sh = sl + std::max<int64_t>(k, 1);
            if (k > 0 &&
                (s = eval_stencils_ordered(x, n, A.st, k, A.eps, &prm.barrier, prm.prec, prm.hess_mode, nullptr, sg, sh,
                                           rank1 ? sl : nullptr, nullptr, A.order, st)) != GIPC_OK)
                return s;
            ctx->prof.stop(GIPC_PROF_ELEMENTS, st);
            grad_base_kernel<<<nb(m3, 256), 256, 0, st>>>(x, xt, sc.mass, n, gb);
            gipc_elements te{sc.tets, T, GIPC_HESS_DENSE, th, nullptr, tg};
            gipc_elements se{A.st, k, prm.hess_mode, sh, rank1 ? sl : nullptr, sg};
            if ((s = ctx->slot[N_ROW].reserve(sizeof(int32_t) * (n + 1))) != GIPC_OK) return s;
            gipc_bsr H{};
            H.prec = prm.prec;
            H.rowptr = ctx->slot[N_ROW].as<int32_t>();
            for (int attempt = 0; attempt < 2; ++attempt) {
                H.capacity = std::min<int64_t>((int64_t)(ctx->slot[N_COL].bytes / sizeof(int32_t)),
                                               (int64_t)(ctx->slot[N_VAL].bytes / (9 * hb)));
                H.colidx = ctx->slot[N_COL].as<int32_t>();
                H.vals = ctx->slot[N_VAL].ptr;
                s = gipc_assemble_bsr(ctx, n, k > 0 ? &se : nullptr, &te, sc.mass, gb, &H, g, st);
                if (s != GIPC_ERR_CAPACITY || H.nnzb <= H.capacity) break;
                const int64_t cap = H.nnzb + H.nnzb / 8 + 1024;
                if ((s = ctx->slot[N_COL].reserve(sizeof(int32_t) * cap)) != GIPC_OK) return s;
                if ((s = ctx->slot[N_VAL].reserve(9 * hb * cap)) != GIPC_OK) return s;
                s = GIPC_ERR_CAPACITY;
            }
            if (s != GIPC_OK) return s;
            // directions of the scenes still iterating; stopped scenes are filtered out (d = 0)
            scene_mask_kernel<<<nb(n, 256), 256, 0, st>>>(sc.fixed, vs, sAct, n, mask);
            negate_kernel<<<nb(m3, 256), 256, 0, st>>>(g, m3, rhs);
            cudaMemsetAsync(d, 0, sizeof(double) * m3, st);
            gipc_pcg_params pp{prm.pcg_tol, prm.max_pcg, 0};
            s = pcg_impl(ctx, &H, rhs, d, mask, &pp, nullptr, nullptr, st, voff, ns, piters.data(), pstat.data(),
                         voff_h.data());
            if (s != GIPC_OK && s != GIPC_ERR_NOT_CONVERGED) return s;
            // per-scene step filter, then backtracking per scene
            if ((s = ccd_impl(ctx, x, d, n, sc.surface, 0.1, alpha_h.data(), st, vs, ns, sA, true)) != GIPC_OK) return s;
            for (int q = 0; q < ns; ++q) {
                accepted[q] = active_h[q] ? 0 : 1;
                if (active_h[q]) S[map[q]].pcg_iters += piters[q];
            }
            cudaMemcpyAsync(xp, x, sizeof(double) * m3, cudaMemcpyDeviceToDevice, st);
            const int nxt = 1 - cur;
            std::vector<int32_t> searching(ns);
            for (int ls = 0; ls < std::max(prm.max_ls, 1); ++ls) {
                // the energies of the scenes still searching (an accepted scene's x stays as it is)
                for (int q = 0; q < ns; ++q) searching[q] = accepted[q] ? 0 : 1;
                cudaMemcpyAsync(sSearch, searching.data(), sizeof(int32_t) * ns, cudaMemcpyHostToDevice, st);
                cudaMemcpyAsync(sA, alpha_h.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, st);
                axpy_scene_kernel<<<nb(m3, 256), 256, 0, st>>>(xp, d, sA, vs, n, x);
                if ((s = potential_b(x, set[nxt], &npt_nxt, Inew_h, sSearch)) != GIPC_OK) return s;
                bool all = true;
                for (int q = 0; q < ns; ++q) {
                    if (accepted[q]) continue;
                    ++S[map[q]].ls_trials;
                    if (Inew_h[q] <= I_h[q]) accepted[q] = 1;
                    else {
                        alpha_h[q] *= 0.5;
                        all = false;
                    }
                }
                if (all) break;
            }
            cur = nxt;
            npt_cur = npt_nxt;
            scene_maxabs_kernel<<<ns, 256, 0, st>>>(d, n, voff, sD);
            cudaMemcpyAsync(dmax_h.data(), sD, sizeof(double) * ns, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_step_batch: step norm");
            for (int q = 0; q < ns; ++q) {
                if (!active_h[q]) continue;
                I_h[q] = Inew_h[q];
                gipc_step_stats& Z = S[map[q]];
                ++Z.newton_iters;
                Z.last_alpha = alpha_h[q];
                if (dmax_h[q] / (l_h[q] * dt) <= prm.eps_d) {
                    Z.converged = 1;
                    active_h[q] = 0;
                }
            }
        }
        for (int k = 0; k < ns; ++k) {
            I_full[map[k]] = I_h[k];
            cont_full[map[k]] = cont_h[k];
        }
        unpack(x_full);
        velocity_kernel<<<nb(m3f, 256), 256, 0, st>>>(x_full, x0, dt, m3f, v);
        for (int q = 0; q < ns_full; ++q) {
            S[q].contacts = cont_full[q];
            S[q].energy = I_full[q];
            if (stats) stats[q] = S[q];
        }
        return check_launch("gipc_newton_step_batch");
    }
};
}  // namespace
}  // namespace gipc

extern "C" gipc_status gipc_newton_step(gipc_ctx* ctx, const gipc_scene* sc, double* x, double* v,
                                        const gipc_step_params* prm, gipc_step_stats* stats, void* stream) {
    using namespace gipc;
    if (!ctx || !sc || !prm || !x || !v) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step: null argument");
    if (sc->n <= 0 || sc->T < 0 || !sc->rest_x || !sc->mass || (sc->T > 0 && (!sc->tets || !sc->Dm_inv || !sc->vol)))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step: incomplete scene");
    if (sc->T > 0x7fffffff) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step: too many tetrahedra");
    if (!(prm->dt > 0.0) || !(sc->l > 0.0) || !(prm->eps_d >= 0.0) || prm->max_newton < 0 || prm->max_pcg < 0 ||
        (prm->prec != GIPC_FP64 && prm->prec != GIPC_MIXED) ||
        (prm->hess_mode != GIPC_HESS_DENSE && prm->hess_mode != GIPC_HESS_RANK1))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step: bad step parameters");
    const gipc_barrier_params& b = prm->barrier;
    if (!(b.dhat > 0.0) || !(b.kappa >= 0.0) || !(b.d_thr_ratio > 0.0 && b.d_thr_ratio < 1.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step: bad barrier parameters");
    Step step(ctx, *sc, *prm, (cudaStream_t)stream);
    return step.run(x, v, stats);
}

extern "C" gipc_status gipc_newton_step_batch(gipc_ctx* ctx, const gipc_scene_batch* b, double* x, double* v,
                                              const gipc_step_params* prm, gipc_step_stats* stats, void* stream) {
    using namespace gipc;
    if (!ctx || !b || !prm || !x || !v) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: null argument");
    const gipc_scene* sc = &b->all;
    if (b->nscenes <= 0 || !b->vert_off_h || !b->l_h) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: no scenes");
    if (sc->n <= 0 || sc->T < 0 || !sc->rest_x || !sc->mass || (sc->T > 0 && (!sc->tets || !sc->Dm_inv || !sc->vol)))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: incomplete scene");
    if (sc->T > 0x7fffffff) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: too many tetrahedra");
    if (b->vert_off_h[0] != 0 || b->vert_off_h[b->nscenes] != sc->n)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: vertex ranges must start at 0 and end at n");
    for (int k = 0; k < b->nscenes; ++k) {
        if (b->vert_off_h[k + 1] <= b->vert_off_h[k]) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: empty or decreasing vertex range %d", k);
        if (!(b->l_h[k] > 0.0)) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: l of scene %d must be > 0", k);
    }
    if (!(prm->dt > 0.0) || !(prm->eps_d >= 0.0) || prm->max_newton < 0 || prm->max_pcg < 0 ||
        (prm->prec != GIPC_FP64 && prm->prec != GIPC_MIXED) ||
        (prm->hess_mode != GIPC_HESS_DENSE && prm->hess_mode != GIPC_HESS_RANK1))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: bad step parameters");
    const gipc_barrier_params& bp = prm->barrier;
    if (!(bp.dhat > 0.0) || !(bp.kappa >= 0.0) || !(bp.d_thr_ratio > 0.0 && bp.d_thr_ratio < 1.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_step_batch: bad barrier parameters");
    BatchStep step(ctx, *sc, *prm, (cudaStream_t)stream, b->nscenes, b->vert_off_h, b->l_h);
    return step.run_batch(x, v, stats);
}
