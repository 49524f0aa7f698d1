// Exact derivatives of the incremental potential and the implicit adjoint of a converged step.
//
// I(x) = 1/2 (x - xt)^T M (x - xt) + scale sum_T vol Psi(F_T) + sum_k kappa btilde_k(x)
// (Sec. 3.1, Eq. 1-2; Psi the Stable neo-Hookean energy, btilde the barrier of Eq. 24 times the
// mollifier of Eq. 25 for the nearly-parallel types).  Unlike the Newton path, nothing here is
// projected: the gradient and the Hessian are those of I itself, so they can be indefinite.
//
// Every element's energy is written once, generically over its number type, and evaluated with
// hyper-dual numbers (Fike and Alonso's second-order forward mode: v + a e1 + b e2 + ab e1 e2 with
// e1^2 = e2^2 = 0).  Seeding e1 with a direction u and e2 with the unit vector of local coordinate j
// gives df/dx_j in b and (H u)_j in ab exactly (no truncation); seeding e1 = e_i, e2 = e_j gives
// H_ij.  Element vectors are summed per vertex by gipc_scatter_elements (fixed order).
//
// Implicit adjoint (one implicit step x_{t+1} = argmin I, v_{t+1} = (x_{t+1} - x_t)/dt): with
// a = dL/dx_{t+1} + dL/dv_{t+1}/dt on free vertices, H lambda = a (H the exact Hessian at x_{t+1},
// fixed vertices filtered) gives dL/dv_t = dt M lambda, dL/dx_t = M lambda - dL/dv_{t+1}/dt on free
// vertices (dL/dx_{t+1} - (H lambda) on fixed ones), and E dL/dE = -lambda . grad I_elastic.
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
gipc_status pcg_impl(gipc_ctx* ctx, const gipc_bsr* A, const double* rhs, double* x, const uint8_t* fixed,
                     const gipc_pcg_params* prm, int* iters_out_h, double* rel_out_h, cudaStream_t st,
                     const int64_t* voff, int nscenes, int* scene_iters_h, int* scene_status_h,
                     const int64_t* voff_h);
gipc_status ccd_impl(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const gipc_surface& srf, double slack,
                     double* alpha_h, cudaStream_t st, const int32_t* vscene, int nscenes, double* amin_dev,
                     bool cached);

namespace {

enum DiffSlot { D_ELEM = 49, D_VEC = 50, D_RED = 51, D_CON = 52, D_HES = 53, D_ADJ = 54, D_ROW = 55, D_COL = 56, D_VAL = 57,
                D_POL = 58 };

// ------------------------------------------------------------------ hyper-dual numbers
struct HD {
    double v, a, b, ab;
};
__device__ __forceinline__ HD operator+(HD x, HD y) { return {x.v + y.v, x.a + y.a, x.b + y.b, x.ab + y.ab}; }
__device__ __forceinline__ HD operator-(HD x, HD y) { return {x.v - y.v, x.a - y.a, x.b - y.b, x.ab - y.ab}; }
__device__ __forceinline__ HD operator*(HD x, HD y) {
    return {x.v * y.v, x.a * y.v + x.v * y.a, x.b * y.v + x.v * y.b, x.ab * y.v + x.a * y.b + x.b * y.a + x.v * y.ab};
}
__device__ __forceinline__ HD operator*(double s, HD x) { return {s * x.v, s * x.a, s * x.b, s * x.ab}; }
__device__ __forceinline__ HD operator*(HD x, double s) { return s * x; }
__device__ __forceinline__ HD operator+(HD x, double s) { return {x.v + s, x.a, x.b, x.ab}; }
__device__ __forceinline__ HD operator-(HD x, double s) { return {x.v - s, x.a, x.b, x.ab}; }
__device__ __forceinline__ HD operator-(double s, HD x) { return {s - x.v, -x.a, -x.b, -x.ab}; }
// chain rule for f with f(v) = f0, f'(v) = f1, f''(v) = f2
__device__ __forceinline__ HD compose(HD x, double f0, double f1, double f2) {
    return {f0, f1 * x.a, f1 * x.b, f1 * x.ab + f2 * x.a * x.b};
}
__device__ __forceinline__ HD recip(HD x) {
    const double r = 1.0 / x.v;
    return compose(x, r, -r * r, 2.0 * r * r * r);
}
__device__ __forceinline__ HD operator/(HD x, HD y) { return x * recip(y); }
__device__ __forceinline__ HD log(HD x) { return compose(x, ::log(x.v), 1.0 / x.v, -1.0 / (x.v * x.v)); }
__device__ __forceinline__ double log(double x) { return ::log(x); }
__device__ __forceinline__ double val(HD x) { return x.v; }
__device__ __forceinline__ double val(double x) { return x; }

template <typename T>
struct V3T {
    T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3T<T> sub(const V3T<T>& a, const V3T<T>& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
template <typename T>
__device__ __forceinline__ T dot(const V3T<T>& a, const V3T<T>& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
template <typename T>
__device__ __forceinline__ V3T<T> cross(const V3T<T>& a, const V3T<T>& b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// ------------------------------------------------------------------ element energies
struct TetConst {
    double mu, lam, alpha, scale;
};

// scale * vol * Psi(F), F = Ds Dm^-1 (Dm^-1 row-major), Stable neo-Hookean Psi
template <typename T>
__device__ T tet_energy(const V3T<T> (&X)[4], const double* Dmi, double vol, const TetConst& K) {
    const V3T<T> d1 = sub(X[1], X[0]), d2 = sub(X[2], X[0]), d3 = sub(X[3], X[0]);
    const T Ds[3][3] = {{d1.x, d2.x, d3.x}, {d1.y, d2.y, d3.y}, {d1.z, d2.z, d3.z}};
    T F[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] = Ds[i][0] * Dmi[0 * 3 + j] + Ds[i][1] * Dmi[1 * 3 + j] + Ds[i][2] * Dmi[2 * 3 + j];
    T Ic = F[0][0] * F[0][0];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            if (i || j) Ic = Ic + F[i][j] * F[i][j];
    const T J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) - F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
    const T Jm = J - K.alpha;
    const T psi = 0.5 * K.mu * (Ic - 3.0) + 0.5 * K.lam * (Jm * Jm) - 0.5 * K.mu * log(Ic + 1.0);
    return (K.scale * vol) * psi;
}

// squared distance of a stencil type (slot order of gipc.h) and, for the parallel types, c
template <typename T>
__device__ T stencil_sqdist(int type, const V3T<T> (&X)[4]) {
    switch (type) {
        case GIPC_PT: {
            const V3T<T> nrm = cross(sub(X[2], X[1]), sub(X[3], X[1]));
            const T vn = dot(sub(X[0], X[1]), nrm);
            return vn * vn / dot(nrm, nrm);
        }
        case GIPC_EE:
        case GIPC_EE_PAR: {
            const V3T<T> nrm = cross(sub(X[1], X[0]), sub(X[3], X[2]));
            const T wn = dot(sub(X[2], X[0]), nrm);
            return wn * wn / dot(nrm, nrm);
        }
        case GIPC_PE: {
            const V3T<T> e = sub(X[2], X[1]);
            const V3T<T> c = cross(sub(X[0], X[1]), e);
            return dot(c, c) / dot(e, e);
        }
        case GIPC_PE_PAR: {
            const V3T<T> e = sub(X[3], X[2]);
            const V3T<T> c = cross(sub(X[0], X[2]), e);
            return dot(c, c) / dot(e, e);
        }
        case GIPC_PP: {
            const V3T<T> r = sub(X[0], X[1]);
            return dot(r, r);
        }
        default: {   // GIPC_PP_PAR
            const V3T<T> r = sub(X[0], X[2]);
            return dot(r, r);
        }
    }
}

// kappa * e(c) * b(g), b(g) = (dhat^2 - dhat^2 g)^2 ln^2 g (Eq. 24), e of Eq. 25; 0 when g >= 1
template <typename T>
__device__ T stencil_energy(int type, const V3T<T> (&X)[4], double eps_x, double dhat, double kappa, bool& active) {
    const double dh2 = dhat * dhat;
    const T g = stencil_sqdist(type, X) * (1.0 / dh2);
    active = val(g) < 1.0 && val(g) > 0.0;
    if (!active) return T(g * 0.0);
    const T u = dh2 - dh2 * g;
    const T lg = log(g);
    T e = u * u * (lg * lg);
    if (type >= GIPC_EE_PAR) {
        const V3T<T> w = cross(sub(X[1], X[0]), sub(X[3], X[2]));
        const T c = dot(w, w);
        if (val(c) < eps_x) e = ((2.0 / eps_x) * c - (c * c) * (1.0 / (eps_x * eps_x))) * e;
    }
    return kappa * e;
}

struct StencilConst {
    double dhat, kappa;
};

// load the element's vertices: tetrahedra (4 ids) or sign-encoded stencils; s = vertex count
__device__ __forceinline__ bool element_verts(bool is_tet, const int32_t* __restrict__ idx, int64_t cnt, int64_t e,
                                              int64_t n, int32_t v[4], int& s, int& type) {
    if (is_tet) {
        for (int a = 0; a < 4; ++a) v[a] = idx[a * cnt + e];
        s = 4;
        type = -1;
    } else {
        type = decode_stencil(idx[e], idx[cnt + e], idx[2 * cnt + e], idx[3 * cnt + e], v);
        if (type < 0) return false;
        s = stencil_verts(type);
    }
    for (int a = 0; a < s; ++a)
        if (v[a] < 0 || v[a] >= n) return false;
    return true;
}

// Per element: energy (optional), local gradient [3s] and local H u [3s] (if u) -> [12][cnt].
__global__ void elem_grad_hvp_kernel(bool is_tet, const int32_t* __restrict__ idx, int64_t cnt,
                                     const double* __restrict__ x, int64_t n, const double* __restrict__ u,
                                     const double* __restrict__ Dm_inv, const double* __restrict__ vol, TetConst K,
                                     const double* __restrict__ eps_x, StencilConst B, double* __restrict__ energy,
                                     double* __restrict__ grad, double* __restrict__ hvp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    int32_t v[4];
    int s, type;
    const bool ok = element_verts(is_tet, idx, cnt, e, n, v, s, type);
    if (!ok) {
        if (energy) energy[e] = 0.0;
        for (int j = 0; j < 12; ++j) {
            if (grad) grad[j * cnt + e] = 0.0;
            if (hvp) hvp[j * cnt + e] = 0.0;
        }
        return;
    }
    double X0[4][3], U[4][3];
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) {
            X0[a][c] = a < s ? x[c * n + v[a]] : 0.0;
            U[a][c] = (a < s && u) ? u[c * n + v[a]] : 0.0;
        }
    double Dmi[9];
    double vl = 0.0, ex = 0.0;
    if (is_tet) {
        for (int q = 0; q < 9; ++q) Dmi[q] = Dm_inv[q * cnt + e];
        vl = vol[e];
    } else {
        ex = eps_x ? eps_x[e] : 0.0;
    }
    if (energy) {
        V3T<double> Xd[4];
        for (int a = 0; a < 4; ++a) Xd[a] = {X0[a][0], X0[a][1], X0[a][2]};
        bool act;
        energy[e] = is_tet ? tet_energy(Xd, Dmi, vl, K) : stencil_energy(type, Xd, ex, B.dhat, B.kappa, act);
    }
    for (int j = 0; j < 3 * s; ++j) {
        V3T<HD> Xh[4];
        for (int a = 0; a < 4; ++a) {
            HD c3[3];
            for (int c = 0; c < 3; ++c) c3[c] = {X0[a][c], U[a][c], (3 * a + c == j) ? 1.0 : 0.0, 0.0};
            Xh[a] = {c3[0], c3[1], c3[2]};
        }
        bool act = true;
        const HD E = is_tet ? tet_energy(Xh, Dmi, vl, K) : stencil_energy(type, Xh, ex, B.dhat, B.kappa, act);
        if (grad) grad[j * cnt + e] = E.b;
        if (hvp) hvp[j * cnt + e] = E.ab;
    }
    for (int j = 3 * s; j < 12; ++j) {
        if (grad) grad[j * cnt + e] = 0.0;
        if (hvp) hvp[j * cnt + e] = 0.0;
    }
}

// Per element: the exact (3s)^2 Hessian block, row-major compact (entry a*3s + b) -> [144][cnt].
__global__ void elem_hessian_kernel(bool is_tet, const int32_t* __restrict__ idx, int64_t cnt,
                                    const double* __restrict__ x, int64_t n, const double* __restrict__ Dm_inv,
                                    const double* __restrict__ vol, TetConst K, const double* __restrict__ eps_x,
                                    StencilConst B, double* __restrict__ hess) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= cnt) return;
    int32_t v[4];
    int s, type;
    if (!element_verts(is_tet, idx, cnt, e, n, v, s, type)) {
        for (int q = 0; q < 144; ++q) hess[q * cnt + e] = 0.0;
        return;
    }
    double X0[4][3];
    for (int a = 0; a < 4; ++a)
        for (int c = 0; c < 3; ++c) X0[a][c] = a < s ? x[c * n + v[a]] : 0.0;
    double Dmi[9];
    double vl = 0.0, ex = 0.0;
    if (is_tet) {
        for (int q = 0; q < 9; ++q) Dmi[q] = Dm_inv[q * cnt + e];
        vl = vol[e];
    } else {
        ex = eps_x ? eps_x[e] : 0.0;
    }
    const int m = 3 * s;
    for (int i = 0; i < m; ++i)
        for (int j = i; j < m; ++j) {
            V3T<HD> Xh[4];
            for (int a = 0; a < 4; ++a) {
                HD c3[3];
                for (int c = 0; c < 3; ++c)
                    c3[c] = {X0[a][c], (3 * a + c == i) ? 1.0 : 0.0, (3 * a + c == j) ? 1.0 : 0.0, 0.0};
                Xh[a] = {c3[0], c3[1], c3[2]};
            }
            bool act = true;
            const HD E = is_tet ? tet_energy(Xh, Dmi, vl, K) : stencil_energy(type, Xh, ex, B.dhat, B.kappa, act);
            hess[(int64_t)(i * m + j) * cnt + e] = E.ab;
            hess[(int64_t)(j * m + i) * cnt + e] = E.ab;
        }
}

// ------------------------------------------------------------------ vector helpers
// base = M (x - xt) (if xt) or M u (if u): the mass part of the gradient / the product
__global__ void mass_times_kernel(const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ m,
                                  int64_t n, double* __restrict__ out) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    out[j] = m[j % n] * (b ? a[j] - b[j] : a[j]);
}

// m |x - xt|^2 per vertex
__global__ void inertia_terms_kernel(const double* __restrict__ x, const double* __restrict__ xt,
                                     const double* __restrict__ m, int64_t n, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dx = x[i] - xt[i], dy = x[n + i] - xt[n + i], dz = x[2 * n + i] - xt[2 * n + i];
    out[i] = m[i] * ((dx * dx + dy * dy) + dz * dz);
}

// a = adj_x + adj_v / dt on free vertices, 0 on fixed ones
__global__ void adjoint_rhs_kernel(const double* __restrict__ ax, const double* __restrict__ av,
                                   const uint8_t* __restrict__ fixed, int64_t n, double dt, double* __restrict__ a) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    const bool fx = fixed && fixed[j % n];
    a[j] = fx ? 0.0 : (ax ? ax[j] : 0.0) + (av ? av[j] / dt : 0.0);
}

// adj_v_old = dt M lambda (free), 0 (fixed); adj_x_old = M lambda - adj_v/dt (free),
// adj_x - (H lambda) (fixed)
__global__ void adjoint_out_kernel(const double* __restrict__ lam, const double* __restrict__ Hl,
                                   const double* __restrict__ m, const double* __restrict__ ax,
                                   const double* __restrict__ av, const uint8_t* __restrict__ fixed, int64_t n, double dt,
                                   double* __restrict__ ox, double* __restrict__ ov) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    const bool fx = fixed && fixed[j % n];
    const double ml = m[j % n] * lam[j];
    if (fx) {
        if (ox) ox[j] = (ax ? ax[j] : 0.0) - Hl[j];
        if (ov) ov[j] = 0.0;
    } else {
        if (ox) ox[j] = ml - (av ? av[j] / dt : 0.0);
        if (ov) ov[j] = dt * ml;
    }
}

// fixed-order sum of a[i] * (b ? b[i] : 1) into *out (one CTA)
__global__ void __launch_bounds__(1024) dot_kernel(const double* __restrict__ a, const double* __restrict__ b, int64_t m,
                                                   double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s += b ? a[i] * b[i] : a[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) *out = s;
    }
}

// xt = x0 + dt v0 + dt^2 g on free vertices, x0 on fixed ones (the inertia target of the step)
__global__ void step_target_kernel(const double* __restrict__ x0, const double* __restrict__ v0,
                                   const uint8_t* __restrict__ fixed, int64_t n, double dt, double g0, double g1,
                                   double g2, double* __restrict__ xt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool fx = fixed && fixed[i];
    const double g[3] = {g0, g1, g2};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double p = x0[q * n + i];
        xt[q * n + i] = fx ? p : __dadd_rn(__dadd_rn(p, __dmul_rn(dt, v0[q * n + i])), g[q]);
    }
}

// rhs = -g on free vertices, 0 on fixed ones
__global__ void neg_free_kernel(const double* __restrict__ g, const uint8_t* __restrict__ fixed, int64_t n,
                                double* __restrict__ rhs) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n) return;
    rhs[j] = (fixed && fixed[j % n]) ? 0.0 : -g[j];
}

// x += alpha d;  v = (x - x0) / dt when v is given
__global__ void step_apply_kernel(double* __restrict__ x, const double* __restrict__ d, double alpha, int64_t m) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) x[j] += alpha * d[j];
}

__global__ void step_velocity_kernel(const double* __restrict__ x, const double* __restrict__ x0, double dt, int64_t m,
                                     double* __restrict__ v) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) v[j] = (x[j] - x0[j]) / dt;
}

// max |a[i]| into *out (one CTA)
__global__ void __launch_bounds__(1024) maxabs_kernel(const double* __restrict__ a, int64_t m, double* __restrict__ out) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fmax(s, fabs(a[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
        if (threadIdx.x == 0) *out = s;
    }
}

inline unsigned nbk(int64_t w, int t) { return (unsigned)std::max<int64_t>(1, (w + t - 1) / t); }

TetConst tet_const(const gipc_elastic_params& ep) {
    return {ep.mu, ep.lambda, 1.0 + ep.mu / ep.lambda - ep.mu / (4.0 * ep.lambda), ep.scale};
}

}  // namespace

// I, grad I and (H u) for a given contact list (internal; the public entry checks arguments)
gipc_status potential_derivs_impl(gipc_ctx* ctx, const gipc_scene& sc, const double* x, const double* xt,
                                  const int32_t* st_idx, const double* eps_x, int64_t k, const gipc_barrier_params& bp,
                                  const gipc_elastic_params& ep, const double* u, double* energy_h, double* grad,
                                  double* Hu, bool tets_only, cudaStream_t st) {
    const int64_t n = sc.n, T = sc.T;
    const int64_t kk = tets_only ? 0 : k;
    gipc_status s;
    const int64_t ne = T + kk;
    if ((s = ctx->slot[D_ELEM].reserve(sizeof(double) * (25 * ne + 16))) != GIPC_OK) return s;
    double* eng = ctx->slot[D_ELEM].as<double>();
    double* tg = eng + ne;
    double* th = tg + 12 * T;
    double* sg = th + 12 * T;
    double* sh = sg + 12 * kk;
    const TetConst K = tet_const(ep);
    const StencilConst B{bp.dhat, bp.kappa};
    if (T > 0)
        elem_grad_hvp_kernel<<<nbk(T, 128), 128, 0, st>>>(true, sc.tets, T, x, n, u, sc.Dm_inv, sc.vol, K, nullptr, B,
                                                          energy_h ? eng : nullptr, grad ? tg : nullptr, Hu ? th : nullptr);
    if (kk > 0)
        elem_grad_hvp_kernel<<<nbk(kk, 128), 128, 0, st>>>(false, st_idx, kk, x, n, u, nullptr, nullptr, K, eps_x, B,
                                                           energy_h ? eng + T : nullptr, grad ? sg : nullptr,
                                                           Hu ? sh : nullptr);
    if ((s = ctx->slot[D_VEC].reserve(sizeof(double) * (3 * n + 8))) != GIPC_OK) return s;
    double* base = ctx->slot[D_VEC].as<double>();
    gipc_elements te{sc.tets, T, GIPC_HESS_DENSE, nullptr, nullptr, nullptr};
    gipc_elements se{st_idx, kk, GIPC_HESS_DENSE, nullptr, nullptr, nullptr};
    if (grad) {
        if (!tets_only && xt) mass_times_kernel<<<nbk(3 * n, 256), 256, 0, st>>>(x, xt, sc.mass, n, base);
        te.grad = tg;
        se.grad = sg;
        if ((s = gipc_scatter_elements(ctx, n, kk > 0 ? &se : nullptr, T > 0 ? &te : nullptr,
                                       (!tets_only && xt) ? base : nullptr, grad, st)) != GIPC_OK)
            return s;
    }
    if (Hu) {
        if (!tets_only) mass_times_kernel<<<nbk(3 * n, 256), 256, 0, st>>>(u, nullptr, sc.mass, n, base);
        te.grad = th;
        se.grad = sh;
        if ((s = gipc_scatter_elements(ctx, n, kk > 0 ? &se : nullptr, T > 0 ? &te : nullptr, tets_only ? nullptr : base,
                                       Hu, st)) != GIPC_OK)
            return s;
    }
    if (energy_h) {
        // (1/2 sum m |x - xt|^2 + sum tet energies) + sum stencil energies, each sum in a fixed order
        if ((s = ctx->slot[D_RED].reserve(sizeof(double) * (n + 8))) != GIPC_OK) return s;
        double* r = ctx->slot[D_RED].as<double>();
        double* terms = r + 4;
        const bool inertia = !tets_only && xt;
        if (inertia) {
            inertia_terms_kernel<<<nbk(n, 256), 256, 0, st>>>(x, xt, sc.mass, n, terms);
            dot_kernel<<<1, 1024, 0, st>>>(terms, nullptr, n, r);
        }
        dot_kernel<<<1, 1024, 0, st>>>(eng, nullptr, T, r + 1);
        dot_kernel<<<1, 1024, 0, st>>>(eng + T, nullptr, kk, r + 2);
        double h[3] = {0.0, 0.0, 0.0};
        cudaMemcpyAsync(h, r, 3 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_potential_derivs: energy");
        *energy_h = ((inertia ? 0.5 * h[0] : 0.0) + h[1]) + h[2];
    }
    return check_launch("gipc_potential_derivs");
}


// Exact element Hessians assembled with the mass (FP64 BSR, capacity protocol of the assembly)
gipc_status potential_hessian_impl(gipc_ctx* ctx, const gipc_scene& sc, const double* x, const int32_t* st_idx,
                                   const double* eps_x, int64_t k, const gipc_barrier_params& bp,
                                   const gipc_elastic_params& ep, gipc_bsr* bsr, cudaStream_t st) {
    const int64_t n = sc.n, T = sc.T;
    gipc_status s;
    if ((s = ctx->slot[D_HES].reserve(sizeof(double) * 144 * (T + k + 1))) != GIPC_OK) return s;
    double* th = ctx->slot[D_HES].as<double>();
    double* sh = th + 144 * T;
    const TetConst K = tet_const(ep);
    const StencilConst B{bp.dhat, bp.kappa};
    if (T > 0)
        elem_hessian_kernel<<<nbk(T, 64), 64, 0, st>>>(true, sc.tets, T, x, n, sc.Dm_inv, sc.vol, K, nullptr, B, th);
    if (k > 0) elem_hessian_kernel<<<nbk(k, 64), 64, 0, st>>>(false, st_idx, k, x, n, nullptr, nullptr, K, eps_x, B, sh);
    gipc_elements te{sc.tets, T, GIPC_HESS_DENSE, th, nullptr, nullptr};
    gipc_elements se{st_idx, k, GIPC_HESS_DENSE, sh, nullptr, nullptr};
    return gipc_assemble_bsr(ctx, n, k > 0 ? &se : nullptr, T > 0 ? &te : nullptr, sc.mass, nullptr, bsr, nullptr, st);
}

}  // namespace gipc

namespace {
gipc_status check_scene(const gipc_scene* sc, const char* who) {
    using namespace gipc;
    if (!sc) return fail(GIPC_ERR_INVALID_ARG, "%s: null scene", who);
    if (sc->n <= 0 || sc->T < 0 || !sc->mass || (sc->T > 0 && (!sc->tets || !sc->Dm_inv || !sc->vol)))
        return fail(GIPC_ERR_INVALID_ARG, "%s: incomplete scene", who);
    return GIPC_OK;
}

// The contact list at x (compact, in the D_CON slot, grown once if it was short).
gipc_status contacts_at(gipc_ctx* ctx, const gipc_scene& sc, const double* x, double dhat, cudaStream_t st,
                        int32_t** sti, double** eps, int64_t* k) {
    using namespace gipc;
    gipc_status s;
    if ((s = ctx->slot[D_CON].reserve(sizeof(double) * 4096 * 3)) != GIPC_OK) return s;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const int64_t cap = (int64_t)(ctx->slot[D_CON].bytes / (4 * sizeof(int32_t) + sizeof(double)));
        *eps = ctx->slot[D_CON].as<double>();
        *sti = reinterpret_cast<int32_t*>(*eps + cap);
        s = find_contacts_impl(ctx, x, sc.rest_x, sc.n, sc.surface, dhat, *sti, *eps, cap, k, true, nullptr, nullptr, st,
                               1, false);
        if (s != GIPC_ERR_CAPACITY) return s;
        if ((s = ctx->slot[D_CON].reserve((size_t)(*k + *k / 4 + 1024) * (4 * sizeof(int32_t) + sizeof(double)))) !=
            GIPC_OK)
            return s;
    }
    return fail(GIPC_ERR_CAPACITY, "contact list still short after growing it");
}

// The exact Hessian at x into the D_ROW / D_COL / D_VAL slots (grown once if they were short).
gipc_status exact_hessian(gipc_ctx* ctx, const gipc_scene& sc, const double* x, const int32_t* sti, const double* eps,
                          int64_t k, const gipc_barrier_params& bp, const gipc_elastic_params& ep, gipc_bsr* H,
                          cudaStream_t st) {
    using namespace gipc;
    gipc_status s;
    *H = gipc_bsr{};
    H->prec = GIPC_FP64;
    if ((s = ctx->slot[D_ROW].reserve(sizeof(int32_t) * (sc.n + 1))) != GIPC_OK) return s;
    H->rowptr = ctx->slot[D_ROW].as<int32_t>();
    for (int attempt = 0; attempt < 2; ++attempt) {
        H->capacity = std::min<int64_t>((int64_t)(ctx->slot[D_COL].bytes / sizeof(int32_t)),
                                        (int64_t)(ctx->slot[D_VAL].bytes / (9 * sizeof(double))));
        H->colidx = ctx->slot[D_COL].as<int32_t>();
        H->vals = ctx->slot[D_VAL].ptr;
        s = potential_hessian_impl(ctx, sc, x, sti, eps, k, bp, ep, H, st);
        if (s != GIPC_ERR_CAPACITY || H->nnzb <= H->capacity) return s;
        const int64_t c2 = H->nnzb + H->nnzb / 8 + 1024;
        if ((s = ctx->slot[D_COL].reserve(sizeof(int32_t) * c2)) != GIPC_OK) return s;
        if ((s = ctx->slot[D_VAL].reserve(sizeof(double) * 9 * c2)) != GIPC_OK) return s;
    }
    return fail(GIPC_ERR_CAPACITY, "exact Hessian still short after growing it");
}
}  // namespace

extern "C" gipc_status gipc_potential_derivs(gipc_ctx* ctx, const gipc_scene* sc, const double* x, const double* xt,
                                             const int32_t* stencils, const double* eps_x, int64_t k,
                                             const gipc_barrier_params* bp, const gipc_elastic_params* ep,
                                             const double* u, double* energy_h, double* grad, double* Hu, void* stream) {
    using namespace gipc;
    gipc_status s;
    if (!ctx || !x || !bp || !ep) return fail(GIPC_ERR_INVALID_ARG, "gipc_potential_derivs: null argument");
    if ((s = check_scene(sc, "gipc_potential_derivs")) != GIPC_OK) return s;
    if (k < 0 || (k > 0 && !stencils) || (Hu && !u)) return fail(GIPC_ERR_INVALID_ARG, "gipc_potential_derivs: bad contacts or u");
    if (!(bp->dhat > 0.0) || !(ep->mu > 0.0) || !(ep->lambda > 0.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_potential_derivs: need dhat, mu, lambda > 0");
    return potential_derivs_impl(ctx, *sc, x, xt, stencils, eps_x, k, *bp, *ep, u, energy_h, grad, Hu, false,
                                 (cudaStream_t)stream);
}

extern "C" gipc_status gipc_potential_hessian(gipc_ctx* ctx, const gipc_scene* sc, const double* x,
                                              const int32_t* stencils, const double* eps_x, int64_t k,
                                              const gipc_barrier_params* bp, const gipc_elastic_params* ep, gipc_bsr* bsr,
                                              void* stream) {
    using namespace gipc;
    gipc_status s;
    if (!ctx || !x || !bp || !ep || !bsr) return fail(GIPC_ERR_INVALID_ARG, "gipc_potential_hessian: null argument");
    if ((s = check_scene(sc, "gipc_potential_hessian")) != GIPC_OK) return s;
    if (k < 0 || (k > 0 && !stencils) || bsr->prec != GIPC_FP64)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_potential_hessian: bad contacts or a non-FP64 matrix");
    return potential_hessian_impl(ctx, *sc, x, stencils, eps_x, k, *bp, *ep, bsr, (cudaStream_t)stream);
}

extern "C" gipc_status gipc_adjoint_step(gipc_ctx* ctx, const gipc_scene* sc, const double* x_new, const double* x_old,
                                         const double* v_old, const gipc_step_params* prm, const double* adj_x_new,
                                         const double* adj_v_new, double* adj_x_old, double* adj_v_old,
                                         double* adj_logE_h, int* pcg_iters_h, void* stream) {
    using namespace gipc;
    cudaStream_t st = (cudaStream_t)stream;
    gipc_status s;
    if (!ctx || !x_new || !prm) return fail(GIPC_ERR_INVALID_ARG, "gipc_adjoint_step: null argument");
    if ((s = check_scene(sc, "gipc_adjoint_step")) != GIPC_OK) return s;
    if (!(prm->dt > 0.0) || !(prm->barrier.dhat > 0.0)) return fail(GIPC_ERR_INVALID_ARG, "gipc_adjoint_step: bad parameters");
    (void)x_old;
    (void)v_old;
    const int64_t n = sc->n, m3 = 3 * n;
    // contacts and the exact Hessian at x_new
    int32_t* sti = nullptr;
    double* eps = nullptr;
    int64_t k = 0;
    if ((s = contacts_at(ctx, *sc, x_new, prm->barrier.dhat, st, &sti, &eps, &k)) != GIPC_OK) return s;
    gipc_elastic_params ep = prm->elastic;
    ep.scale = prm->dt * prm->dt;
    gipc_bsr H{};
    if ((s = exact_hessian(ctx, *sc, x_new, sti, eps, k, prm->barrier, ep, &H, st)) != GIPC_OK) return s;
    // H lambda = a
    if ((s = ctx->slot[D_ADJ].reserve(sizeof(double) * (4 * m3 + 8))) != GIPC_OK) return s;
    double* a = ctx->slot[D_ADJ].as<double>();
    double* lam = a + m3;
    double* Hl = lam + m3;
    double* gel = Hl + m3;
    double* red = gel + m3;
    adjoint_rhs_kernel<<<nbk(m3, 256), 256, 0, st>>>(adj_x_new, adj_v_new, sc->fixed, n, prm->dt, a);
    cudaMemsetAsync(lam, 0, sizeof(double) * m3, st);
    gipc_pcg_params pp{prm->pcg_tol, std::max(prm->max_pcg, 1), 0, GIPC_PRODUCT_NATIVE, GIPC_PCG_STOP_ON_INDEFINITE};
    int pit = 0;
    const gipc_status ps = pcg_impl(ctx, &H, a, lam, sc->fixed, &pp, &pit, nullptr, st, nullptr, 1, nullptr, nullptr, nullptr);
    if (pcg_iters_h) *pcg_iters_h = pit;
    if (ps != GIPC_OK && ps != GIPC_ERR_NOT_CONVERGED) return ps;
    // H lambda (fixed rows), then the outputs
    if ((s = potential_derivs_impl(ctx, *sc, x_new, nullptr, sti, eps, k, prm->barrier, ep, lam, nullptr, nullptr, Hl,
                                   false, st)) != GIPC_OK)
        return s;
    adjoint_out_kernel<<<nbk(m3, 256), 256, 0, st>>>(lam, Hl, sc->mass, adj_x_new, adj_v_new, sc->fixed, n, prm->dt,
                                                     adj_x_old, adj_v_old);
    if (adj_logE_h) {
        if ((s = potential_derivs_impl(ctx, *sc, x_new, nullptr, sti, eps, k, prm->barrier, ep, nullptr, nullptr, gel,
                                       nullptr, true, st)) != GIPC_OK)
            return s;
        dot_kernel<<<1, 1024, 0, st>>>(lam, gel, m3, red);
        double h = 0.0;
        cudaMemcpyAsync(&h, red, sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_adjoint_step: sync");
        *adj_logE_h += -h;
    } else if (cudaStreamSynchronize(st) != cudaSuccess) {
        return check_launch("gipc_adjoint_step: sync");
    }
    if (ps == GIPC_ERR_NOT_CONVERGED) return fail(GIPC_ERR_NOT_CONVERGED, "gipc_adjoint_step: the adjoint solve did not converge");
    return check_launch("gipc_adjoint_step");
}

extern "C" gipc_status gipc_newton_polish(gipc_ctx* ctx, const gipc_scene* sc, double* x, double* v, const double* x_old,
                                          const double* v_old, const gipc_step_params* prm, double eps_polish,
                                          int max_iters, int* iters_h, double* step_h, void* stream) {
    using namespace gipc;
    cudaStream_t st = (cudaStream_t)stream;
    gipc_status s;
    if (!ctx || !x || !x_old || !v_old || !prm) return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_polish: null argument");
    if ((s = check_scene(sc, "gipc_newton_polish")) != GIPC_OK) return s;
    if (!(prm->dt > 0.0) || !(prm->barrier.dhat > 0.0) || !(sc->l > 0.0) || !(eps_polish >= 0.0) || max_iters < 0)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_newton_polish: bad parameters");
    const int64_t n = sc->n, m3 = 3 * n;
    const double dt = prm->dt;
    if ((s = ctx->slot[D_POL].reserve(sizeof(double) * (4 * m3 + 8))) != GIPC_OK) return s;
    double* xt = ctx->slot[D_POL].as<double>();
    double* g = xt + m3;
    double* rhs = g + m3;
    double* d = rhs + m3;
    double* red = d + m3;
    step_target_kernel<<<nbk(n, 256), 256, 0, st>>>(x_old, v_old, sc->fixed, n, dt, dt * dt * prm->gravity[0],
                                                    dt * dt * prm->gravity[1], dt * dt * prm->gravity[2], xt);
    gipc_elastic_params ep = prm->elastic;
    ep.scale = dt * dt;
    int it = 0;
    double step = INFINITY;
    bool converged = false;
    for (; it < max_iters && !converged; ++it) {
        int32_t* sti = nullptr;
        double* eps = nullptr;
        int64_t k = 0;
        if ((s = contacts_at(ctx, *sc, x, prm->barrier.dhat, st, &sti, &eps, &k)) != GIPC_OK) return s;
        if ((s = potential_derivs_impl(ctx, *sc, x, xt, sti, eps, k, prm->barrier, ep, nullptr, nullptr, g, nullptr, false,
                                       st)) != GIPC_OK)
            return s;
        gipc_bsr H{};
        if ((s = exact_hessian(ctx, *sc, x, sti, eps, k, prm->barrier, ep, &H, st)) != GIPC_OK) return s;
        neg_free_kernel<<<nbk(m3, 256), 256, 0, st>>>(g, sc->fixed, n, rhs);
        cudaMemsetAsync(d, 0, sizeof(double) * m3, st);
        gipc_pcg_params pp{prm->pcg_tol, std::max(prm->max_pcg, 1), 0, GIPC_PRODUCT_NATIVE, GIPC_PCG_STOP_ON_INDEFINITE};
        const gipc_status ps = pcg_impl(ctx, &H, rhs, d, sc->fixed, &pp, nullptr, nullptr, st, nullptr, 1, nullptr, nullptr, nullptr);
        if (ps != GIPC_OK && ps != GIPC_ERR_NOT_CONVERGED && ps != GIPC_ERR_INDEFINITE) return ps;
        // a Newton direction of the exact Hessian descends only where that Hessian is positive
        // definite: stop (leaving x as it is) when it is not, or when the direction does not descend
        if (ps == GIPC_ERR_INDEFINITE) break;
        dot_kernel<<<1, 1024, 0, st>>>(g, d, m3, red);
        maxabs_kernel<<<1, 1024, 0, st>>>(d, m3, red + 1);
        double h[2] = {0.0, 0.0};
        cudaMemcpyAsync(h, red, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_newton_polish: direction");
        if (!(h[0] < 0.0) && h[1] > 0.0) break;
        step = h[1] / (sc->l * dt);
        if (!(h[1] > 0.0)) {
            converged = true;
            break;
        }
        double alpha = 1.0;
        if ((s = ccd_impl(ctx, x, d, n, sc->surface, 0.1, &alpha, st, nullptr, 1, nullptr, false)) != GIPC_OK) return s;
        step_apply_kernel<<<nbk(m3, 256), 256, 0, st>>>(x, d, std::min(alpha, 1.0), m3);
        converged = alpha >= 1.0 && step <= eps_polish;
    }
    if (v) step_velocity_kernel<<<nbk(m3, 256), 256, 0, st>>>(x, x_old, dt, m3, v);
    if (iters_h) *iters_h = it;
    if (step_h) *step_h = step;
    if ((s = check_launch("gipc_newton_polish")) != GIPC_OK) return s;
    if (!converged) return fail(GIPC_ERR_NOT_CONVERGED, "gipc_newton_polish: step %.3e of l dt after %d iterations", step, it);
    return GIPC_OK;
}
