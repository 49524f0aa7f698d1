// Per-stencil barrier energy, gradient and analytically projected Hessian.
//
// One thread evaluates one contact stencil (paper Alg. 2): it decodes the type
// from the index signs (Sec. 7.2), gathers the stencil's vertices, measures the
// gap function g = (d/dhat)^2 of its distance type (Eq. 4-5, 9-11), evaluates
// the stiffened barrier of Eq. 24 and its g-derivatives, applies the proximal
// filter of Eq. 23, and for the nearly-parallel family the mollifier of Eq. 25
// with the 2x2 eigensystem of Eq. 33-35.  Every projected Hessian is rank one
// in x-space (H = lambda w w^T), so the dense block is an outer product and the
// RANK1 output mode writes (lambda, w) only.
//
// Geometry.  Distances and the parallel measure cancel strongly on contact
// inputs (a point 1e-7 from a unit triangle; edges 1e-7 rad from parallel), so
// the FP64 path forms coordinate differences exactly and carries the cross and
// dot products in double-double (dd.cuh): g and c are correctly rounded.  The
// gradient terms use the envelope-theorem form of the squared-distance
// gradient (the closest-point parameters times the closest-point vector); for
// nearly-parallel edge-edge the closest-point parameters are themselves taken
// in double-double because they are ill-conditioned in the edge directions.
// The mixed-precision path keeps plain float64 geometry (double-double only for
// nearly-parallel edge-edge, whose line-line distance loses ~|v|/(d sin theta)
// relative accuracy in plain float64) and the float64 barrier and log, and
// forms and stores the Hessian block in float32.
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "dd.cuh"

namespace gipc {
namespace {

struct BarrierConst {
    double dhat2_hi, dhat2_lo;  // dhat^2 as an exact double-double
    double inv_dhat2;           // 1 / dhat^2
    double dhat4;               // dhat^4
    double eps_g;               // (d_thr / dhat)^2
    double lam1_thr;            // lambda_1 at g = eps_g (Eq. 23)
    double kappa;
};

__device__ __forceinline__ void sub3(const double* a, const double* b, double* o) {
    o[0] = a[0] - b[0];
    o[1] = a[1] - b[1];
    o[2] = a[2] - b[2];
}
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot3(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ---------------------------------------------------------------------- distance types
// Each writes g = d^2/dhat^2 and dg/dx for the vertices it involves into dg at
// the given slot offsets (in units of coordinates).

// Point p vs the plane of triangle (a, b, c).  r = p - foot, foot barycentrics (b0, b1, b2).
template <bool ACC>
__device__ __forceinline__ void geo_point_plane(const double* p, const double* a, const double* b,
                                                const double* c, const BarrierConst& K, double& g,
                                                double* dg) {
    double v[3], e1[3], e2[3], n[3], vn, nn;
    if (ACC) {
        const dd3 V = dd3_diff(p, a), E1 = dd3_diff(b, a), E2 = dd3_diff(c, a);
        const dd3 N = dd3_cross(E1, E2);
        const dd VN = dd3_dot(V, N), NN = dd3_dot(N, N);
        g = dd_div(dd_div(dd_mul(VN, VN), NN), dd{K.dhat2_hi, K.dhat2_lo}).hi;
        dd3_hi(V, v);
        dd3_hi(E1, e1);
        dd3_hi(E2, e2);
        dd3_hi(N, n);
        vn = VN.hi;
        nn = NN.hi;
    } else {
        sub3(p, a, v);
        sub3(b, a, e1);
        sub3(c, a, e2);
        cross3(e1, e2, n);
        vn = dot3(v, n);
        nn = dot3(n, n);
        g = vn * vn / nn * K.inv_dhat2;
    }
    const double inn = 1.0 / nn;
    const double sc = vn * inn;
    double t[3];
    cross3(v, e2, t);
    const double b1 = dot3(t, n) * inn;
    cross3(e1, v, t);
    const double b2 = dot3(t, n) * inn;
    const double b0 = 1.0 - b1 - b2;
    const double k2 = 2.0 * K.inv_dhat2 * sc;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double r = k2 * n[q];
        dg[q] = r;
        dg[3 + q] = -b0 * r;
        dg[6 + q] = -b1 * r;
        dg[9 + q] = -b2 * r;
    }
}

// Line (a0, a1) vs line (b0, b1).  Writes g, dg (4 slots) and optionally the parallel
// measure c = |(a1-a0) x (b1-b0)|^2 and its gradient.
template <bool ACC, bool ACC_PARAM, bool WANT_C>
__device__ __forceinline__ void geo_line_line(const double* a0, const double* a1, const double* b0,
                                              const double* b1, const BarrierConst& K, double& g,
                                              double* dg, double& c, double* dc) {
    double v[3], e1[3], e2[3], n[3], vn, nn, gam1, gam2;
    if (ACC) {
        const dd3 E1 = dd3_diff(a1, a0), E2 = dd3_diff(b1, b0), V = dd3_diff(b0, a0);
        const dd3 N = dd3_cross(E1, E2);
        const dd VN = dd3_dot(V, N), NN = dd3_dot(N, N);
        g = dd_div(dd_div(dd_mul(VN, VN), NN), dd{K.dhat2_hi, K.dhat2_lo}).hi;
        dd3_hi(V, v);
        dd3_hi(E1, e1);
        dd3_hi(E2, e2);
        dd3_hi(N, n);
        vn = VN.hi;
        nn = NN.hi;
        if (ACC_PARAM) {
            gam1 = dd_div(dd3_dot(dd3_cross(V, E2), N), NN).hi;
            gam2 = dd_div(dd3_dot(dd3_cross(V, E1), N), NN).hi;
        }
    } else {
        sub3(a1, a0, e1);
        sub3(b1, b0, e2);
        sub3(b0, a0, v);
        cross3(e1, e2, n);
        vn = dot3(v, n);
        nn = dot3(n, n);
        g = vn * vn / nn * K.inv_dhat2;
    }
    const double inn = 1.0 / nn;
    if (!(ACC && ACC_PARAM)) {
        double t[3];
        cross3(v, e2, t);
        gam1 = dot3(t, n) * inn;
        cross3(v, e1, t);
        gam2 = dot3(t, n) * inn;
    }
    // r = p1 - p2 = -(vn/nn) n ; d(d^2)/d a0 = 2r(1-gam1), a1: 2r gam1, b0: -2r(1-gam2), b1: -2r gam2
    const double k2 = -2.0 * K.inv_dhat2 * vn * inn;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double r = k2 * n[q];
        dg[q] = (1.0 - gam1) * r;
        dg[3 + q] = gam1 * r;
        dg[6 + q] = -(1.0 - gam2) * r;
        dg[9 + q] = -gam2 * r;
    }
    if (WANT_C) {
        c = nn;
        double t1[3], t2[3];
        cross3(e2, n, t1);  // dc/de1 = 2 e2 x n
        cross3(n, e1, t2);  // dc/de2 = 2 n x e1
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            dc[q] = -2.0 * t1[q];
            dc[3 + q] = 2.0 * t1[q];
            dc[6 + q] = -2.0 * t2[q];
            dc[9 + q] = 2.0 * t2[q];
        }
    }
}

// Point p vs the line (e0, e1): r = (e x (v x e)) / |e|^2 is p minus its foot at parameter t.
template <bool ACC>
__device__ __forceinline__ void geo_point_line(const double* p, const double* e0, const double* e1,
                                               const BarrierConst& K, double& g, double* dgp,
                                               double* dg0, double* dg1) {
    double v[3], e[3], w[3], ee;
    if (ACC) {
        const dd3 V = dd3_diff(p, e0), E = dd3_diff(e1, e0);
        const dd3 W = dd3_cross(V, E);
        const dd WW = dd3_dot(W, W), EE = dd3_dot(E, E);
        g = dd_div(dd_div(WW, EE), dd{K.dhat2_hi, K.dhat2_lo}).hi;
        dd3_hi(V, v);
        dd3_hi(E, e);
        dd3_hi(W, w);
        ee = EE.hi;
    } else {
        sub3(p, e0, v);
        sub3(e1, e0, e);
        cross3(v, e, w);
        ee = dot3(e, e);
        g = dot3(w, w) / ee * K.inv_dhat2;
    }
    const double iee = 1.0 / ee;
    const double t = dot3(v, e) * iee;
    double r[3];
    cross3(e, w, r);
    const double k2 = 2.0 * K.inv_dhat2 * iee;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double rr = k2 * r[q];
        dgp[q] = rr;
        dg0[q] = -(1.0 - t) * rr;
        dg1[q] = -t * rr;
    }
}

template <bool ACC>
__device__ __forceinline__ void geo_point_point(const double* p, const double* q, const BarrierConst& K,
                                                double& g, double* dgp, double* dgq) {
    double r[3];
    if (ACC) {
        const dd3 R = dd3_diff(p, q);
        g = dd_div(dd3_dot(R, R), dd{K.dhat2_hi, K.dhat2_lo}).hi;
        dd3_hi(R, r);
    } else {
        sub3(p, q, r);
        g = dot3(r, r) * K.inv_dhat2;
    }
    const double k2 = 2.0 * K.inv_dhat2;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        dgp[j] = k2 * r[j];
        dgq[j] = -k2 * r[j];
    }
}

// Parallel measure of edges (x0, x1) and (x2, x3) with its gradient (PE/PP nearly parallel).
template <bool ACC>
__device__ __forceinline__ void geo_parallel(const double* x0, const double* x1, const double* x2,
                                             const double* x3, double& c, double* dc) {
    double e1[3], e2[3], w[3];
    if (ACC) {
        const dd3 E1 = dd3_diff(x1, x0), E2 = dd3_diff(x3, x2);
        const dd3 W = dd3_cross(E1, E2);
        c = dd3_dot(W, W).hi;
        dd3_hi(E1, e1);
        dd3_hi(E2, e2);
        dd3_hi(W, w);
    } else {
        sub3(x1, x0, e1);
        sub3(x3, x2, e2);
        cross3(e1, e2, w);
        c = dot3(w, w);
    }
    double t1[3], t2[3];
    cross3(e2, w, t1);
    cross3(w, e1, t2);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        dc[q] = -2.0 * t1[q];
        dc[3 + q] = 2.0 * t1[q];
        dc[6 + q] = -2.0 * t2[q];
        dc[9 + q] = 2.0 * t2[q];
    }
}

// b(g) = dhat^4 (1-g)^2 ln^2 g (Eq. 24) and its first two g-derivatives.
__device__ __forceinline__ void barrier_b(double g, double dhat4, double& b, double& bg, double& bgg) {
    const double L = log(g);
    const double u = 1.0 - g;
    const double ig = 1.0 / g;
    const double uL = u * L;
    b = dhat4 * uL * uL;
    bg = 2.0 * dhat4 * uL * (u * ig - L);
    bgg = 2.0 * dhat4 * ((u * u - u * uL) * ig * ig - 4.0 * uL * ig + L * L);
}

template <typename T>
__device__ __forceinline__ void st_out(T* p, int64_t idx, double v) {
    p[idx] = static_cast<T>(v);
}

// Position of dense entry (a, b) (a, b < 3s) of element e in the dense layouts.
template <int MODE>
__device__ __forceinline__ int64_t dense_at(int a, int b, int n3, int64_t k, int64_t e) {
    if (MODE == GIPC_HESS_BLOCKS) return (e * 16 + (a / 3) * 4 + b / 3) * 9 + (a % 3) * 3 + b % 3;
    return (int64_t)(a * n3 + b) * k + e;
}

// One stencil (paper Alg. 2): decode, gather, gap and barrier, projected eigensystem.  Returns
// false for a malformed stencil (fl = GIPC_FLAG_INVALID, nothing else set).  Otherwise sets the
// energy, the rank-one factors (H = lam_out w w^T), the gradient over the first n3 = 3s entries
// and the flags; entries past n3 stay as the caller initialised them (zero).
template <int PREC>
__device__ __forceinline__ bool eval_one(const double* __restrict__ x, int64_t n, const int32_t* __restrict__ st,
                                         int64_t k, const double* __restrict__ eps_x, const BarrierConst& K, int64_t i,
                                         double& e_out, double& lam_out, double (&w)[12], double (&gr)[12],
                                         uint8_t& fl, int& n3) {
    constexpr bool ACC = (PREC == GIPC_FP64);
    int32_t vid[4];
    const int type = decode_stencil(__ldg(st + i), __ldg(st + k + i), __ldg(st + 2 * k + i),
                                    __ldg(st + 3 * k + i), vid);
    const int s = type >= 0 ? stencil_verts(type) : 0;
    bool ok = type >= 0;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < s && vid[j] >= n) ok = false;
    if (!ok) {
        fl = GIPC_FLAG_INVALID;
        return false;
    }
    double X[4][3];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int64_t vj = j < s ? vid[j] : vid[0];
#pragma unroll
        for (int q = 0; q < 3; ++q) X[j][q] = __ldg(x + q * n + vj);
    }

    double g = 2.0, dg[12], c = 0.0, dc[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        dg[j] = 0.0;
        dc[j] = 0.0;
    }
    const bool par = type >= GIPC_EE_PAR;
    switch (type) {
        case GIPC_PT:
            geo_point_plane<ACC>(X[0], X[1], X[2], X[3], K, g, dg);
            break;
        case GIPC_EE:
            geo_line_line<ACC, false, false>(X[0], X[1], X[2], X[3], K, g, dg, c, dc);
            break;
        case GIPC_EE_PAR:  // ill-conditioned in both precisions: always double-double
            geo_line_line<true, true, true>(X[0], X[1], X[2], X[3], K, g, dg, c, dc);
            break;
        case GIPC_PE:
            geo_point_line<ACC>(X[0], X[1], X[2], K, g, dg, dg + 3, dg + 6);
            break;
        case GIPC_PE_PAR:
            geo_point_line<ACC>(X[0], X[2], X[3], K, g, dg, dg + 6, dg + 9);
            geo_parallel<ACC>(X[0], X[1], X[2], X[3], c, dc);
            break;
        case GIPC_PP:
            geo_point_point<ACC>(X[0], X[1], K, g, dg, dg + 3);
            break;
        default:  // GIPC_PP_PAR
            geo_point_point<ACC>(X[0], X[2], K, g, dg, dg + 6);
            geo_parallel<ACC>(X[0], X[1], X[2], X[3], c, dc);
            break;
    }

    n3 = 3 * s;
    if (g < 1.0) {
        fl = GIPC_FLAG_ACTIVE;
        double b, bg, bgg;
        barrier_b(g, K.dhat4, b, bg, bgg);
        double lam1 = 4.0 * g * bgg + 2.0 * bg;  // Eq. 18
        if (g < K.eps_g) {                        // Eq. 23
            lam1 = K.lam1_thr;
            fl |= GIPC_FLAG_FILTERED;
        }
        const double f = sqrt(g);
        const double h2f = 0.5 / f;
        if (!par) {
            e_out = K.kappa * b;
            lam_out = K.kappa * lam1;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                gr[j] = K.kappa * bg * dg[j];
                w[j] = dg[j] * h2f;  // df/dx
            }
        } else {
            const double ex = eps_x ? __ldg(eps_x + i) : 0.0;
            double e = 1.0, e1 = 0.0, e2 = 0.0;  // e, e', e'' of Eq. 25 at gamma = c
            if (c < ex) {
                const double r = c / ex;
                e = r * (2.0 - r);
                e1 = 2.0 / ex * (1.0 - r);
                e2 = -2.0 / (ex * ex);
                fl |= GIPC_FLAG_MOLLIFIED;
            }
            const double sc = sqrt(c);
            const double lg1 = 2.0 * b * (e1 + 2.0 * c * e2);  // lambda_gamma1
            const double lb1 = e * lam1;                       // lambda_g1 (filtered)
            const double t = e1 * bg * sc * f;                 // Eq. 33
            const double A = lg1 - lb1;
            const double p = sqrt(0.25 * A * A + 16.0 * t * t);
            const double l8 = 0.5 * (lg1 + lb1) + p;           // Eq. 35
            double q0, q1;
            if (p == 0.0) {
                q0 = 0.0;
                q1 = 1.0;
            } else if (A >= 0.0) {
                q0 = A + 2.0 * p;
                q1 = 8.0 * t;
                if (t < 0.0) {
                    q0 = -q0;
                    q1 = -q1;
                }
            } else {
                q0 = 8.0 * t;
                q1 = 2.0 * p - A;
            }
            const double qn = 1.0 / sqrt(q0 * q0 + q1 * q1);
            q0 *= qn;
            q1 *= qn;
            const double hs = sc > 0.0 ? 0.5 / sc : 0.0;  // d sqrt(c) = dc / (2 sqrt(c))
            e_out = K.kappa * e * b;
            lam_out = K.kappa * l8;
#pragma unroll
            for (int j = 0; j < 12; ++j) {
                gr[j] = K.kappa * (e1 * b * dc[j] + e * bg * dg[j]);
                w[j] = q0 * (dc[j] * hs) + q1 * (dg[j] * h2f);
            }
        }
    }
    return true;
}

// Writes the blocks of m staged stencils (element-major 3x3 sub-blocks) with coalesced stores.
// Stencil e of the stage holds t = lam w (12 values) then w (12 values) at e * kStageStride (an
// odd stride, so the lanes' staging writes fall in distinct banks); entry (p, q) of its block is
// t_P w_Q with P = max(p, q), Q = min(p, q) -- the product the per-stencil form computes.  Only
// the sub-block rows and columns below smax (the largest stencil of the warp, in vertices) are
// visited: for each stencil, block rows a < smax are runs of smax * 9 entries at a * 36.  Entries
// outside a stencil's own 3s x 3s block are not written, except that a stored pair that straddles
// the edge of the block writes a zero beside it (pairs are used when the runs have even length).
constexpr int kStageStride = 25;

template <typename HT>
__device__ __forceinline__ HT staged_entry(const HT* stage, const int* n3s, int e, int idx, bool& used) {
    const int b16 = idx / 9, w9 = idx - 9 * b16;
    const int p = 3 * (b16 >> 2) + w9 / 3, q = 3 * (b16 & 3) + w9 % 3;
    const int P = p > q ? p : q, Q = p > q ? q : p;
    const bool in = P < n3s[e];
    used |= in;
    return in ? stage[e * kStageStride + P] * stage[e * kStageStride + 12 + Q] : HT(0);
}

template <typename HT, int SMAX>
__device__ __forceinline__ void write_staged_blocks(HT* out, int m, const HT* stage, const int* n3s, int lane) {
    constexpr int run = SMAX * 9, per = SMAX * run;   // entries per block row, per stencil
    if constexpr ((run & 1) == 0) {
        for (int wd = 2 * lane; wd < m * per; wd += 64) {
            const int e = wd / per, r = wd - e * per, a = r / run;
            const int idx = a * 36 + (r - a * run);
            bool used = false;
            const HT v0 = staged_entry(stage, n3s, e, idx, used);
            const HT v1 = staged_entry(stage, n3s, e, idx + 1, used);
            if (!used) continue;
            HT* dst = out + (int64_t)e * 144 + idx;
            if constexpr (std::is_same<HT, double>::value) *reinterpret_cast<double2*>(dst) = make_double2(v0, v1);
            else *reinterpret_cast<float2*>(dst) = make_float2(v0, v1);
        }
    } else {
        for (int wd = lane; wd < m * per; wd += 32) {
            const int e = wd / per, r = wd - e * per, a = r / run;
            const int idx = a * 36 + (r - a * run);
            bool used = false;
            const HT v = staged_entry(stage, n3s, e, idx, used);
            if (used) out[(int64_t)e * 144 + idx] = v;
        }
    }
}

constexpr int kEvalThreads = 128;

template <int PREC, int MODE>
__global__ void __launch_bounds__(kEvalThreads)
eval_stencils_kernel(const double* __restrict__ x, int64_t n, const int32_t* __restrict__ st, int64_t k,
                     const double* __restrict__ eps_x, const BarrierConst K, double* __restrict__ energy,
                     double* __restrict__ grad, void* __restrict__ hess_v, double* __restrict__ lam,
                     uint8_t* __restrict__ flags, const int32_t* __restrict__ order) {
    using HT = typename std::conditional<PREC == GIPC_FP64, double, float>::type;
    HT* __restrict__ hess = static_cast<HT*>(hess_v);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    constexpr bool kCoop = (MODE == GIPC_HESS_BLOCKS);
    if (!kCoop && tid >= k) return;   // (the element-major output is written by whole warps)
    const bool live = tid < k;
    // thread tid evaluates stencil order[tid] (stencils grouped by type, so that a warp runs one
    // type's branch) and writes its outputs at that stencil's own index
    const int64_t i = (!kCoop && order) ? (int64_t)order[tid] : tid;

    double e_out = 0.0, lam_out = 0.0, w[12], gr[12];
    uint8_t fl = 0;
    int n3 = 0;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        w[j] = 0.0;
        gr[j] = 0.0;
    }
    const bool valid = live && eval_one<PREC>(x, n, st, k, eps_x, K, i, e_out, lam_out, w, gr, fl, n3);
    if (live && !valid) {
        if (energy) energy[i] = 0.0;
        if (lam) lam[i] = 0.0;
        if (flags) flags[i] = GIPC_FLAG_INVALID;
        if (!kCoop) return;
    }
    if (valid) {
        if (energy) energy[i] = e_out;
        if (flags) flags[i] = fl;
        if (grad) {
#pragma unroll
            for (int j = 0; j < 12; ++j)
                if (j < n3) grad[j * k + i] = gr[j];
        }
        if (MODE == GIPC_HESS_RANK1) {
            if (lam) lam[i] = lam_out;
            if (hess) {
#pragma unroll
                for (int j = 0; j < 12; ++j)
                    if (j < n3) st_out(hess, j * k + i, w[j]);
            }
        } else if (hess && !kCoop) {
            if (PREC == GIPC_FP64) {
#pragma unroll
                for (int a = 0; a < 12; ++a) {
                    if (a < n3) {
                        const double ta = lam_out * w[a];
#pragma unroll
                        for (int bcol = 0; bcol <= a; ++bcol) {
                            const double h = ta * w[bcol];
                            hess[dense_at<MODE>(a, bcol, n3, k, i)] = h;
                            if (bcol != a) hess[dense_at<MODE>(bcol, a, n3, k, i)] = h;
                        }
                    }
                }
            } else {
                float wf[12];
#pragma unroll
                for (int j = 0; j < 12; ++j) wf[j] = (float)w[j];
                const float lf = (float)lam_out;
#pragma unroll
                for (int a = 0; a < 12; ++a) {
                    if (a < n3) {
                        const float ta = lf * wf[a];
#pragma unroll
                        for (int bcol = 0; bcol <= a; ++bcol) {
                            const float h = ta * wf[bcol];
                            hess[dense_at<MODE>(a, bcol, n3, k, i)] = h;
                            if (bcol != a) hess[dense_at<MODE>(bcol, a, n3, k, i)] = h;
                        }
                    }
                }
            }
        }

    }
    if constexpr (kCoop) {
        // element-major 3x3 sub-blocks: stage each stencil's rank-one factors, then one coalesced
        // run of the warp's 32 blocks
        __shared__ HT stage[kEvalThreads / 32][32 * kStageStride];
        __shared__ int stage_n3[kEvalThreads / 32][32];
        if (!hess) return;   // (uniform)
        const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
        const HT lf = (HT)lam_out;
        HT* my = &stage[wi][lane * kStageStride];
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            const HT wj = (HT)w[j];
            my[j] = lf * wj;
            my[12 + j] = wj;
        }
        stage_n3[wi][lane] = valid ? n3 : 0;
        const int smax = (int)__reduce_max_sync(0xffffffffu, (unsigned)(valid ? n3 : 0)) / 3;
        __syncwarp();
        const int64_t e0 = i - lane;
        const int64_t m = k - e0 < 32 ? k - e0 : 32;
        if (m > 0) {
            HT* out = hess + e0 * 144;
            if (smax == 4) write_staged_blocks<HT, 4>(out, (int)m, stage[wi], stage_n3[wi], lane);
            else if (smax == 3) write_staged_blocks<HT, 3>(out, (int)m, stage[wi], stage_n3[wi], lane);
            else if (smax == 2) write_staged_blocks<HT, 2>(out, (int)m, stage[wi], stage_n3[wi], lane);
        }
    }
}

// Stencils grouped by type: counts[t] (t = 0..6, 7 for a malformed tuple) then, per type, the
// stencil indices in order[counts[0] + ... + counts[t-1] ...].  The order within a type is
// arbitrary (one atomic per type present in a warp); the evaluation writes every output at the
// stencil's own index, so it changes no result.
__device__ __forceinline__ int stencil_kind(const int32_t* __restrict__ st, int64_t k, int64_t i) {
    int32_t v[4];
    const int t = decode_stencil(st[i], st[k + i], st[2 * k + i], st[3 * k + i], v);
    return t < 0 || t > 6 ? 7 : t;
}
__global__ void type_count_kernel(const int32_t* __restrict__ st, int64_t k, unsigned* __restrict__ counts) {
    __shared__ unsigned c[8];
    if (threadIdx.x < 8) c[threadIdx.x] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&c[stencil_kind(st, k, i)], 1u);
    __syncthreads();
    if (threadIdx.x < 8 && c[threadIdx.x]) atomicAdd(&counts[threadIdx.x], c[threadIdx.x]);
}
// counts: [0, 8) the type counts, [8, 16) zeroed cursors.  Launched with whole warps.
__global__ void type_scatter_kernel(const int32_t* __restrict__ st, int64_t k, unsigned* __restrict__ counts,
                                    int32_t* __restrict__ order) {
    __shared__ unsigned off[8];
    if (threadIdx.x == 0) {
        unsigned a = 0;
        for (int t = 0; t < 8; ++t) {
            off[t] = a;
            a += counts[t];
        }
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int t = i < k ? stencil_kind(st, k, i) : 8;
    const unsigned grp = __match_any_sync(0xffffffffu, t);
    const int leader = __ffs(grp) - 1;
    unsigned base = 0;
    if (t < 8 && lane == leader) base = atomicAdd(&counts[8 + t], (unsigned)__popc(grp));
    base = __shfl_sync(grp, base, leader);
    if (t < 8) order[off[t] + base + __popc(grp & ((1u << lane) - 1u))] = (int32_t)i;
}

// eps_x = 1e-3 |x1-x0|^2 |x3-x2|^2 from rest positions, evaluated left to right without
// contraction so the value is the plain IEEE float64 result of that expression.
__global__ void eps_x_kernel(const double* __restrict__ x, int64_t n, const int32_t* __restrict__ st,
                             int64_t k, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= k) return;
    int32_t v[4];
    const int type = decode_stencil(st[i], st[k + i], st[2 * k + i], st[3 * k + i], v);
    double r = 0.0;
    if ((type == GIPC_EE || type >= GIPC_EE_PAR) && v[0] < n && v[1] < n && v[2] < n && v[3] < n) {
        double a[3], b[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            a[q] = __dsub_rn(x[q * n + v[1]], x[q * n + v[0]]);
            b[q] = __dsub_rn(x[q * n + v[3]], x[q * n + v[2]]);
        }
        const double aa = __dadd_rn(__dadd_rn(__dmul_rn(a[0], a[0]), __dmul_rn(a[1], a[1])), __dmul_rn(a[2], a[2]));
        const double bb = __dadd_rn(__dadd_rn(__dmul_rn(b[0], b[0]), __dmul_rn(b[1], b[1])), __dmul_rn(b[2], b[2]));
        r = __dmul_rn(__dmul_rn(1e-3, aa), bb);
    }
    out[i] = r;
}

// lambda_1 = 4 g b_gg + 2 b_g of Eq. 24's barrier on the host (for the filter constant).
double host_lambda1(double g, double dhat4) {
    const double L = std::log(g), u = 1.0 - g, ig = 1.0 / g, uL = u * L;
    const double bg = 2.0 * dhat4 * uL * (u * ig - L);
    const double bgg = 2.0 * dhat4 * ((u * u - u * uL) * ig * ig - 4.0 * uL * ig + L * L);
    return 4.0 * g * bgg + 2.0 * bg;
}

inline unsigned grid_for(int64_t k, int threads) { return (unsigned)((k + threads - 1) / threads); }

}  // namespace
}  // namespace gipc

extern "C" gipc_status gipc_compute_eps_x(const double* rest_x, int64_t n, const int32_t* stencils,
                                          int64_t k, double* eps_x_out, void* stream) {
    using namespace gipc;
    if (n < 0 || k < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_compute_eps_x: negative size");
    if (k == 0) return GIPC_OK;
    if (!rest_x || !stencils || !eps_x_out)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_compute_eps_x: null pointer");
    eps_x_kernel<<<grid_for(k, 256), 256, 0, (cudaStream_t)stream>>>(rest_x, n, stencils, k, eps_x_out);
    return check_launch("gipc_compute_eps_x");
}

namespace gipc {

// The stencils' type grouping for eval_stencils_ordered: order [k], counts [16] device scratch.
gipc_status stencil_type_order(const int32_t* stencils, int64_t k, int32_t* order, unsigned* counts, cudaStream_t s) {
    if (k <= 0) return GIPC_OK;
    cudaMemsetAsync(counts, 0, 16 * sizeof(unsigned), s);
    type_count_kernel<<<std::min<unsigned>(grid_for(k, 256), 1024u), 256, 0, s>>>(stencils, k, counts);
    type_scatter_kernel<<<grid_for(k, 256), 256, 0, s>>>(stencils, k, counts, order);
    return check_launch("stencil type order");
}

// gipc_eval_stencils with thread t evaluating stencil order[t] (null: t) -- the same outputs.
gipc_status eval_stencils_ordered(const double* x, int64_t n, const int32_t* stencils, int64_t k,
                                  const double* eps_x, const gipc_barrier_params* prm, int prec, int mode,
                                  double* energy, double* grad, void* hess, double* lam, uint8_t* flags,
                                  const int32_t* order, cudaStream_t s) {
    if (n < 0 || k < 0) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: negative size");
    if (!prm) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: null parameters");
    if (!(prm->dhat > 0.0) || !(prm->kappa >= 0.0) || !(prm->d_thr_ratio > 0.0 && prm->d_thr_ratio < 1.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: need dhat > 0, kappa >= 0, 0 < d_thr_ratio < 1");
    if (prec != GIPC_FP64 && prec != GIPC_MIXED)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: unknown precision %d", prec);
    if (mode != GIPC_HESS_DENSE && mode != GIPC_HESS_RANK1 && mode != GIPC_HESS_BLOCKS)
        return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: unknown Hessian mode %d", mode);
    if (k == 0) return GIPC_OK;
    if (!x || !stencils) return fail(GIPC_ERR_INVALID_ARG, "gipc_eval_stencils: null x or stencils");

    BarrierConst K;
    const double d = prm->dhat;
    K.dhat2_hi = d * d;
    K.dhat2_lo = std::fma(d, d, -K.dhat2_hi);
    K.inv_dhat2 = 1.0 / K.dhat2_hi;
    K.dhat4 = K.dhat2_hi * K.dhat2_hi;
    K.eps_g = prm->d_thr_ratio * prm->d_thr_ratio;
    K.lam1_thr = host_lambda1(K.eps_g, K.dhat4);
    K.kappa = prm->kappa;

    const unsigned blocks = grid_for(k, kEvalThreads);
    if (mode == GIPC_HESS_BLOCKS) order = nullptr;   // (its output is written by whole warps in place)
#define GIPC_LAUNCH(P, M) \
    eval_stencils_kernel<P, M><<<blocks, kEvalThreads, 0, s>>>(x, n, stencils, k, eps_x, K, energy, grad, hess, lam, \
                                                               flags, order)
    if (prec == GIPC_FP64 && mode == GIPC_HESS_DENSE) GIPC_LAUNCH(GIPC_FP64, GIPC_HESS_DENSE);
    else if (prec == GIPC_FP64 && mode == GIPC_HESS_BLOCKS) GIPC_LAUNCH(GIPC_FP64, GIPC_HESS_BLOCKS);
    else if (prec == GIPC_FP64) GIPC_LAUNCH(GIPC_FP64, GIPC_HESS_RANK1);
    else if (mode == GIPC_HESS_DENSE) GIPC_LAUNCH(GIPC_MIXED, GIPC_HESS_DENSE);
    else if (mode == GIPC_HESS_BLOCKS) GIPC_LAUNCH(GIPC_MIXED, GIPC_HESS_BLOCKS);
    else GIPC_LAUNCH(GIPC_MIXED, GIPC_HESS_RANK1);
#undef GIPC_LAUNCH
    return check_launch("gipc_eval_stencils");
}

}  // namespace gipc

extern "C" gipc_status gipc_eval_stencils(const double* x, int64_t n, const int32_t* stencils, int64_t k,
                                          const double* eps_x, const gipc_barrier_params* prm, int prec,
                                          int mode, double* energy, double* grad, void* hess, double* lam,
                                          uint8_t* flags, void* stream) {
    return gipc::eval_stencils_ordered(x, n, stencils, k, eps_x, prm, prec, mode, energy, grad, hess, lam, flags,
                                       nullptr, (cudaStream_t)stream);
}
