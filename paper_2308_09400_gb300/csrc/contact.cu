// Contact detection (broad phase + closest-feature classification) and the CCD step filter.
//
// Contact set (Eq. 3 over the pairs of Eq. 4 / Eq. 5): every surface point-triangle pair
// (point not a corner of the triangle) and every surface edge-edge pair (no shared vertex)
// closer than dhat, each classified by the closest features of its constrained minimum into a
// stencil type (Sec. 7.2 encoding); edge-edge pairs with parallel measure c < eps_x use the
// nearly-parallel types (Sec. 6.1).
//
// Broad phase: a uniform grid stored as a spatial hash.  Every target primitive (triangle or
// edge) is inserted into each cell its float64 box (padded by dhat for detection, swept for CCD)
// overlaps; every query (a surface vertex, or an edge i looking for edges j > i) visits the cells
// of its own box.  A pair is taken only in the cell holding the low corner of the intersection of
// the two boxes, so each overlapping pair is met exactly once, whatever the cell size or hash
// collisions.  The cell size is the mean target-box extent, doubled until no box spans more than
// a few hundred cells.  The grid only proposes candidates: the float64 box test and the
// classification decide, written as a fixed sequence of IEEE operations without contraction
// (__d*_rn), so they take exactly the decisions of any implementation of the same formulas.
// Two passes (count, then write at scanned offsets) and a per-query sort by target index give
// a deterministic list: point-triangle pairs ordered by (surface vertex, triangle), then
// edge-edge pairs by (edge i, edge j > i).
//
// Step filter (Alg. 1 "maxFeasibleStepSize"): additive CCD (conservative advancement with
// the common displacement removed) for every pair whose swept float64 boxes overlap; the step
// is min(1, min over pairs), reduced with an order-independent minimum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "context.cuh"
#include "scan.cuh"

namespace gipc {
namespace {

constexpr int kThreads = 128;
constexpr int64_t kMaxCellsPerBox = 512;   // cell-size doubling threshold
// context scratch slots: query counts / sort keys, query offsets, target boxes, scalars, hash
// tables, per-target cell counts, their offsets
enum ContactSlot { C_CNT = 16, C_QOFF = 17, C_BOX = 18, C_MISC = 19, C_GRID = 30, C_TCNT = 31, C_TOFF = 32 };

struct V3 {
    double x, y, z;
};

__device__ __forceinline__ V3 ld3(const double* __restrict__ X, int64_t n, int64_t i) {
    return {X[i], X[n + i], X[2 * n + i]};
}
__device__ __forceinline__ V3 vsub(V3 a, V3 b) { return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y), __dsub_rn(a.z, b.z)}; }
__device__ __forceinline__ double vdot(V3 a, V3 b) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)), __dmul_rn(a.z, b.z));
}
__device__ __forceinline__ V3 vcross(V3 a, V3 b) {
    return {__dsub_rn(__dmul_rn(a.y, b.z), __dmul_rn(a.z, b.y)), __dsub_rn(__dmul_rn(a.z, b.x), __dmul_rn(a.x, b.z)),
            __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x))};
}

// kind 0: interior of the segment, 1: end a, 2: end b
__device__ __forceinline__ int point_segment(V3 p, V3 a, V3 b, double& d2) {
    const V3 ab = vsub(b, a), ap = vsub(p, a);
    const double L = vdot(ab, ab);
    const double t = __ddiv_rn(vdot(ap, ab), L);
    if (t <= 0.0) {
        d2 = vdot(ap, ap);
        return 1;
    }
    if (t >= 1.0) {
        const V3 bp = vsub(p, b);
        d2 = vdot(bp, bp);
        return 2;
    }
    const V3 c = vcross(ap, ab);
    d2 = __ddiv_rn(vdot(c, c), L);
    return 0;
}

// type: 0 PT interior, 1 PE (corners i, j), 2 PP (corner i)
__device__ __forceinline__ int classify_pt(V3 p, V3 t0, V3 t1, V3 t2, double& d2, int& ci, int& cj) {
    const V3 e0 = vsub(t1, t0), e1 = vsub(t2, t0), v = vsub(p, t0);
    const double a = vdot(e0, e0), b = vdot(e0, e1), c = vdot(e1, e1), d = vdot(e0, v), e = vdot(e1, v);
    const double det = __dsub_rn(__dmul_rn(a, c), __dmul_rn(b, b));
    if (det > 0.0) {
        const double s1 = __ddiv_rn(__dsub_rn(__dmul_rn(c, d), __dmul_rn(b, e)), det);
        const double s2 = __ddiv_rn(__dsub_rn(__dmul_rn(a, e), __dmul_rn(b, d)), det);
        if (s1 >= 0.0 && s2 >= 0.0 && __dadd_rn(s1, s2) <= 1.0) {
            const V3 nn = vcross(e0, e1);
            const double vn = vdot(v, nn);
            d2 = __ddiv_rn(__dmul_rn(vn, vn), vdot(nn, nn));
            return 0;
        }
    }
    const V3 T[3] = {t0, t1, t2};
    int best = -1;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int i = k, j = (k + 1) % 3;
        double dd;
        const int kind = point_segment(p, T[i], T[j], dd);
        if (best < 0 || dd < d2) {
            d2 = dd;
            if (kind == 0) {
                best = 1;
                ci = i;
                cj = j;
            } else {
                best = 2;
                ci = kind == 1 ? i : j;
            }
        }
    }
    return best;
}

// type: 0 EE interior, 1 PE (point P, opposite edge E), 2 PP (points P, Q); local indices 0..3
__device__ __forceinline__ int classify_ee(V3 a0, V3 a1, V3 b0, V3 b1, double& d2, int& P, int& Q) {
    const V3 e1 = vsub(a1, a0), e2 = vsub(b1, b0), w = vsub(a0, b0);
    const double a = vdot(e1, e1), b = vdot(e1, e2), c = vdot(e2, e2), d = vdot(e1, w), e = vdot(e2, w);
    const double det = __dsub_rn(__dmul_rn(a, c), __dmul_rn(b, b));
    if (det > __dmul_rn(__dmul_rn(1e-14, a), c)) {
        const double s = __ddiv_rn(__dsub_rn(__dmul_rn(b, e), __dmul_rn(c, d)), det);
        const double t = __ddiv_rn(__dsub_rn(__dmul_rn(a, e), __dmul_rn(b, d)), det);
        if (s > 0.0 && s < 1.0 && t > 0.0 && t < 1.0) {
            const V3 nn = vcross(e1, e2);
            const double wn = vdot(w, nn);
            d2 = __ddiv_rn(__dmul_rn(wn, wn), vdot(nn, nn));
            return 0;
        }
    }
    const V3 X[4] = {a0, a1, b0, b1};
    int best = -1;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int sa = k < 2 ? 2 : 0, sb = sa + 1, E = k < 2 ? 1 : 0;
        double dd;
        const int kind = point_segment(X[k], X[sa], X[sb], dd);
        if (best < 0 || dd < d2) {
            d2 = dd;
            P = k;
            if (kind == 0) {
                best = 1;
                Q = E;
            } else {
                best = 2;
                Q = kind == 1 ? sa : sb;
            }
        }
    }
    return best;
}

__device__ __forceinline__ int32_t neg(int32_t i) { return -(i + 1); }

struct Surf {
    const int32_t* tris;
    int64_t ntri;
    const int32_t* edges;
    int64_t nedge;
    const int32_t* verts;
    int64_t nvert;
};

// ------------------------------------------------------------------------------ grid
struct Grid {
    const double* lo;        // [3][m] target box low corners
    const double* hi;        // [3][m]
    int64_t m;
    const double* inv_h;     // device scalar: 1 / cell size
    uint64_t mask;           // buckets - 1 (power of two)
    const int64_t* boff;     // [buckets + 1] bucket offsets into ent
    const int32_t* ent;      // target ids grouped by bucket
};

__device__ __forceinline__ int64_t cell_of(double v, double inv_h) { return (int64_t)floor(__dmul_rn(v, inv_h)); }

__device__ __forceinline__ uint64_t bucket_of(int64_t cx, int64_t cy, int64_t cz, uint64_t mask) {
    // Teschner et al. (2003) spatial hash of the three cell coordinates, then a splitmix64 finaliser
    uint64_t h = ((uint64_t)cx * 73856093ull) ^ ((uint64_t)cy * 19349663ull) ^ ((uint64_t)cz * 83492791ull);
    h ^= h >> 31;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 29;
    return h & mask;
}

// Box of target t: min / max over its corners (and their swept positions when d is given),
// padded by pad -- the same values as the reference formulas (min and max are exact).
__global__ void target_boxes_kernel(const double* __restrict__ x, const double* __restrict__ d, int64_t n,
                                    const int32_t* __restrict__ prim, int nv, int64_t m, double pad,
                                    double* __restrict__ lo, double* __restrict__ hi, double* __restrict__ ext_sum) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double ext = 0.0;
    if (t < m) {
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            double l = INFINITY, h = -INFINITY;
            for (int a = 0; a < nv; ++a) {
                const int32_t v = prim[a * m + t];
                const double p = x[q * n + v];
                l = fmin(l, p);
                h = fmax(h, p);
                if (d) {
                    const double y = __dadd_rn(p, d[q * n + v]);
                    l = fmin(l, y);
                    h = fmax(h, y);
                }
            }
            l = __dsub_rn(l, pad);
            h = __dadd_rn(h, pad);
            lo[q * m + t] = l;
            hi[q * m + t] = h;
            ext = fmax(ext, __dsub_rn(h, l));
        }
    }
    // block sum of the extents, one atomic per block (the cell size only steers the search)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ext += __shfl_xor_sync(0xffffffffu, ext, o);
    if ((threadIdx.x & 31) == 0 && ext > 0.0) atomicAdd(ext_sum, ext);
}

__global__ void cell_size_kernel(const double* __restrict__ ext_sum, int64_t m, double scale, double* __restrict__ inv_h) {
    double h = m > 0 ? *ext_sum / (double)m : 1.0;
    if (!(h > 0.0) || !isfinite(h)) h = 1.0;
    *inv_h = 1.0 / (h * scale);
}

__device__ __forceinline__ int64_t box_cells(double lx, double ly, double lz, double hx, double hy, double hz,
                                             double ih, int64_t c0[3], int64_t c1[3]) {
    c0[0] = cell_of(lx, ih); c0[1] = cell_of(ly, ih); c0[2] = cell_of(lz, ih);
    c1[0] = cell_of(hx, ih); c1[1] = cell_of(hy, ih); c1[2] = cell_of(hz, ih);
    const int64_t a = c1[0] - c0[0] + 1, b = c1[1] - c0[1] + 1, c = c1[2] - c0[2] + 1;
    // saturate: a box this large asks for a coarser grid (a non-finite box never fits)
    if (!(a >= 1 && b >= 1 && c >= 1) || a > kMaxCellsPerBox || b > kMaxCellsPerBox || c > kMaxCellsPerBox)
        return kMaxCellsPerBox + 1;
    return a * b * c;
}

// Cells per target (int32, saturated) and the largest count over targets and query boxes.
__global__ void cells_count_kernel(const double* __restrict__ lo, const double* __restrict__ hi, int64_t m,
                                   const double* __restrict__ inv_h, int32_t* __restrict__ cnt,
                                   unsigned long long* __restrict__ max_cells) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int64_t c0[3], c1[3];
    const int64_t c = box_cells(lo[t], lo[m + t], lo[2 * m + t], hi[t], hi[m + t], hi[2 * m + t], *inv_h, c0, c1);
    cnt[t] = (int32_t)std::min<int64_t>(c, kMaxCellsPerBox + 1);
    atomicMax(max_cells, (unsigned long long)c);
}

// Swept point boxes of the surface vertices (CCD queries) only report their cell counts.
__global__ void point_cells_kernel(const double* __restrict__ x, const double* __restrict__ d, int64_t n,
                                   const int32_t* __restrict__ verts, int64_t nv, const double* __restrict__ inv_h,
                                   unsigned long long* __restrict__ max_cells) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nv) return;
    const int32_t p = verts[k];
    double l[3], h[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double a = x[q * n + p], b = __dadd_rn(a, d[q * n + p]);
        l[q] = fmin(a, b);
        h[q] = fmax(a, b);
    }
    int64_t c0[3], c1[3];
    atomicMax(max_cells, (unsigned long long)box_cells(l[0], l[1], l[2], h[0], h[1], h[2], *inv_h, c0, c1));
}

// Insert target t into the bucket of each cell its box overlaps, at most once per bucket (two
// cells of one box may hash to the same bucket): with the reference-cell rule of the queries a
// pair is then met exactly once.
template <bool FILL>
__global__ void bucket_kernel(const double* __restrict__ lo, const double* __restrict__ hi, int64_t m,
                              const double* __restrict__ inv_h, uint64_t mask, int32_t* __restrict__ bcnt,
                              const int64_t* __restrict__ boff, int32_t* __restrict__ ent) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int64_t c0[3], c1[3];
    const int64_t nc = box_cells(lo[t], lo[m + t], lo[2 * m + t], hi[t], hi[m + t], hi[2 * m + t], *inv_h, c0, c1);
    if (nc > kMaxCellsPerBox) return;
    const int64_t nx = c1[0] - c0[0] + 1, ny = c1[1] - c0[1] + 1;
    auto bucket_at = [&](int64_t li) {
        return bucket_of(c0[0] + li % nx, c0[1] + (li / nx) % ny, c0[2] + li / (nx * ny), mask);
    };
    for (int64_t li = 0; li < nc; ++li) {
        const uint64_t b = bucket_at(li);
        bool seen = false;
        for (int64_t lj = 0; lj < li && !seen; ++lj) seen = bucket_at(lj) == b;
        if (seen) continue;
        const int32_t slot = atomicAdd(&bcnt[b], 1);
        if (FILL) ent[boff[b] + slot] = (int32_t)t;
    }
}

// Visit every candidate target of the query box [ql, qh] exactly once per overlapping pair:
// f(t) is called for targets whose box overlaps the query box in the float64 test of the
// caller (`overlap`), in the reference cell of the pair.
template <class F>
__device__ __forceinline__ void for_each_candidate(const Grid& G, const double ql[3], const double qh[3], double ih,
                                                   F&& f) {
    int64_t c0[3], c1[3];
    if (box_cells(ql[0], ql[1], ql[2], qh[0], qh[1], qh[2], ih, c0, c1) > kMaxCellsPerBox) return;
    for (int64_t cz = c0[2]; cz <= c1[2]; ++cz)
        for (int64_t cy = c0[1]; cy <= c1[1]; ++cy)
            for (int64_t cx = c0[0]; cx <= c1[0]; ++cx) {
                const uint64_t b = bucket_of(cx, cy, cz, G.mask);
                for (int64_t e = G.boff[b], e1 = G.boff[b + 1]; e < e1; ++e) {
                    const int32_t t = G.ent[e];
                    const double tl[3] = {G.lo[t], G.lo[G.m + t], G.lo[2 * G.m + t]};
                    const double th[3] = {G.hi[t], G.hi[G.m + t], G.hi[2 * G.m + t]};
                    if (!(ql[0] <= th[0] && qh[0] >= tl[0] && ql[1] <= th[1] && qh[1] >= tl[1] && ql[2] <= th[2] &&
                          qh[2] >= tl[2]))
                        continue;
                    // reference cell: the low corner of the intersection
                    if (cell_of(fmax(ql[0], tl[0]), ih) != cx || cell_of(fmax(ql[1], tl[1]), ih) != cy ||
                        cell_of(fmax(ql[2], tl[2]), ih) != cz)
                        continue;
                    f(t);
                }
            }
}

// ------------------------------------------------------------------------------ detection
// Point-triangle queries: PASS 0 counts, PASS 1 writes (unsorted within a query) at off[k].
template <int PASS>
__global__ void __launch_bounds__(kThreads)
pt_query_kernel(const double* __restrict__ x, int64_t n, Surf S, Grid G, double dh2, int32_t* __restrict__ cnt,
                const int64_t* __restrict__ off, int32_t* __restrict__ st, double* __restrict__ eps,
                int32_t* __restrict__ key, int64_t stride) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.nvert) return;
    const int32_t p = S.verts[k];
    const V3 xp = ld3(x, n, p);
    const double q[3] = {xp.x, xp.y, xp.z};
    int32_t c = 0;
    int64_t w = PASS == 1 ? off[k] : 0;
    for_each_candidate(G, q, q, *G.inv_h, [&](int32_t t) {
        const int32_t a = S.tris[t], b = S.tris[S.ntri + t], cc = S.tris[2 * S.ntri + t];
        if (p == a || p == b || p == cc) return;
        double d2;
        int ci = 0, cj = 0;
        const int type = classify_pt(xp, ld3(x, n, a), ld3(x, n, b), ld3(x, n, cc), d2, ci, cj);
        if (!(d2 < dh2)) return;
        if (PASS == 0) {
            ++c;
            return;
        }
        const int32_t T[3] = {a, b, cc};
        int32_t s1, s2, s3;
        if (type == 0) { s1 = a; s2 = b; s3 = cc; }
        else if (type == 1) { s1 = T[ci]; s2 = T[cj]; s3 = GIPC_NULL_INDEX; }
        else { s1 = T[ci]; s2 = GIPC_NULL_INDEX; s3 = GIPC_NULL_INDEX; }
        st[w] = neg(p);
        st[stride + w] = s1;
        st[2 * stride + w] = s2;
        st[3 * stride + w] = s3;
        eps[w] = 0.0;
        key[w] = t;
        ++w;
    });
    if (PASS == 0) cnt[k] = c;
}

template <int PASS>
__global__ void __launch_bounds__(kThreads)
ee_query_kernel(const double* __restrict__ x, const double* __restrict__ rx, int64_t n, Surf S, Grid G, double dh2,
                int32_t* __restrict__ cnt, const int64_t* __restrict__ off, int32_t* __restrict__ st,
                double* __restrict__ eps, int32_t* __restrict__ key, int64_t stride) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.nedge) return;
    const int32_t ia = S.edges[i], ib = S.edges[S.nedge + i];
    const V3 A0 = ld3(x, n, ia), A1 = ld3(x, n, ib);
    const double ql[3] = {G.lo[i], G.lo[G.m + i], G.lo[2 * G.m + i]};
    const double qh[3] = {G.hi[i], G.hi[G.m + i], G.hi[2 * G.m + i]};
    int32_t c = 0;
    int64_t w = PASS == 1 ? off[i] : 0;
    for_each_candidate(G, ql, qh, *G.inv_h, [&](int32_t j) {
        if (j <= i) return;
        const int32_t jb0 = S.edges[j], jb1 = S.edges[S.nedge + j];
        if (jb0 == ia || jb0 == ib || jb1 == ia || jb1 == ib) return;
        const V3 B0 = ld3(x, n, jb0), B1 = ld3(x, n, jb1);
        double d2;
        int P = 0, Q = 0;
        const int type = classify_ee(A0, A1, B0, B1, d2, P, Q);
        if (!(d2 < dh2)) return;
        if (PASS == 0) {
            ++c;
            return;
        }
        // eps_x from rest positions, then the parallel test at the current positions
        const V3 ra = vsub(ld3(rx, n, ib), ld3(rx, n, ia)), rb = vsub(ld3(rx, n, jb1), ld3(rx, n, jb0));
        const double ex = __dmul_rn(__dmul_rn(1e-3, vdot(ra, ra)), vdot(rb, rb));
        const V3 cr = vcross(vsub(A1, A0), vsub(B1, B0));
        const bool par = vdot(cr, cr) < ex;
        const int32_t V[4] = {ia, ib, jb0, jb1};
        const int mate[4] = {1, 0, 3, 2};
        int32_t s0, s1, s2, s3;
        if (type == 0) {
            s0 = V[0]; s1 = par ? neg(V[1]) : V[1]; s2 = V[2]; s3 = V[3];
        } else if (type == 1) {
            const int32_t e0 = Q == 0 ? V[0] : V[2], e1 = Q == 0 ? V[1] : V[3];
            if (par) { s0 = neg(V[P]); s1 = neg(V[mate[P]]); s2 = e0; s3 = neg(e1); }
            else { s0 = neg(V[P]); s1 = e0; s2 = e1; s3 = GIPC_NULL_INDEX; }
        } else {
            if (par) { s0 = neg(V[P]); s1 = neg(V[mate[P]]); s2 = neg(V[Q]); s3 = neg(V[mate[Q]]); }
            else { s0 = neg(V[P]); s1 = V[Q]; s2 = GIPC_NULL_INDEX; s3 = GIPC_NULL_INDEX; }
        }
        st[w] = s0;
        st[stride + w] = s1;
        st[2 * stride + w] = s2;
        st[3 * stride + w] = s3;
        eps[w] = ex;
        key[w] = j;
        ++w;
    });
    if (PASS == 0) cnt[i] = c;
}

// Sort each query's outputs by target index (insertion sort: a query meets few targets).
__global__ void segment_sort_kernel(const int64_t* __restrict__ off, int64_t nq, int32_t* __restrict__ key,
                                    int32_t* __restrict__ st, double* __restrict__ eps, int64_t stride) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nq) return;
    const int64_t b = off[q], e = off[q + 1];
    for (int64_t i = b + 1; i < e; ++i) {
        const int32_t k = key[i];
        const int32_t v0 = st[i], v1 = st[stride + i], v2 = st[2 * stride + i], v3 = st[3 * stride + i];
        const double ev = eps[i];
        int64_t j = i - 1;
        while (j >= b && key[j] > k) {
            key[j + 1] = key[j];
            st[j + 1] = st[j];
            st[stride + j + 1] = st[stride + j];
            st[2 * stride + j + 1] = st[2 * stride + j];
            st[3 * stride + j + 1] = st[3 * stride + j];
            eps[j + 1] = eps[j];
            --j;
        }
        key[j + 1] = k;
        st[j + 1] = v0;
        st[stride + j + 1] = v1;
        st[2 * stride + j + 1] = v2;
        st[3 * stride + j + 1] = v3;
        eps[j + 1] = ev;
    }
}

// ---------------------------------------------------------------------------------- CCD
__device__ __forceinline__ double pair_dist(const V3 (&X)[4], bool pt) {
    double d2;
    int a = 0, b = 0;
    if (pt) classify_pt(X[0], X[1], X[2], X[3], d2, a, b);
    else classify_ee(X[0], X[1], X[2], X[3], d2, a, b);
    return __dsqrt_rn(d2);
}

__device__ double accd(V3 (&X)[4], const V3 (&P)[4], bool pt, double s, int max_iter) {
    const V3 pb = {__dmul_rn(0.25, __dadd_rn(__dadd_rn(__dadd_rn(P[0].x, P[1].x), P[2].x), P[3].x)),
                   __dmul_rn(0.25, __dadd_rn(__dadd_rn(__dadd_rn(P[0].y, P[1].y), P[2].y), P[3].y)),
                   __dmul_rn(0.25, __dadd_rn(__dadd_rn(__dadd_rn(P[0].z, P[1].z), P[2].z), P[3].z))};
    V3 Pc[4];
    double nr[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Pc[i] = vsub(P[i], pb);
        nr[i] = __dsqrt_rn(vdot(Pc[i], Pc[i]));
    }
    const double lp = pt ? __dadd_rn(nr[0], fmax(fmax(nr[1], nr[2]), nr[3]))
                         : __dadd_rn(fmax(nr[0], nr[1]), fmax(nr[2], nr[3]));
    if (lp == 0.0) return 1.0;
    double d = pair_dist(X, pt);
    if (!(d > 0.0)) return 0.0;
    const double g = __dmul_rn(s, d);
    double t = 0.0;
    double tl = __ddiv_rn(__dmul_rn(__dsub_rn(1.0, s), d), lp);
    for (int it = 0; it < max_iter; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
            X[i] = {__dadd_rn(X[i].x, __dmul_rn(tl, Pc[i].x)), __dadd_rn(X[i].y, __dmul_rn(tl, Pc[i].y)),
                    __dadd_rn(X[i].z, __dmul_rn(tl, Pc[i].z))};
        d = pair_dist(X, pt);
        if (t > 0.0 && d < g) break;
        t = __dadd_rn(t, tl);
        if (t > 1.0) return 1.0;
        tl = __ddiv_rn(__dmul_rn(0.9, d), lp);
    }
    return t;
}

__device__ __forceinline__ void atomic_min_pos(unsigned long long* addr, double v) {
    // positive doubles order like their bit patterns
    atomicMin(addr, (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(kThreads)
pt_ccd_kernel(const double* __restrict__ x, const double* __restrict__ dx, int64_t n, Surf S, Grid G, double s,
              int max_iter, unsigned long long* __restrict__ amin) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= S.nvert) return;
    const int32_t p = S.verts[k];
    double ql[3], qh[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const double a = x[q * n + p], b = __dadd_rn(a, dx[q * n + p]);
        ql[q] = fmin(a, b);
        qh[q] = fmax(a, b);
    }
    double best = 1.0;
    for_each_candidate(G, ql, qh, *G.inv_h, [&](int32_t t) {
        const int32_t ids[4] = {p, S.tris[t], S.tris[S.ntri + t], S.tris[2 * S.ntri + t]};
        if (p == ids[1] || p == ids[2] || p == ids[3]) return;
        V3 X[4], P[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            X[a] = ld3(x, n, ids[a]);
            P[a] = ld3(dx, n, ids[a]);
        }
        best = fmin(best, accd(X, P, true, s, max_iter));
    });
    if (best < 1.0) atomic_min_pos(amin, best);
}

__global__ void __launch_bounds__(kThreads)
ee_ccd_kernel(const double* __restrict__ x, const double* __restrict__ dx, int64_t n, Surf S, Grid G, double s,
              int max_iter, unsigned long long* __restrict__ amin) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= S.nedge) return;
    const int32_t ia = S.edges[i], ib = S.edges[S.nedge + i];
    const double ql[3] = {G.lo[i], G.lo[G.m + i], G.lo[2 * G.m + i]};
    const double qh[3] = {G.hi[i], G.hi[G.m + i], G.hi[2 * G.m + i]};
    double best = 1.0;
    for_each_candidate(G, ql, qh, *G.inv_h, [&](int32_t j) {
        if (j <= i) return;
        const int32_t ids[4] = {ia, ib, S.edges[j], S.edges[S.nedge + j]};
        if (ids[2] == ia || ids[2] == ib || ids[3] == ia || ids[3] == ib) return;
        V3 X[4], P[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            X[a] = ld3(x, n, ids[a]);
            P[a] = ld3(dx, n, ids[a]);
        }
        best = fmin(best, accd(X, P, false, s, max_iter));
    });
    if (best < 1.0) atomic_min_pos(amin, best);
}

inline unsigned nblk(int64_t w, int t) { return (unsigned)std::max<int64_t>(1, (w + t - 1) / t); }

// Insert the m primitives (nv vertices each) into a hashed grid over their boxes (x, swept by
// d if given, padded by pad).  Synchronises once per cell-size attempt.
gipc_status build_grid(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const int32_t* prim, int nv,
                       int64_t m, double pad, const gipc_surface* pts, Grid& G, cudaStream_t st) {
    gipc_status s;
    // layout of C_MISC: [0] ext_sum, [1] inv_h, [2] max_cells, [3] amin (CCD)
    if ((s = ctx->slot[C_MISC].reserve(64)) != GIPC_OK) return s;
    double* misc = ctx->slot[C_MISC].as<double>();
    unsigned long long* max_cells = reinterpret_cast<unsigned long long*>(misc + 2);
    if ((s = ctx->slot[C_BOX].reserve(sizeof(double) * 6 * (m + 1))) != GIPC_OK) return s;
    double* lo = ctx->slot[C_BOX].as<double>();
    double* hi = lo + 3 * m;
    if ((s = ctx->slot[C_TCNT].reserve(sizeof(int32_t) * (m + 1))) != GIPC_OK) return s;
    int32_t* cnt = ctx->slot[C_TCNT].as<int32_t>();
    if ((s = ctx->slot[C_TOFF].reserve(sizeof(int64_t) * (m + 2 + scan_scratch_words(m + 1)))) != GIPC_OK) return s;
    int64_t* off = ctx->slot[C_TOFF].as<int64_t>();
    cudaMemsetAsync(misc, 0, sizeof(double), st);
    if (m > 0) target_boxes_kernel<<<nblk(m, 256), 256, 0, st>>>(x, d, n, prim, nv, m, pad, lo, hi, misc);
    int64_t total = 0;
    unsigned long long mc = 0;
    for (double scale = 1.0;; scale *= 2.0) {
        cell_size_kernel<<<1, 1, 0, st>>>(misc, m, scale, misc + 1);
        cudaMemsetAsync(max_cells, 0, sizeof(unsigned long long), st);
        if (m > 0) cells_count_kernel<<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, misc + 1, cnt, max_cells);
        if (pts && pts->nvert > 0)
            point_cells_kernel<<<nblk(pts->nvert, 256), 256, 0, st>>>(x, d, n, pts->verts, pts->nvert, misc + 1, max_cells);
        if (m > 0 && exclusive_scan<int32_t>(cnt, off, m, off + m + 2, st) != cudaSuccess)
            return check_launch("contact grid: scan");
        cudaMemcpyAsync(&mc, max_cells, sizeof(mc), cudaMemcpyDeviceToHost, st);
        if (m > 0) cudaMemcpyAsync(&total, off + m, sizeof(total), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("contact grid: sync");
        if ((int64_t)mc <= kMaxCellsPerBox) break;
        if (scale > 1e12) return fail(GIPC_ERR_NONFINITE, "contact grid: non-finite or unbounded positions");
    }
    uint64_t buckets = 1024;
    while ((int64_t)buckets < 2 * total) buckets <<= 1;
    const size_t grid_bytes = sizeof(int64_t) * (buckets + 2 + scan_scratch_words(buckets + 1)) +
                              sizeof(int32_t) * (buckets + total + 1);
    if ((s = ctx->slot[C_GRID].reserve(grid_bytes)) != GIPC_OK) return s;
    int64_t* boff = ctx->slot[C_GRID].as<int64_t>();
    int64_t* btmp = boff + buckets + 2;
    int32_t* bcnt = reinterpret_cast<int32_t*>(btmp + scan_scratch_words(buckets + 1));
    int32_t* ent = bcnt + buckets;
    cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * buckets, st);
    if (m > 0) bucket_kernel<false><<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, misc + 1, buckets - 1, bcnt, nullptr, nullptr);
    if (exclusive_scan<int32_t>(bcnt, boff, (int64_t)buckets, btmp, st) != cudaSuccess)
        return check_launch("contact grid: bucket scan");
    cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * buckets, st);
    if (m > 0) bucket_kernel<true><<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, misc + 1, buckets - 1, bcnt, boff, ent);
    G = Grid{lo, hi, m, misc + 1, buckets - 1, boff, ent};
    return check_launch("contact grid");
}

}  // namespace

// Internal entry points shared with the time-step driver (newton.cu).
gipc_status find_contacts_impl(gipc_ctx* ctx, const double* x, const double* rest_x, int64_t n, const gipc_surface& srf,
                               double dhat, int32_t* stencils, double* eps_x, int64_t cap, int64_t* count,
                               bool compact, cudaStream_t st) {
    Surf S{srf.tris, srf.ntri, srf.edges, srf.nedge, srf.verts, srf.nvert};
    const double pad = dhat * (1.0 + 1e-9);
    const double dh2 = dhat * dhat;
    const int64_t nq = S.nvert + S.nedge;
    *count = 0;
    if (nq == 0) return GIPC_OK;
    gipc_status s;
    if ((s = ctx->slot[C_CNT].reserve(sizeof(int32_t) * (nq + 1))) != GIPC_OK) return s;
    int32_t* cnt = ctx->slot[C_CNT].as<int32_t>();
    // Count pass: triangle grid + point queries, then edge grid + edge queries.  One scratch set
    // holds one grid at a time, so the triangle grid is built again for its write pass.
    int64_t total = 0;
    Grid Gt{}, Ge{};
    if (S.nvert > 0 && S.ntri > 0) {
        if ((s = build_grid(ctx, x, nullptr, n, S.tris, 3, S.ntri, pad, nullptr, Gt, st)) != GIPC_OK) return s;
        pt_query_kernel<0><<<nblk(S.nvert, kThreads), kThreads, 0, st>>>(x, n, S, Gt, dh2, cnt, nullptr, nullptr, nullptr,
                                                                          nullptr, 0);
    } else if (S.nvert > 0) {
        cudaMemsetAsync(cnt, 0, sizeof(int32_t) * S.nvert, st);
    }
    if (S.nedge > 0) {
        if ((s = build_grid(ctx, x, nullptr, n, S.edges, 2, S.nedge, pad, nullptr, Ge, st)) != GIPC_OK) return s;
        ee_query_kernel<0><<<nblk(S.nedge, kThreads), kThreads, 0, st>>>(x, rest_x, n, S, Ge, dh2, cnt + S.nvert, nullptr,
                                                                          nullptr, nullptr, nullptr, 0);
    }
    // offsets over both kinds (point-triangle pairs first)
    if ((s = ctx->slot[C_QOFF].reserve(sizeof(int64_t) * (nq + 2 + scan_scratch_words(nq + 1)))) != GIPC_OK) return s;
    int64_t* off = ctx->slot[C_QOFF].as<int64_t>();
    if (exclusive_scan<int32_t>(cnt, off, nq, off + nq + 2, st) != cudaSuccess)
        return check_launch("gipc_find_contacts: scan");
    cudaMemcpyAsync(&total, off + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_find_contacts: sync");
    *count = total;
    if (total > cap) return fail(GIPC_ERR_CAPACITY, "gipc_find_contacts: %lld contacts, capacity %lld", (long long)total, (long long)cap);
    if (total == 0) return GIPC_OK;
    // rows of the output are `stride` apart: the caller's capacity, or the count itself (compact)
    const int64_t stride = compact ? total : cap;
    // the counts are consumed: their slot now holds the sort keys
    if ((s = ctx->slot[C_CNT].reserve(sizeof(int32_t) * (total + 1))) != GIPC_OK) return s;
    int32_t* key = ctx->slot[C_CNT].as<int32_t>();
    // write passes: the edge grid is the one currently built; then rebuild the triangle grid
    if (S.nedge > 0)
        ee_query_kernel<1><<<nblk(S.nedge, kThreads), kThreads, 0, st>>>(x, rest_x, n, S, Ge, dh2, nullptr, off + S.nvert,
                                                                          stencils, eps_x, key, stride);
    if (S.nvert > 0 && S.ntri > 0) {
        if ((s = build_grid(ctx, x, nullptr, n, S.tris, 3, S.ntri, pad, nullptr, Gt, st)) != GIPC_OK) return s;
        pt_query_kernel<1><<<nblk(S.nvert, kThreads), kThreads, 0, st>>>(x, n, S, Gt, dh2, nullptr, off, stencils, eps_x,
                                                                          key, stride);
    }
    segment_sort_kernel<<<nblk(nq, 256), 256, 0, st>>>(off, nq, key, stencils, eps_x, stride);
    return check_launch("gipc_find_contacts");
}

gipc_status ccd_impl(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const gipc_surface& srf, double slack,
                     double* alpha, cudaStream_t st) {
    Surf S{srf.tris, srf.ntri, srf.edges, srf.nedge, srf.verts, srf.nvert};
    const int max_iter = 100000;
    gipc_status s;
    if ((s = ctx->slot[C_MISC].reserve(64)) != GIPC_OK) return s;
    unsigned long long* amin = reinterpret_cast<unsigned long long*>(ctx->slot[C_MISC].as<double>() + 3);
    const double one = 1.0;
    cudaMemcpyAsync(amin, &one, sizeof(double), cudaMemcpyHostToDevice, st);
    Grid G{};
    if (S.nvert > 0 && S.ntri > 0) {
        if ((s = build_grid(ctx, x, d, n, S.tris, 3, S.ntri, 0.0, &srf, G, st)) != GIPC_OK) return s;
        pt_ccd_kernel<<<nblk(S.nvert, kThreads), kThreads, 0, st>>>(x, d, n, S, G, slack, max_iter, amin);
    }
    if (S.nedge > 0) {
        if ((s = build_grid(ctx, x, d, n, S.edges, 2, S.nedge, 0.0, nullptr, G, st)) != GIPC_OK) return s;
        ee_ccd_kernel<<<nblk(S.nedge, kThreads), kThreads, 0, st>>>(x, d, n, S, G, slack, max_iter, amin);
    }
    double a = 1.0;
    cudaMemcpyAsync(&a, amin, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_ccd_max_step: sync");
    *alpha = a;
    return check_launch("gipc_ccd_max_step");
}

}  // namespace gipc

extern "C" gipc_status gipc_find_contacts(gipc_ctx* ctx, const double* x, const double* rest_x, int64_t n,
                                          const gipc_surface* srf, double dhat, int32_t* stencils, double* eps_x,
                                          int64_t capacity, int64_t* count_h, void* stream) {
    using namespace gipc;
    if (!ctx || !srf || !count_h) return fail(GIPC_ERR_INVALID_ARG, "gipc_find_contacts: null context, surface or count");
    if (n < 0 || capacity < 0 || srf->ntri < 0 || srf->nedge < 0 || srf->nvert < 0 || !(dhat > 0.0))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_find_contacts: bad sizes or dhat");
    if (!x || !rest_x || (srf->ntri && !srf->tris) || (srf->nedge && !srf->edges) || (srf->nvert && !srf->verts) ||
        (capacity > 0 && (!stencils || !eps_x)))
        return fail(GIPC_ERR_INVALID_ARG, "gipc_find_contacts: null pointer");
    return find_contacts_impl(ctx, x, rest_x, n, *srf, dhat, stencils, eps_x, capacity, count_h, false,
                              (cudaStream_t)stream);
}

extern "C" gipc_status gipc_ccd_max_step(gipc_ctx* ctx, const double* x, const double* d, int64_t n,
                                         const gipc_surface* srf, double slack, double* alpha_h, void* stream) {
    using namespace gipc;
    if (!ctx || !srf || !alpha_h || !x || !d) return fail(GIPC_ERR_INVALID_ARG, "gipc_ccd_max_step: null pointer");
    if (n < 0 || !(slack > 0.0 && slack < 1.0)) return fail(GIPC_ERR_INVALID_ARG, "gipc_ccd_max_step: need 0 < slack < 1");
    return ccd_impl(ctx, x, d, n, *srf, slack, alpha_h, (cudaStream_t)stream);
}
