// Contact detection (broad phase + closest-feature classification) and the CCD step filter.
//
// Contact set (Eq. 3 over the pairs of Eq. 4 / Eq. 5): every surface point-triangle pair
// (point not a corner of the triangle) and every surface edge-edge pair (no shared vertex)
// closer than dhat, each classified by the closest features of its constrained minimum into a
// stencil type (Sec. 7.2 encoding); edge-edge pairs with parallel measure c < eps_x use the
// nearly-parallel types (Sec. 6.1).
//
// Broad phase: a uniform grid stored as a spatial hash.  Every target primitive (triangle or
// edge) is inserted into each cell its box (padded by dhat for detection, swept for CCD), rounded
// outward to float32, overlaps (at most once per hash bucket), as a 32-byte entry holding its id
// and that float32 box.  One warp serves one query (a surface vertex, or an edge i looking for
// edges j > i): it walks the cells of the query's float32 box and scans each bucket 32 entries at
// a time with coalesced loads, testing the float32 boxes.  A pair is taken only in the cell
// holding the low corner of the intersection of the two boxes; targets, queries and this rule
// compute cells with the same float32 expression, so each overlapping pair is met exactly once,
// whatever the cell size or hash collisions.  The cell size is the mean target-box extent,
// doubled until no box spans more than a few hundred cells.  The grid only proposes candidates
// (every pair whose float64 boxes overlap, and a few whose float32 boxes alone do): the
// classification decides contacts, and for the CCD the float64 swept-box test picks the pairs
// whose step is evaluated, both written as fixed sequences of IEEE operations without
// contraction (__d*_rn), so they take exactly the decisions of any implementation of the same
// formulas.  Two passes (count, then write at scanned
// offsets) and a per-query sort by target index give a deterministic list: point-triangle pairs
// ordered by (surface vertex, triangle), then edge-edge pairs by (edge i, edge j > i).
//
// Step filter (Alg. 1 "maxFeasibleStepSize"): additive CCD (conservative advancement with
// the common displacement removed) for every pair whose swept float64 boxes overlap; the step
// is min(1, min over pairs), reduced with an order-independent minimum.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <cmath>

#include "common.cuh"
#include "context.cuh"
#include "scan.cuh"

namespace gipc {
namespace {

constexpr int kThreads = 128;
constexpr int64_t kMaxCellsPerBox = 64;    // cell-size doubling threshold (cells per box)
constexpr int kWarps = kThreads / 32;
// context scratch slots: query counts (then cursors), query offsets, scalars, sort keys, candidate
// pairs, pair codes; per grid (triangles,
// edges): float64 target boxes, hash tables, per-target cell counts and their offsets
enum ContactSlot { C_CNT = 16, C_QOFF = 17, C_MISC = 19, C_KEY = 37, C_PAIRS = 38, C_CODE = 39, C_CPAIRS = 59, C_CX = 60,
                   C_X32 = 63, C_LIST = 64 };
constexpr int kGridSlots[2][5] = {{18, 30, 31, 32, 45}, {33, 34, 35, 36, 46}};
// scalars in C_MISC: per grid g the largest cell count at 4g + 2; CCD minimum at 8, pair counter
// at 9.  Per-scene extent sums, counts and inverse cell sizes live in the grid's last slot.
constexpr int kMiscAmin = 8;
constexpr int kMiscPairs = 9;
constexpr int kMiscDisp = 10;   // cached candidates: max |x - x_b| at 10, max |d| at 11 (bit patterns)
constexpr int kMiscList = 12;   // length of the prefilter's list (unsigned)

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
// Bucket entry: target id and its box rounded outward to float32 (two 16-byte halves).
struct __align__(16) Entry {
    float lx, ly, lz;
    int32_t id;
    float hx, hy, hz;
    int32_t scene;   // scene of the target (batched scenes never pair across scenes)
};

struct Grid {
    const double* lo;        // [3][m] target box low corners (float64)
    const double* hi;        // [3][m]
    int64_t m;
    const double* inv_h;     // device [scenes]: 1 / cell size of each scene
    uint64_t mask;           // buckets - 1 (power of two)
    const int64_t* boff;     // [buckets + 1] bucket offsets into ent
    const Entry* ent;        // entries grouped by bucket
};


__device__ __forceinline__ uint64_t bucket_of(int64_t cx, int64_t cy, int64_t cz, int32_t scene, uint64_t mask) {
    // Teschner et al. (2003) spatial hash of the three cell coordinates and the scene, then a
    // splitmix64 finaliser
    uint64_t h = ((uint64_t)cx * 73856093ull) ^ ((uint64_t)cy * 19349663ull) ^ ((uint64_t)cz * 83492791ull) ^
                 ((uint64_t)(uint32_t)scene * 2654435761ull);
    h ^= h >> 31;
    h *= 0xbf58476d1ce4e5b9ull;
    h ^= h >> 29;
    return h & mask;
}

// Box of target t: min / max over its corners (and their swept positions when d is given),
// padded by pad -- the same values as the reference formulas (min and max are exact).
__global__ void target_boxes_kernel(const double* __restrict__ x, const double* __restrict__ d, int64_t n,
                                    const int32_t* __restrict__ prim, int nv, int64_t m, double pad,
                                    const int32_t* __restrict__ vscene, double* __restrict__ lo, double* __restrict__ hi,
                                    double* __restrict__ ext_sum, double* __restrict__ ext_cnt) {
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
    // extent sums per scene (the cell size only steers the search): one scene -> one atomic per
    // warp; batched scenes -> one per target
    if (vscene) {   // the lists are ordered by scene: a warp whose targets share one scene adds once
        const int32_t sc = t < m ? vscene[prim[t]] : -1;
        const unsigned same = __match_any_sync(0xffffffffu, sc);
        if (same == 0xffffffffu && sc >= 0) {
            double c = 1.0, ex = ext;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ex += __shfl_xor_sync(0xffffffffu, ex, o);
                c += __shfl_xor_sync(0xffffffffu, c, o);
            }
            if ((threadIdx.x & 31) == 0) {
                atomicAdd(ext_sum + sc, ex);
                atomicAdd(ext_cnt + sc, c);
            }
        } else if (sc >= 0) {
            atomicAdd(ext_sum + sc, ext);
            atomicAdd(ext_cnt + sc, 1.0);
        }
        return;
    }
    double c = t < m ? 1.0 : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ext += __shfl_xor_sync(0xffffffffu, ext, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0 && c > 0.0) {
        atomicAdd(ext_sum, ext);
        atomicAdd(ext_cnt, c);
    }
}

// Cell size of each scene: the mean extent of its target boxes, times `scale`.
__global__ void cell_size_kernel(const double* __restrict__ ext_sum, const double* __restrict__ ext_cnt, int ns,
                                 double scale, double* __restrict__ inv_h) {
    const int sc = blockIdx.x * blockDim.x + threadIdx.x;
    if (sc >= ns) return;
    double h = ext_cnt[sc] > 0.0 ? ext_sum[sc] / ext_cnt[sc] : 1.0;
    if (!(h > 0.0) || !isfinite(h)) h = 1.0;
    inv_h[sc] = 1.0 / (h * scale);
}

// Grid cells in float32 (see the header): the cell of a float32 box bound v is floor(v ih) with
// ih the float32 inverse cell size, clamped to +-2^30.
__device__ __forceinline__ int cell32(float v, float ih) {
    return (int)fminf(fmaxf(floorf(v * ih), -1073741824.f), 1073741824.f);
}
__device__ __forceinline__ void box32(const double* l, const double* h, float* fl, float* fh) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        fl[q] = __double2float_rd(l[q]);
        fh[q] = __double2float_ru(h[q]);
    }
}
__device__ __forceinline__ int64_t box_cells(const float* fl, const float* fh, float ih, int c0[3], int c1[3]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        if (!(isfinite(fl[q]) && isfinite(fh[q]))) return kMaxCellsPerBox + 1;   // never fits
        c0[q] = cell32(fl[q], ih);
        c1[q] = cell32(fh[q], ih);
    }
    const int64_t a = (int64_t)c1[0] - c0[0] + 1, b = (int64_t)c1[1] - c0[1] + 1, c = (int64_t)c1[2] - c0[2] + 1;
    // saturate: a box this large asks for a coarser grid
    if (!(a >= 1 && b >= 1 && c >= 1) || a > kMaxCellsPerBox || b > kMaxCellsPerBox || c > kMaxCellsPerBox)
        return kMaxCellsPerBox + 1;
    return a * b * c;
}

// Cells per target (int32, saturated) and the largest count over the targets.
__global__ void cells_count_kernel(const double* __restrict__ lo, const double* __restrict__ hi, int64_t m,
                                   const int32_t* __restrict__ prim, const int32_t* __restrict__ vscene,
                                   const double* __restrict__ inv_h, int32_t* __restrict__ cnt,
                                   unsigned long long* __restrict__ max_cells) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    int c0[3], c1[3];
    const float ih = (float)inv_h[vscene ? vscene[prim[t]] : 0];
    const double l[3] = {lo[t], lo[m + t], lo[2 * m + t]}, h[3] = {hi[t], hi[m + t], hi[2 * m + t]};
    float fl[3], fh[3];
    box32(l, h, fl, fh);
    const int64_t c = box_cells(fl, fh, ih, c0, c1);
    cnt[t] = (int32_t)std::min<int64_t>(c, kMaxCellsPerBox + 1);
    // one atomic per warp (counts are at most kMaxCellsPerBox + 1 after the saturation above)
    const unsigned active = __activemask();
    const unsigned wmax = __reduce_max_sync(active, (unsigned)std::min<int64_t>(c, kMaxCellsPerBox + 1));
    if ((threadIdx.x & 31) == __ffs(active) - 1) atomicMax(max_cells, (unsigned long long)wmax);
}

// Swept point boxes of the surface vertices (CCD queries) only report their cell counts.
__global__ void point_cells_kernel(const double* __restrict__ x, const double* __restrict__ d, int64_t n,
                                   const int32_t* __restrict__ verts, int64_t nv, const int32_t* __restrict__ vscene,
                                   const double* __restrict__ inv_h, unsigned long long* __restrict__ max_cells) {
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
    int c0[3], c1[3];
    float fl[3], fh[3];
    box32(l, h, fl, fh);
    const float ih = (float)inv_h[vscene ? vscene[p] : 0];
    const unsigned active = __activemask();
    const unsigned wmax = __reduce_max_sync(active, (unsigned)box_cells(fl, fh, ih, c0, c1));
    if ((threadIdx.x & 31) == __ffs(active) - 1) atomicMax(max_cells, (unsigned long long)wmax);
}

// Insert target t into the bucket of each cell its box overlaps, at most once per bucket (two
// cells of one box may hash to the same bucket): with the reference-cell rule of the queries a
// pair is then met exactly once.
template <bool FILL>
__global__ void bucket_kernel(const double* __restrict__ lo, const double* __restrict__ hi, int64_t m,
                              const int32_t* __restrict__ prim, const int32_t* __restrict__ vscene,
                              const double* __restrict__ inv_h, uint64_t mask, int32_t* __restrict__ bcnt,
                              const int64_t* __restrict__ boff, Entry* __restrict__ ent) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    const int32_t scene = vscene ? vscene[prim[t]] : 0;
    const double l[3] = {lo[t], lo[m + t], lo[2 * m + t]}, h[3] = {hi[t], hi[m + t], hi[2 * m + t]};
    float fl[3], fh[3];
    box32(l, h, fl, fh);
    int c0[3], c1[3];
    const int64_t nc = box_cells(fl, fh, (float)inv_h[scene], c0, c1);
    if (nc > kMaxCellsPerBox) return;
    const int64_t nx = c1[0] - c0[0] + 1, ny = c1[1] - c0[1] + 1;
    auto bucket_at = [&](int64_t li) {
        return bucket_of(c0[0] + li % nx, c0[1] + (li / nx) % ny, c0[2] + li / (nx * ny), scene, mask);
    };
    Entry E;
    if (FILL) {
        E.lx = fl[0]; E.ly = fl[1]; E.lz = fl[2];
        E.hx = fh[0]; E.hy = fh[1]; E.hz = fh[2];
        E.id = (int32_t)t;
        E.scene = scene;
    }
    for (int64_t li = 0; li < nc; ++li) {
        const uint64_t b = bucket_at(li);
        bool seen = false;
        for (int64_t lj = 0; lj < li && !seen; ++lj) seen = bucket_at(lj) == b;
        if (seen) continue;
        const int32_t slot = atomicAdd(&bcnt[b], 1);
        if (FILL) ent[boff[b] + slot] = E;
    }
}

// Candidate pairs.  Each warp takes queries q = warp, warp + nw, ... and walks the cells of the
// query box (the same box in every lane); each round every lane tests one bucket entry: the
// float32 boxes, whether this cell is the pair's reference cell (the low corner of the
// intersection of the two boxes) and the kind's index filters.  Survivors are queued in shared
// memory (64 per warp) and appended to the global pair list 32 at a time with one atomic.  The
// list order is arbitrary; the pair SET is fixed by the float32 boxes.
enum PairKind { K_PT = 0, K_EE = 1, K_PT_SWEPT = 2 };

struct PairList {
    int32_t* q;                  // [cap] query index (surface-vertex position, or edge id)
    int32_t* t;                  // [cap] target index (triangle or edge id)
    int64_t cap;
    unsigned long long* count;   // device counter (may exceed cap: the caller grows and retries)
};

template <int KIND>
__global__ void __launch_bounds__(kThreads)
scan_pairs_kernel(const double* __restrict__ x, const double* __restrict__ dx, int64_t n, Surf S, Grid G,
                  const int32_t* __restrict__ vscene, PairList L) {
    __shared__ int32_t qq_sh[kWarps][64], qt_sh[kWarps][64];
    int32_t* qq = qq_sh[threadIdx.x >> 5];
    int32_t* qt = qt_sh[threadIdx.x >> 5];
    const int lane = threadIdx.x & 31;
    const int64_t nq = KIND == K_EE ? S.nedge : S.nvert;
    const int64_t nw = (int64_t)gridDim.x * kWarps;
    const float4* ent4 = reinterpret_cast<const float4*>(G.ent);
    auto flush = [&](int cnt) {   // append the first cnt queued pairs (cnt <= 32)
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(L.count, (unsigned long long)cnt);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (lane < cnt && (int64_t)(base + lane) < L.cap) {
            L.q[base + lane] = qq[lane];
            L.t[base + lane] = qt[lane];
        }
    };
    int queued = 0;   // same value in every lane
    for (int64_t q = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); q < nq; q += nw) {
        double ql[3], qh[3];
        int32_t p = 0, ia = 0, ib = 0;
        if (KIND == K_EE) {
            ia = S.edges[q];
            ib = S.edges[S.nedge + q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                ql[c] = G.lo[c * G.m + q];
                qh[c] = G.hi[c * G.m + q];
            }
        } else {
            p = S.verts[q];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double a = x[c * n + p];
                const double b = KIND == K_PT_SWEPT ? __dadd_rn(a, dx[c * n + p]) : a;
                ql[c] = fmin(a, b);
                qh[c] = fmax(a, b);
            }
        }
        const int32_t qs = vscene ? vscene[KIND == K_EE ? ia : p] : 0;   // the query's scene
        const float ih = (float)G.inv_h[qs];
        float fl[3], fh[3];
        box32(ql, qh, fl, fh);
        int c0[3], c1[3];
        if (box_cells(fl, fh, ih, c0, c1) > kMaxCellsPerBox) continue;
        for (int cz = c0[2]; cz <= c1[2]; ++cz)
            for (int cy = c0[1]; cy <= c1[1]; ++cy)
                for (int cx = c0[0]; cx <= c1[0]; ++cx) {
                    const uint64_t b = bucket_of(cx, cy, cz, qs, G.mask);
                    const int64_t e0 = G.boff[b], e1 = G.boff[b + 1];
                    for (int64_t base = e0; base < e1; base += 32) {
                        const int64_t e = base + lane;
                        bool ok = false;
                        int32_t t = 0;
                        if (e < e1) {
                            const float4 A = __ldg(ent4 + 2 * e), B = __ldg(ent4 + 2 * e + 1);
                            t = __float_as_int(A.w);
                            // the float32 boxes overlap, and this is the pair's reference cell
                            ok = __float_as_int(B.w) == qs && fl[0] <= B.x && fh[0] >= A.x && fl[1] <= B.y &&
                                 fh[1] >= A.y && fl[2] <= B.z && fh[2] >= A.z && (KIND != K_EE || t > q) &&
                                 cell32(fmaxf(fl[0], A.x), ih) == cx && cell32(fmaxf(fl[1], A.y), ih) == cy &&
                                 cell32(fmaxf(fl[2], A.z), ih) == cz;
                            if (ok) {   // no shared vertex
                                if (KIND == K_EE) {
                                    const int32_t j0 = S.edges[t], j1 = S.edges[S.nedge + t];
                                    ok = j0 != ia && j0 != ib && j1 != ia && j1 != ib;
                                } else {
                                    ok = p != S.tris[t] && p != S.tris[S.ntri + t] && p != S.tris[2 * S.ntri + t];
                                }
                            }
                        }
                        const unsigned m = __ballot_sync(0xffffffffu, ok);
                        if (ok) {
                            const int at = queued + __popc(m & ((1u << lane) - 1u));
                            qq[at] = (int32_t)q;
                            qt[at] = t;
                        }
                        queued += __popc(m);
                        __syncwarp();
                        if (queued >= 32) {
                            flush(32);
                            const int rest = queued - 32;
                            const int32_t mq = lane < rest ? qq[32 + lane] : 0, mt = lane < rest ? qt[32 + lane] : 0;
                            __syncwarp();
                            if (lane < rest) {
                                qq[lane] = mq;
                                qt[lane] = mt;
                            }
                            queued = rest;
                            __syncwarp();
                        }
                    }
                }
    }
    if (queued > 0) flush(queued);
}

// ------------------------------------------------------------------------------ detection
// Classify every candidate pair once: code = type | i << 2 | j << 4 (closest features) for a pair
// closer than dhat, -1 otherwise; hits are counted per query (combined query index: surface
// vertices first, then edges).
// ------------------------------------------------------------- certified float32 prefilter
// Most candidate pairs are not contacts: on the sphere-grid scene about 85% of the point-triangle
// and edge-edge candidates are more than dhat apart, and classifying them costs the float64
// closest-feature computation, whose branches leave half of each warp idle.  A float32 pass first
// bounds each pair's distance from below, on float32 roundings of the float64 points, with
// margins that cover that rounding and the float32 arithmetic.  A pair is dropped only when the
// bound proves the float64 classification would find it farther than dhat (or, for the CCD, that
// the additive CCD's first step would already pass t = 1), so every result stays bit-identical;
// the rest are classified as before, densely, from a compacted list.
//
// The bound is certified only for well-shaped primitives: a triangle with |e0 x e1|^2 >= 0.02 a c
// (a = |e0|^2, c = |e1|^2), an edge pair with |e1 x e2|^2 >= 0.02 a c.  There the float64
// classification's region decisions err only within rounding of a region boundary, so the
// distance it computes is the true distance to within rounding; near-degenerate triangles and
// nearly parallel edges are always classified in float64.
struct F3 {
    float x, y, z;
};
__device__ __forceinline__ F3 ld3f(const float* __restrict__ X, int64_t n, int64_t i) {
    return {X[i], X[n + i], X[2 * n + i]};
}
__device__ __forceinline__ F3 fsub(F3 a, F3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ float fdot(F3 a, F3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ F3 fcross(F3 a, F3 b) {
    return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ float fabsmax(F3 a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// Lower bound on the distance between the pair's primitives (point X[0] and triangle X[1..3], or
// edges X[0..1] and X[2..3]), less the rounding margins; -1 where not certified.
//   point-triangle: the point's offset from the triangle's plane, h, and its largest signed
//   distance past an edge within the plane, s (outward normal of edge k: d_k x n), give
//   dist^2 >= h^2 + max(s, 0)^2;
//   edge-edge: the line-line distance h (along n = e1 x e2) and the in-plane gaps of each edge
//   from the other's line (along e1 x n and e2 x n) give dist^2 >= h^2 + max(g1, g2, 0)^2.
// Margins: rounding the points to float32 moves each by at most sqrt(3) 2^-24 max|x| (4e-7 max|x|
// covers both primitives); the float32 arithmetic errs by far less than 1e-4 of the pair's extent
// for the shapes certified (amplification below sqrt(a c / |n|^2) < 8).
__device__ __forceinline__ float pair_lb32(const F3 (&X)[4], bool pt) {
    float amax = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) amax = fmaxf(amax, fabsmax(X[k]));
    float h, side = 0.f, ext;
    if (pt) {
        const F3 e0 = fsub(X[2], X[1]), e1 = fsub(X[3], X[1]), v = fsub(X[0], X[1]);
        const float a = fdot(e0, e0), c = fdot(e1, e1);
        const F3 nr = fcross(e0, e1);
        const float nn = fdot(nr, nr);
        if (!(nn >= 0.02f * a * c) || !(nn > 0.f)) return -1.f;
        const float ln = sqrtf(nn);
        h = fabsf(fdot(v, nr)) / ln;
        const F3 d[3] = {e0, fsub(X[3], X[2]), fsub(X[1], X[3])};
        const F3 w[3] = {v, fsub(X[0], X[2]), fsub(X[0], X[3])};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const F3 m = fcross(d[k], nr);
            side = fmaxf(side, fdot(w[k], m) / (sqrtf(fdot(d[k], d[k])) * ln));
        }
        ext = sqrtf(fmaxf(fmaxf(a, c), fdot(v, v)));
    } else {
        const F3 e1 = fsub(X[1], X[0]), e2 = fsub(X[3], X[2]), w = fsub(X[0], X[2]);
        const float a = fdot(e1, e1), c = fdot(e2, e2);
        const F3 nr = fcross(e1, e2);
        const float nn = fdot(nr, nr);
        if (!(nn >= 0.02f * a * c) || !(nn > 0.f)) return -1.f;
        const float ln = sqrtf(nn);
        h = fabsf(fdot(w, nr)) / ln;
        const F3 u1 = fcross(e1, nr), u2 = fcross(e2, nr);
        // edge b relative to the line of edge a, edge a relative to the line of edge b
        const float pb0 = -fdot(w, u1), pb1 = fdot(fsub(X[3], X[0]), u1);
        const float qa0 = fdot(w, u2), qa1 = fdot(fsub(X[1], X[2]), u2);
        const float g1 = fmaxf(fminf(pb0, pb1), -fmaxf(pb0, pb1)) / (sqrtf(a) * ln);
        const float g2 = fmaxf(fminf(qa0, qa1), -fmaxf(qa0, qa1)) / (sqrtf(c) * ln);
        side = fmaxf(g1, g2);
        ext = sqrtf(fmaxf(fmaxf(a, c), fdot(w, w)));
    }
    side = fmaxf(side, 0.f);
    const float lb = sqrtf(h * h + side * side) - 4e-7f * amax - 1e-4f * ext;
    return lb == lb ? lb : -1.f;   // (a NaN certifies nothing)
}

// Appends r to the list when keep (one atomic per warp; the list's order does not matter).
__device__ __forceinline__ void append_kept(bool keep, int64_t r, int32_t* __restrict__ list, unsigned* __restrict__ count) {
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    const int lane = threadIdx.x & 31;
    unsigned base = 0;
    if (lane == 0 && mask) base = atomicAdd(count, (unsigned)__popc(mask));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (keep) list[base + __popc(mask & ((1u << lane) - 1u))] = (int32_t)r;
}

__device__ __forceinline__ void pair_ids(const Surf& S, int32_t q, int32_t t, bool pt, int32_t (&ids)[4]) {
    if (pt) {
        ids[0] = S.verts[q]; ids[1] = S.tris[t]; ids[2] = S.tris[S.ntri + t]; ids[3] = S.tris[2 * S.ntri + t];
    } else {
        ids[0] = S.edges[q]; ids[1] = S.edges[S.nedge + q]; ids[2] = S.edges[t]; ids[3] = S.edges[S.nedge + t];
    }
}

__global__ void to_f32_kernel(const double* __restrict__ a, int64_t m, float* __restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) b[i] = (float)a[i];
}

// Classification prefilter: pairs proven farther than thr (dhat plus a relative margin, rounded
// up) get code -1; the others are listed for classify_pairs_kernel.  Launched with whole warps.
__global__ void prefilter_pairs_kernel(const float* __restrict__ x32, int64_t n, Surf S, const int32_t* __restrict__ pq,
                                       const int32_t* __restrict__ ptg, int64_t npt, int64_t np, float thr,
                                       int32_t* __restrict__ code, int32_t* __restrict__ list, unsigned* __restrict__ count) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (r < np) {
        int32_t ids[4];
        pair_ids(S, pq[r], ptg[r], r < npt, ids);
        F3 X[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) X[k] = ld3f(x32, n, ids[k]);
        keep = !(pair_lb32(X, r < npt) > thr);
        if (!keep) code[r] = -1;
    }
    append_kept(keep, r, list, count);
}

// Classifies the listed pairs (list[0 .. *count)), or every pair when list is null.
__global__ void classify_pairs_kernel(const double* __restrict__ x, int64_t n, Surf S, const int32_t* __restrict__ pq,
                                      const int32_t* __restrict__ pt, int64_t npt, int64_t np, double dh2,
                                      int32_t* __restrict__ code, int32_t* __restrict__ cnt,
                                      const int32_t* __restrict__ list, const unsigned* __restrict__ count) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        if (r >= (int64_t)*count) return;
        r = list[r];
    } else if (r >= np) {
        return;
    }
    const int32_t q = pq[r], t = pt[r];
    double d2;
    int type, i = 0, j = 0;
    int64_t qc;
    if (r < npt) {
        const int32_t p = S.verts[q];
        type = classify_pt(ld3(x, n, p), ld3(x, n, S.tris[t]), ld3(x, n, S.tris[S.ntri + t]),
                           ld3(x, n, S.tris[2 * S.ntri + t]), d2, i, j);
        qc = q;
    } else {
        type = classify_ee(ld3(x, n, S.edges[q]), ld3(x, n, S.edges[S.nedge + q]), ld3(x, n, S.edges[t]),
                           ld3(x, n, S.edges[S.nedge + t]), d2, i, j);
        qc = S.nvert + q;
    }
    const bool hit = d2 < dh2;
    code[r] = hit ? (type | i << 2 | j << 4) : -1;
    if (hit) atomicAdd(&cnt[qc], 1);
}

// Write the stencil of every hit at off[query] + a per-query cursor (the order within a query is
// fixed afterwards by sorting on the target index).
__global__ void write_pairs_kernel(const double* __restrict__ x, const double* __restrict__ rx, int64_t n, Surf S,
                                   const int32_t* __restrict__ pq, const int32_t* __restrict__ ptg,
                                   const int32_t* __restrict__ code, int64_t npt, int64_t np,
                                   const int64_t* __restrict__ off, int32_t* __restrict__ cur, int32_t* __restrict__ st,
                                   double* __restrict__ eps, int32_t* __restrict__ key, int64_t stride) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= np) return;
    const int32_t c = code[r];
    if (c < 0) return;
    const int32_t q = pq[r], t = ptg[r];
    const int type = c & 3, i = (c >> 2) & 3, j = (c >> 4) & 3;
    int32_t s0, s1, s2, s3;
    double ex = 0.0;
    int64_t at;
    if (r < npt) {
        at = off[q] + atomicAdd(&cur[q], 1);
        const int32_t p = S.verts[q];
        const int32_t T[3] = {S.tris[t], S.tris[S.ntri + t], S.tris[2 * S.ntri + t]};
        s0 = neg(p);
        if (type == 0) { s1 = T[0]; s2 = T[1]; s3 = T[2]; }
        else if (type == 1) { s1 = T[i]; s2 = T[j]; s3 = GIPC_NULL_INDEX; }
        else { s1 = T[i]; s2 = GIPC_NULL_INDEX; s3 = GIPC_NULL_INDEX; }
    } else {
        const int64_t qc = S.nvert + q;
        at = off[qc] + atomicAdd(&cur[qc], 1);
        const int32_t V[4] = {S.edges[q], S.edges[S.nedge + q], S.edges[t], S.edges[S.nedge + t]};
        // eps_x from rest positions, then the parallel test at the current positions
        const V3 ra = vsub(ld3(rx, n, V[1]), ld3(rx, n, V[0])), rb = vsub(ld3(rx, n, V[3]), ld3(rx, n, V[2]));
        ex = __dmul_rn(__dmul_rn(1e-3, vdot(ra, ra)), vdot(rb, rb));
        const V3 cr = vcross(vsub(ld3(x, n, V[1]), ld3(x, n, V[0])), vsub(ld3(x, n, V[3]), ld3(x, n, V[2])));
        const bool par = vdot(cr, cr) < ex;
        const int mate[4] = {1, 0, 3, 2};
        const int P = i, Q = j;
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
    }
    st[at] = s0;
    st[stride + at] = s1;
    st[2 * stride + at] = s2;
    st[3 * stride + at] = s3;
    eps[at] = ex;
    key[at] = t;
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
    // the first step already passes t = 1: the distance at the advanced point would go unused
    if (tl > 1.0) return 1.0;
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

__device__ __forceinline__ double warp_min(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// ACCD of every candidate pair (point-triangle pairs first); the step is the minimum over pairs.
// Swept box (x and x + d) of the vertices ids[a0..a1), as the grid builds it (unpadded).
__device__ __forceinline__ void swept_box(const V3* X, const V3* P, int a0, int a1, double (&lo)[3], double (&hi)[3]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        lo[c] = INFINITY;
        hi[c] = -INFINITY;
    }
    for (int a = a0; a < a1; ++a) {
        const double p[3] = {X[a].x, X[a].y, X[a].z}, d[3] = {P[a].x, P[a].y, P[a].z};
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double y = __dadd_rn(p[c], d[c]);
            lo[c] = fmin(lo[c], fmin(p[c], y));
            hi[c] = fmax(hi[c], fmax(p[c], y));
        }
    }
}

// ACCD of every candidate pair (point-triangle pairs first); the step is the minimum over pairs.
// With box_filter the pairs come from a superset (the time step's cached candidates) and only
// those whose swept boxes overlap -- the pairs the swept grid would propose -- are tested.
// CCD prefilter: a pair whose certified distance bound lb (float32 prefilter above) satisfies
// (1 - s) lb > lp, lp the additive CCD's motion bound (recomputed in float32 with a margin), would
// leave the CCD at its first step with t = 1: it cannot lower the step and is dropped.  The others
// are listed for ccd_pairs_kernel.  omss = 1 - s rounded down.  Launched with whole warps.
__global__ void prefilter_ccd_kernel(const float* __restrict__ x32, const float* __restrict__ d32, int64_t n, Surf S,
                                     const int32_t* __restrict__ pq, const int32_t* __restrict__ ptg, int64_t npt,
                                     int64_t np, float omss, int32_t* __restrict__ list, unsigned* __restrict__ count) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool keep = false;
    if (r < np) {
        const bool pt = r < npt;
        int32_t ids[4];
        pair_ids(S, pq[r], ptg[r], pt, ids);
        F3 X[4], P[4];
        float pmax = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            X[k] = ld3f(x32, n, ids[k]);
            P[k] = ld3f(d32, n, ids[k]);
            pmax = fmaxf(pmax, fabsmax(P[k]));
        }
        const F3 pb = {0.25f * (P[0].x + P[1].x + P[2].x + P[3].x), 0.25f * (P[0].y + P[1].y + P[2].y + P[3].y),
                       0.25f * (P[0].z + P[1].z + P[2].z + P[3].z)};
        float nr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const F3 c = fsub(P[k], pb);
            nr[k] = sqrtf(fdot(c, c));
        }
        const float lp = pt ? nr[0] + fmaxf(fmaxf(nr[1], nr[2]), nr[3]) : fmaxf(nr[0], nr[1]) + fmaxf(nr[2], nr[3]);
        const float lb = pair_lb32(X, pt);
        keep = !(lb > 0.f && omss * lb > 1.0001f * lp + 1e-5f * pmax);
    }
    append_kept(keep, r, list, count);
}

// The listed pairs (list[0 .. *count)), or every pair when list is null.
__global__ void ccd_pairs_kernel(const double* __restrict__ x, const double* __restrict__ dx, int64_t n, Surf S,
                                 const int32_t* __restrict__ pq, const int32_t* __restrict__ ptg, int64_t npt,
                                 int64_t np, double s, int max_iter, const int32_t* __restrict__ vscene,
                                 unsigned long long* __restrict__ amin, bool box_filter,
                                 const int32_t* __restrict__ list, const unsigned* __restrict__ count) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool valid;
    if (list) {
        valid = r < (int64_t)*count;
        if (valid) r = list[r];
    } else {
        valid = r < np;
    }
    double best = 1.0;
    int32_t scene = 0;
    if (valid) {
        int32_t ids[4];
        pair_ids(S, pq[r], ptg[r], r < npt, ids);
        V3 X[4], P[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            X[a] = ld3(x, n, ids[a]);
            P[a] = ld3(dx, n, ids[a]);
        }
        bool test = true;
        if (box_filter) {
            const int split = r < npt ? 1 : 2;   // query vertices: the point, or the first edge
            double ql[3], qh[3], tl[3], th[3];
            swept_box(X, P, 0, split, ql, qh);
            swept_box(X, P, split, 4, tl, th);
            test = ql[0] <= th[0] && qh[0] >= tl[0] && ql[1] <= th[1] && qh[1] >= tl[1] && ql[2] <= th[2] &&
                   qh[2] >= tl[2];
        }
        if (test) best = accd(X, P, r < npt, s, max_iter);
        if (vscene) scene = vscene[ids[0]];
    }
    if (!vscene) {   // one scene: one atomic per warp
        best = warp_min(best);
        if ((threadIdx.x & 31) == 0 && best < 1.0) atomic_min_pos(amin, best);
    } else if (best < 1.0) {
        atomic_min_pos(amin + scene, best);
    }
}

inline unsigned nblk(int64_t w, int t) { return (unsigned)std::max<int64_t>(1, (w + t - 1) / t); }

__global__ void fill_kernel(double* __restrict__ a, int64_t m, double v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) a[i] = v;
}
// out[0] = max over surface vertices and axes of |x - xb|, out[1] = of |d| (when d), as the bit
// patterns of nonnegative doubles (which order like the values).
__global__ void disp_kernel(const double* __restrict__ x, const double* __restrict__ xb, const double* __restrict__ d,
                            int64_t n, const int32_t* __restrict__ verts, int64_t nvert,
                            unsigned long long* __restrict__ out) {
    double a = 0.0, b = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvert; i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v = verts[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a = fmax(a, fabs(x[c * n + v] - xb[c * n + v]));
            if (d) b = fmax(b, fabs(d[c * n + v]));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
        b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(out, (unsigned long long)__double_as_longlong(a));
        atomicMax(out + 1, (unsigned long long)__double_as_longlong(b));
    }
}

// persistent warp-per-query grids: at most 16 blocks of kWarps warps per SM
inline unsigned wblk(int64_t queries) { return grid_for(queries, kWarps, 16); }

// Insert the m primitives (nv vertices each) into hashed grid g over their boxes (x, swept by
// d if given, padded by pad).  Synchronises once per cell-size attempt.  `pts`: surface
// vertices whose swept boxes also bound the cell size (CCD).
gipc_status build_grid(gipc_ctx* ctx, int g, const double* x, const double* d, int64_t n, const int32_t* prim, int nv,
                       int64_t m, double pad, const gipc_surface* pts, const int32_t* vscene, int nscenes, Grid& G,
                       cudaStream_t st) {
    gipc_status s;
    gipc_scratch* slot = ctx->slot;
    const int* gs = kGridSlots[g];
    if ((s = slot[C_MISC].reserve(16 * sizeof(double))) != GIPC_OK) return s;
    double* misc = slot[C_MISC].as<double>() + 4 * g;
    unsigned long long* max_cells = reinterpret_cast<unsigned long long*>(misc + 2);
    if ((s = slot[gs[0]].reserve(sizeof(double) * 6 * (m + 1))) != GIPC_OK) return s;
    double* lo = slot[gs[0]].as<double>();
    double* hi = lo + 3 * m;
    if ((s = slot[gs[2]].reserve(sizeof(int32_t) * (m + 1))) != GIPC_OK) return s;
    int32_t* cnt = slot[gs[2]].as<int32_t>();
    if ((s = slot[gs[3]].reserve(sizeof(int64_t) * (m + 2 + scan_scratch_words(m + 1)))) != GIPC_OK) return s;
    int64_t* off = slot[gs[3]].as<int64_t>();
    // per-scene extent sums and counts, then 1 / cell size per scene
    const int ns = vscene ? nscenes : 1;
    if ((s = slot[gs[4]].reserve(sizeof(double) * 3 * ns)) != GIPC_OK) return s;
    double* ext_sum = slot[gs[4]].as<double>();
    double* ext_cnt = ext_sum + ns;
    double* inv_h = ext_cnt + ns;
    cudaMemsetAsync(ext_sum, 0, sizeof(double) * 2 * ns, st);
    target_boxes_kernel<<<nblk(m, 256), 256, 0, st>>>(x, d, n, prim, nv, m, pad, vscene, lo, hi, ext_sum, ext_cnt);
    int64_t total = 0;
    unsigned long long mc = 0;
    for (double scale = 1.0;; scale *= 2.0) {
        cell_size_kernel<<<nblk(ns, 256), 256, 0, st>>>(ext_sum, ext_cnt, ns, scale, inv_h);
        cudaMemsetAsync(max_cells, 0, sizeof(unsigned long long), st);
        cells_count_kernel<<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, prim, vscene, inv_h, cnt, max_cells);
        if (pts && pts->nvert > 0)
            point_cells_kernel<<<nblk(pts->nvert, 256), 256, 0, st>>>(x, d, n, pts->verts, pts->nvert, vscene, inv_h,
                                                                       max_cells);
        if (exclusive_scan<int32_t>(cnt, off, m, off + m + 2, st) != cudaSuccess)
            return check_launch("contact grid: scan");
        cudaMemcpyAsync(&mc, max_cells, sizeof(mc), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&total, off + m, sizeof(total), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("contact grid: sync");
        if ((int64_t)mc <= kMaxCellsPerBox) break;
        if (scale > 1e12) return fail(GIPC_ERR_NONFINITE, "contact grid: non-finite or unbounded positions");
    }
    uint64_t buckets = 1024;
    while ((int64_t)buckets < 2 * total) buckets <<= 1;
    const int64_t head = buckets + 2 + scan_scratch_words(buckets + 1);   // int64 words before the counts
    const int64_t cnt_words = (buckets + 1) / 2 + 1;                       // int32 counts, in int64 words
    const size_t grid_bytes = sizeof(int64_t) * (head + cnt_words) + sizeof(Entry) * (total + 1) + 16;
    if ((s = slot[gs[1]].reserve(grid_bytes)) != GIPC_OK) return s;
    int64_t* boff = slot[gs[1]].as<int64_t>();
    int64_t* btmp = boff + buckets + 2;
    int32_t* bcnt = reinterpret_cast<int32_t*>(boff + head);
    // entries start on a 16-byte boundary after the counts
    uintptr_t ep = reinterpret_cast<uintptr_t>(boff + head + cnt_words);
    ep = (ep + 15) & ~uintptr_t(15);
    Entry* ent = reinterpret_cast<Entry*>(ep);
    cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * buckets, st);
    bucket_kernel<false><<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, prim, vscene, inv_h, buckets - 1, bcnt, nullptr,
                                                        nullptr);
    if (exclusive_scan<int32_t>(bcnt, boff, (int64_t)buckets, btmp, st) != cudaSuccess)
        return check_launch("contact grid: bucket scan");
    cudaMemsetAsync(bcnt, 0, sizeof(int32_t) * buckets, st);
    bucket_kernel<true><<<nblk(m, 256), 256, 0, st>>>(lo, hi, m, prim, vscene, inv_h, buckets - 1, bcnt, boff, ent);
    G = Grid{lo, hi, m, inv_h, buckets - 1, boff, ent};
    return check_launch("contact grid");
}

// Candidate pairs of the point-triangle grid Gt (if any) followed by those of the edge grid Ge
// (if any) into the context's pair list; *npt / *np: point-triangle pairs / all pairs.
// Synchronises once per attempt (the list grows when the count exceeds its capacity).
gipc_status collect_pairs(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const Surf& S, const Grid* Gt,
                          const Grid* Ge, bool swept, const int32_t* vscene, int64_t* npt, int64_t* np, PairList& L,
                          cudaStream_t st) {
    gipc_status s;
    unsigned long long* counter = reinterpret_cast<unsigned long long*>(ctx->slot[C_MISC].as<double>() + kMiscPairs);
    for (int attempt = 0; attempt < 2; ++attempt) {
        L.cap = (int64_t)(ctx->slot[C_PAIRS].bytes / (2 * sizeof(int32_t)));
        L.q = ctx->slot[C_PAIRS].as<int32_t>();
        L.t = L.q + L.cap;
        L.count = counter;
        unsigned long long c[2] = {0, 0};
        cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st);
        if (Gt) {
            if (swept) scan_pairs_kernel<K_PT_SWEPT><<<wblk(S.nvert), kThreads, 0, st>>>(x, d, n, S, *Gt, vscene, L);
            else scan_pairs_kernel<K_PT><<<wblk(S.nvert), kThreads, 0, st>>>(x, d, n, S, *Gt, vscene, L);
        }
        cudaMemcpyAsync(&c[0], counter, sizeof(c[0]), cudaMemcpyDeviceToHost, st);
        if (Ge) scan_pairs_kernel<K_EE><<<wblk(S.nedge), kThreads, 0, st>>>(x, d, n, S, *Ge, vscene, L);
        cudaMemcpyAsync(&c[1], counter, sizeof(c[1]), cudaMemcpyDeviceToHost, st);
        if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("contact pairs: sync");
        if ((int64_t)c[1] <= L.cap) {
            *npt = (int64_t)c[0];
            *np = (int64_t)c[1];
            return check_launch("contact pairs");
        }
        const int64_t want = (int64_t)c[1] + (int64_t)c[1] / 4 + 4096;
        if ((s = ctx->slot[C_PAIRS].reserve(sizeof(int32_t) * 2 * want)) != GIPC_OK) return s;
    }
    return fail(GIPC_ERR_CUDA, "contact pairs: candidate count changed between passes");
}

bool cache_matches(const gipc_ctx* ctx, int64_t n, const gipc_surface& srf, double dhat, const int32_t* vscene,
                   int nscenes) {
    const gipc_contact_cache& C = ctx->ccache;
    return C.valid && C.n == n && C.dhat == dhat && C.tris == srf.tris && C.edges == srf.edges &&
           C.verts == srf.verts && C.ntri == srf.ntri && C.nedge == srf.nedge && C.nvert == srf.nvert &&
           C.vscene == vscene && C.nscenes == (vscene ? nscenes : 1);
}

// Largest per-axis move of a surface vertex since the cached candidates were built, and the
// largest per-axis entry of d over the surface vertices.  Synchronises once.
gipc_status cache_disp(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const gipc_surface& srf,
                       double* delta, double* dmax, cudaStream_t st) {
    unsigned long long* out = reinterpret_cast<unsigned long long*>(ctx->slot[C_MISC].as<double>() + kMiscDisp);
    cudaMemsetAsync(out, 0, 2 * sizeof(unsigned long long), st);
    const unsigned blocks = grid_for(srf.nvert, 256, 4);
    disp_kernel<<<blocks, 256, 0, st>>>(x, ctx->slot[C_CX].as<double>(), d, n, srf.verts, srf.nvert, out);
    unsigned long long h[2] = {0, 0};
    cudaMemcpyAsync(h, out, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("contact cache: sync");
    std::memcpy(delta, &h[0], sizeof(double));
    std::memcpy(dmax, &h[1], sizeof(double));
    return check_launch("contact cache");
}

// Float32 copies of x (and d) for the prefilters, the list they fill and its length (zeroed).
gipc_status prefilter_setup(gipc_ctx* ctx, const double* x, const double* d, int64_t n, int64_t np, float** x32,
                            float** d32, int32_t** list, unsigned** count, cudaStream_t st) {
    gipc_status s;
    if ((s = ctx->slot[C_X32].reserve(sizeof(float) * 6 * (n + 1))) != GIPC_OK) return s;
    if ((s = ctx->slot[C_LIST].reserve(sizeof(int32_t) * (np + 32))) != GIPC_OK) return s;
    *x32 = ctx->slot[C_X32].as<float>();
    *d32 = *x32 + 3 * n;
    *list = ctx->slot[C_LIST].as<int32_t>();
    *count = reinterpret_cast<unsigned*>(ctx->slot[C_MISC].as<double>() + kMiscList);
    cudaMemsetAsync(*count, 0, sizeof(unsigned), st);
    to_f32_kernel<<<nblk(3 * n, 256), 256, 0, st>>>(x, 3 * n, *x32);
    if (d) to_f32_kernel<<<nblk(3 * n, 256), 256, 0, st>>>(d, 3 * n, *d32);
    return GIPC_OK;
}

// Margin tuner (see gipc_contact_cache): GPU time of the cached detections and CCD steps.  A span
// is read back at the next cached call, after the stream synchronisations in between.
void tuner_harvest(gipc_contact_cache& C) {
    for (int k = 0; k < 2; ++k) {
        if (!C.pending[k]) continue;
        C.pending[k] = false;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, C.ev[k][0], C.ev[k][1]) == cudaSuccess)
            C.epoch_ms += ms;
        else
            cudaGetLastError();   // not complete: the sample is dropped
    }
}

// Records the spans of one cached call of kind k (0 detection, 1 CCD) on the stream.
struct TunerSpan {
    gipc_contact_cache& C;
    int k;
    cudaStream_t st;
    bool on = false;
    TunerSpan(gipc_contact_cache& c, int kind, cudaStream_t s, bool enable) : C(c), k(kind), st(s) {
        if (!enable) return;
        tuner_harvest(C);
        for (auto& e : C.ev[k])
            if (!e && cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
                return;
            }
        on = cudaEventRecord(C.ev[k][0], st) == cudaSuccess;
    }
    ~TunerSpan() {
        if (on) C.pending[k] = cudaEventRecord(C.ev[k][1], st) == cudaSuccess;
    }
};

// Ends the epoch of the current candidates (`outran`: the surface moved past their margin) and
// picks the level of the next build.
void tuner_close_epoch(gipc_contact_cache& C, bool outran, double dhat, bool batched) {
    if (C.tuned_dhat != dhat || C.tuned_batch != batched) {   // another scene: start over
        for (int l = 0; l < C.kLevels; ++l) C.cost[l] = C.dets[l] = 0.0;
        C.level = 0;
        C.tuned_dhat = dhat;
        C.tuned_batch = batched;
        C.epoch_ms = 0.0;
        C.epoch_dets = 0;
        return;
    }
    if (C.epoch_dets > 0) {
        const int b = C.built;
        C.cost[b] = 0.5 * C.cost[b] + C.epoch_ms;
        C.dets[b] = 0.5 * C.dets[b] + C.epoch_dets;
    }
    C.epoch_ms = 0.0;
    C.epoch_dets = 0;
    int best = C.built;
    for (int l = 0; l < C.kLevels; ++l)
        if (C.dets[l] > 0.0 && (C.dets[best] <= 0.0 || C.cost[l] / C.dets[l] < C.cost[best] / C.dets[best])) best = l;
    // widen into an untried level only from the best one, and only when its margin was outrun
    C.level = (outran && best == C.built && C.built + 1 < C.kLevels && C.dets[C.built + 1] <= 0.0) ? C.built + 1 : best;
}

}  // namespace

// Internal entry points shared with the time-step driver (newton.cu).
// cached: use and refill the context's candidate cache (one scene; the time step's detections).
gipc_status find_contacts_impl(gipc_ctx* ctx, const double* x, const double* rest_x, int64_t n, const gipc_surface& srf,
                               double dhat, int32_t* stencils, double* eps_x, int64_t cap, int64_t* count,
                               bool compact, const int32_t* vscene, int64_t* npt_out, cudaStream_t st, int nscenes,
                               bool cached) {
    gipc_prof_span span(ctx->prof, GIPC_PROF_CONTACTS, st);
    Surf S{srf.tris, srf.ntri, srf.edges, srf.nedge, srf.verts, srf.nvert};
    const double pad = dhat * (1.0 + 1e-9);
    const double dh2 = dhat * dhat;
    const int64_t nq = S.nvert + S.nedge;
    *count = 0;
    if (nq == 0) return GIPC_OK;
    gipc_status s;
    if ((s = ctx->slot[C_MISC].reserve(16 * sizeof(double))) != GIPC_OK) return s;
    const bool pt = S.nvert > 0 && S.ntri > 0;
    // cached candidates: valid while no surface vertex has moved more than the margin since they
    // were collected (boxes padded by dhat + 2 margin); the classification below decides exactly
    const bool use_cache = cached;
    gipc_contact_cache& CC = ctx->ccache;
    TunerSpan tspan(CC, 0, st, use_cache);
    bool hit = false, outran = false;
    if (use_cache && cache_matches(ctx, n, srf, dhat, vscene, nscenes)) {
        double delta = 0.0, dm = 0.0;
        if ((s = cache_disp(ctx, x, nullptr, n, srf, &delta, &dm, st)) != GIPC_OK) return s;
        hit = delta * (1.0 + 1e-9) <= CC.margin;
        outran = !hit;
    }
    if (use_cache) {
        if (hit) {
            ++CC.epoch_dets;
        } else {
            tuner_close_epoch(CC, outran, dhat, vscene != nullptr);
            CC.built = CC.level;
            CC.epoch_dets = 1;
        }
    }
    const double margin = CC.kMargin[use_cache ? CC.built : 0] * dhat;
    PairList L{};
    int64_t npt = 0, np = 0;
    if (hit) {
        np = ctx->ccache.np;
        npt = ctx->ccache.npt;
        L.q = ctx->slot[C_CPAIRS].as<int32_t>();
        L.t = L.q + np;
    } else {
        const double pad_b = use_cache ? (dhat + 2.0 * margin) * (1.0 + 1e-9) : pad;
        Grid Gt{}, Ge{};
        if (pt && (s = build_grid(ctx, 0, x, nullptr, n, S.tris, 3, S.ntri, pad_b, nullptr, vscene, nscenes, Gt, st)) !=
                      GIPC_OK)
            return s;
        if (S.nedge > 0 &&
            (s = build_grid(ctx, 1, x, nullptr, n, S.edges, 2, S.nedge, pad_b, nullptr, vscene, nscenes, Ge, st)) !=
                GIPC_OK)
            return s;
        if ((s = collect_pairs(ctx, x, nullptr, n, S, pt ? &Gt : nullptr, S.nedge > 0 ? &Ge : nullptr, false, vscene,
                               &npt, &np, L, st)) != GIPC_OK)
            return s;
        if (use_cache) {   // keep the candidates and the positions they were collected at
            ctx->ccache.valid = false;
            if ((s = ctx->slot[C_CPAIRS].reserve(sizeof(int32_t) * 2 * (np + 1))) != GIPC_OK) return s;
            if ((s = ctx->slot[C_CX].reserve(sizeof(double) * 3 * n)) != GIPC_OK) return s;
            int32_t* cq = ctx->slot[C_CPAIRS].as<int32_t>();
            cudaMemcpyAsync(cq, L.q, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(cq + np, L.t, sizeof(int32_t) * np, cudaMemcpyDeviceToDevice, st);
            cudaMemcpyAsync(ctx->slot[C_CX].as<double>(), x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, st);
            gipc_contact_cache& C = ctx->ccache;
            C.n = n;
            C.npt = npt;
            C.np = np;
            C.tris = srf.tris;
            C.edges = srf.edges;
            C.verts = srf.verts;
            C.ntri = srf.ntri;
            C.nedge = srf.nedge;
            C.nvert = srf.nvert;
            C.vscene = vscene;
            C.nscenes = vscene ? nscenes : 1;
            C.dhat = dhat;
            C.margin = margin;
            C.pad = pad_b;
            C.valid = true;
            L.q = cq;
            L.t = cq + np;
        }
    }
    // classify once, count per query
    if ((s = ctx->slot[C_CNT].reserve(sizeof(int32_t) * (nq + 1))) != GIPC_OK) return s;
    if ((s = ctx->slot[C_CODE].reserve(sizeof(int32_t) * (np + 1))) != GIPC_OK) return s;
    int32_t* cnt = ctx->slot[C_CNT].as<int32_t>();
    int32_t* code = ctx->slot[C_CODE].as<int32_t>();
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nq, st);
    if (np > 0) {
        float *x32, *d32;
        int32_t* list;
        unsigned* nlist;
        if ((s = prefilter_setup(ctx, x, nullptr, n, np, &x32, &d32, &list, &nlist, st)) != GIPC_OK) return s;
        const float thr = nextafterf((float)(dhat * (1.0 + 1e-4)), INFINITY);
        prefilter_pairs_kernel<<<nblk(np, 128), 128, 0, st>>>(x32, n, S, L.q, L.t, npt, np, thr, code, list, nlist);
        classify_pairs_kernel<<<nblk(np, 128), 128, 0, st>>>(x, n, S, L.q, L.t, npt, np, dh2, code, cnt, list, nlist);
    }
    // offsets over both kinds (point-triangle pairs first)
    if ((s = ctx->slot[C_QOFF].reserve(sizeof(int64_t) * (nq + 2 + scan_scratch_words(nq + 1)))) != GIPC_OK) return s;
    int64_t* off = ctx->slot[C_QOFF].as<int64_t>();
    if (exclusive_scan<int32_t>(cnt, off, nq, off + nq + 2, st) != cudaSuccess)
        return check_launch("gipc_find_contacts: scan");
    int64_t total = 0, npt_contacts = 0;
    cudaMemcpyAsync(&total, off + nq, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&npt_contacts, off + S.nvert, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_find_contacts: sync");
    *count = total;
    if (npt_out) *npt_out = npt_contacts;
    if (total > cap) return fail(GIPC_ERR_CAPACITY, "gipc_find_contacts: %lld contacts, capacity %lld", (long long)total, (long long)cap);
    if (total == 0) return GIPC_OK;
    // rows of the output are `stride` apart: the caller's capacity, or the count itself (compact)
    const int64_t stride = compact ? total : cap;
    if ((s = ctx->slot[C_KEY].reserve(sizeof(int32_t) * (total + 1))) != GIPC_OK) return s;
    int32_t* key = ctx->slot[C_KEY].as<int32_t>();
    cudaMemsetAsync(cnt, 0, sizeof(int32_t) * nq, st);   // the counts become per-query cursors
    write_pairs_kernel<<<nblk(np, 256), 256, 0, st>>>(x, rest_x, n, S, L.q, L.t, code, npt, np, off, cnt, stencils, eps_x,
                                                       key, stride);
    segment_sort_kernel<<<nblk(nq, 256), 256, 0, st>>>(off, nq, key, stencils, eps_x, stride);
    return check_launch("gipc_find_contacts");
}

// alpha_h: host [nscenes] step per scene (nscenes = 1 and vscene = NULL for one scene);
// amin_dev: device [nscenes] scratch for the per-scene minima when vscene is given.
// cached: when the context's candidate cache covers every pair the swept grid would propose
// (2 (max |x - x_b| + max |d|) <= its padding), test its pairs through the same swept-box
// overlap instead of building the swept grid; the step is the same.
gipc_status ccd_impl(gipc_ctx* ctx, const double* x, const double* d, int64_t n, const gipc_surface& srf, double slack,
                     double* alpha_h, cudaStream_t st, const int32_t* vscene, int nscenes, double* amin_dev,
                     bool cached) {
    gipc_prof_span span(ctx->prof, GIPC_PROF_CCD, st);
    Surf S{srf.tris, srf.ntri, srf.edges, srf.nedge, srf.verts, srf.nvert};
    const int max_iter = 100000;
    const float omss = nextafterf((float)((1.0 - slack) * (1.0 - 1e-6)), 0.0f);   // 1 - s, rounded down
    gipc_status s;
    if ((s = ctx->slot[C_MISC].reserve(16 * sizeof(double))) != GIPC_OK) return s;
    double* amin_d = vscene ? amin_dev : ctx->slot[C_MISC].as<double>() + kMiscAmin;
    const int ns = vscene ? nscenes : 1;
    fill_kernel<<<nblk(ns, 256), 256, 0, st>>>(amin_d, ns, 1.0);
    unsigned long long* amin = reinterpret_cast<unsigned long long*>(amin_d);
    TunerSpan tspan(ctx->ccache, 1, st, cached);
    if (cached && cache_matches(ctx, n, srf, ctx->ccache.dhat, vscene, nscenes)) {
        double delta = 0.0, dm = 0.0;
        if ((s = cache_disp(ctx, x, d, n, srf, &delta, &dm, st)) != GIPC_OK) return s;
        if (2.0 * (delta + dm) * (1.0 + 1e-9) <= ctx->ccache.pad) {
            const int64_t np = ctx->ccache.np;
            const int32_t* cq = ctx->slot[C_CPAIRS].as<int32_t>();
            if (np > 0) {
                float *x32, *d32;
                int32_t* list;
                unsigned* nlist;
                if ((s = prefilter_setup(ctx, x, d, n, np, &x32, &d32, &list, &nlist, st)) != GIPC_OK) return s;
                prefilter_ccd_kernel<<<nblk(np, 128), 128, 0, st>>>(x32, d32, n, S, cq, cq + np, ctx->ccache.npt, np,
                                                                     omss, list, nlist);
                ccd_pairs_kernel<<<nblk(np, 128), 128, 0, st>>>(x, d, n, S, cq, cq + np, ctx->ccache.npt, np, slack,
                                                                 max_iter, vscene, amin, true, list, nlist);
            }
            cudaMemcpyAsync(alpha_h, amin_d, sizeof(double) * ns, cudaMemcpyDeviceToHost, st);
            if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_ccd_max_step: sync");
            return check_launch("gipc_ccd_max_step");
        }
    }
    Grid Gt{}, Ge{};
    const bool pt = S.nvert > 0 && S.ntri > 0;
    if (pt && (s = build_grid(ctx, 0, x, d, n, S.tris, 3, S.ntri, 0.0, &srf, vscene, nscenes, Gt, st)) != GIPC_OK) return s;
    if (S.nedge > 0 && (s = build_grid(ctx, 1, x, d, n, S.edges, 2, S.nedge, 0.0, nullptr, vscene, nscenes, Ge, st)) != GIPC_OK)
        return s;
    PairList L{};
    int64_t npt = 0, np = 0;
    if ((s = collect_pairs(ctx, x, d, n, S, pt ? &Gt : nullptr, S.nedge > 0 ? &Ge : nullptr, true, vscene, &npt, &np, L,
                           st)) != GIPC_OK)
        return s;
    if (np > 0) {
        float *x32, *d32;
        int32_t* list;
        unsigned* nlist;
        if ((s = prefilter_setup(ctx, x, d, n, np, &x32, &d32, &list, &nlist, st)) != GIPC_OK) return s;
        prefilter_ccd_kernel<<<nblk(np, 128), 128, 0, st>>>(x32, d32, n, S, L.q, L.t, npt, np, omss, list, nlist);
        // the swept grid proposes every pair whose float32 swept boxes overlap: the float64 swept-box
        // test picks the pairs whose step is taken
        ccd_pairs_kernel<<<nblk(np, 128), 128, 0, st>>>(x, d, n, S, L.q, L.t, npt, np, slack, max_iter, vscene, amin,
                                                         true, list, nlist);
    }
    cudaMemcpyAsync(alpha_h, amin_d, sizeof(double) * ns, cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) return check_launch("gipc_ccd_max_step: sync");
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
    return find_contacts_impl(ctx, x, rest_x, n, *srf, dhat, stencils, eps_x, capacity, count_h, false, nullptr,
                              nullptr, (cudaStream_t)stream, 1, false);
}

extern "C" gipc_status gipc_ccd_max_step(gipc_ctx* ctx, const double* x, const double* d, int64_t n,
                                         const gipc_surface* srf, double slack, double* alpha_h, void* stream) {
    using namespace gipc;
    if (!ctx || !srf || !alpha_h || !x || !d) return fail(GIPC_ERR_INVALID_ARG, "gipc_ccd_max_step: null pointer");
    if (n < 0 || !(slack > 0.0 && slack < 1.0)) return fail(GIPC_ERR_INVALID_ARG, "gipc_ccd_max_step: need 0 < slack < 1");
    return ccd_impl(ctx, x, d, n, *srf, slack, alpha_h, (cudaStream_t)stream, nullptr, 1, nullptr, false);
}
