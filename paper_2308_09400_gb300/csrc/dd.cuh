// Double-double arithmetic built from error-free transformations.
//
//   two_sum      Knuth's branch-free exact addition: a + b = s + e exactly.
//   fast_two_sum Dekker's exact addition for |a| >= |b|.
//   two_prod     exact product via fused multiply-add: a * b = p + e exactly.
//   dd_add/mul/div  Dekker / Shewchuk-style double-double operations with
//                relative error of a few units of 2^-104.
//
// Used for the contact geometry: differences of float64 coordinates are formed
// exactly (two_sum), and the cross and dot products whose results cancel
// strongly (a point a distance 1e-7 from a unit triangle; two edges at 1e-7
// rad) are then carried in ~106-bit precision before rounding to float64.
#pragma once

struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd dd_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dd dd_fast_two_sum(double a, double b) {
    const double s = __dadd_rn(a, b);
    return {s, __dsub_rn(b, __dsub_rn(s, a))};
}

__device__ __forceinline__ dd dd_two_prod(double a, double b) {
    const double p = __dmul_rn(a, b);
    return {p, __fma_rn(a, b, -p)};
}

__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi);
    const dd t = dd_two_sum(a.lo, b.lo);
    s.lo = __dadd_rn(s.lo, t.hi);
    s = dd_fast_two_sum(s.hi, s.lo);
    s.lo = __dadd_rn(s.lo, t.lo);
    return dd_fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }

__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = dd_two_prod(a.hi, b.hi);
    p.lo = __fma_rn(a.hi, b.lo, p.lo);
    p.lo = __fma_rn(a.lo, b.hi, p.lo);
    return dd_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = dd_two_prod(a.hi, b);
    p.lo = __fma_rn(a.lo, b, p.lo);
    return dd_fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ dd dd_div(dd a, dd b) {
    const double q1 = __ddiv_rn(a.hi, b.hi);
    const dd r = dd_sub(a, dd_mul_d(b, q1));
    const double q2 = __ddiv_rn(r.hi, b.hi);
    return dd_fast_two_sum(q1, q2);
}

struct dd3 {
    dd x, y, z;
};

// exact difference a - b of two float64 points
__device__ __forceinline__ dd3 dd3_diff(const double* a, const double* b) {
    return {dd_two_sum(a[0], -b[0]), dd_two_sum(a[1], -b[1]), dd_two_sum(a[2], -b[2])};
}

__device__ __forceinline__ dd3 dd3_cross(const dd3& a, const dd3& b) {
    return {dd_sub(dd_mul(a.y, b.z), dd_mul(a.z, b.y)),
            dd_sub(dd_mul(a.z, b.x), dd_mul(a.x, b.z)),
            dd_sub(dd_mul(a.x, b.y), dd_mul(a.y, b.x))};
}

__device__ __forceinline__ dd dd3_dot(const dd3& a, const dd3& b) {
    return dd_add(dd_add(dd_mul(a.x, b.x), dd_mul(a.y, b.y)), dd_mul(a.z, b.z));
}

__device__ __forceinline__ void dd3_hi(const dd3& a, double* out) {
    out[0] = a.x.hi;
    out[1] = a.y.hi;
    out[2] = a.z.hi;
}
