// dd.cuh -- complex double double arithmetic on the device (the refinement
// of endpoints in refine.cu and the double double tracker in track_dd.cu).
//
// Double double numbers are unevaluated sums hi + lo with |lo| <= ulp(hi)/2
// (Hida, Li and Bailey, the paper's [HLB00]).  Error-free transforms:
// Knuth's TwoSum and the fused multiply-add form of TwoProduct
// (a*b - fl(a*b) is exact as fma(a, b, -fl(a*b))).
#pragma once
#include "phc_internal.h"

namespace phc {

struct dd {
    double hi, lo;
};
struct cdd {
    dd re, im;
};

__device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = a + b;
    const double bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b)
{
    const double s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dd two_prod(double a, double b)
{
    const double p = a * b;
    return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd dd_add(dd a, dd b)
{
    dd s = two_sum(a.hi, b.hi);
    const dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_mul(dd a, dd b)
{
    dd p = two_prod(a.hi, b.hi);
    p.lo = fma(a.hi, b.lo, fma(a.lo, b.hi, p.lo));
    return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_div(dd a, dd b)
{
    const double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul({q1, 0.0}, b));
    const double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul({q2, 0.0}, b));
    const double q3 = r.hi / b.hi;
    return dd_add(quick_two_sum(q1, q2), {q3, 0.0});
}

__device__ __forceinline__ cdd cdd_from(double2 z) { return {{z.x, 0.0}, {z.y, 0.0}}; }
__device__ __forceinline__ cdd cdd_add(cdd a, cdd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_sub(cdd a, cdd b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_mul(cdd a, cdd b)
{
    return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)), dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
__device__ __forceinline__ cdd cdd_div(cdd a, cdd b)
{
    const dd den = dd_add(dd_mul(b.re, b.re), dd_mul(b.im, b.im));
    const dd nr = dd_add(dd_mul(a.re, b.re), dd_mul(a.im, b.im));
    const dd ni = dd_sub(dd_mul(a.im, b.re), dd_mul(a.re, b.im));
    return {dd_div(nr, den), dd_div(ni, den)};
}
__device__ __forceinline__ double cdd_abs1(cdd a) { return fabs(a.re.hi) + fabs(a.im.hi); }
__device__ __forceinline__ double cdd_absinf(cdd a)
{
    const double u = fabs(a.re.hi), v = fabs(a.im.hi);
    return u > v ? u : v;
}

__device__ __forceinline__ cdd cdd_scale(double a, cdd z) { return {dd_mul({a, 0.0}, z.re), dd_mul({a, 0.0}, z.im)}; }
__device__ __forceinline__ cdd cdd_neg(cdd a) { return {dd_neg(a.re), dd_neg(a.im)}; }

}  // namespace phc
