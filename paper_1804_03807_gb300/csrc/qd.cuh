// qd.cuh -- quad double arithmetic for the device (and the host): a value is
// an unevaluated sum x0 + x1 + x2 + x3 of doubles of decreasing magnitude,
// about 4 x 53 bits (Section 5 and Table 2 of the paper run the solver in
// quad double; the paper's arithmetic is [HLB00]'s).
//
// Every operation forms its exact result as terms grouped by level (level k
// of order u^k relative to the leading term, u = 2^-53): TwoSum and the
// fused-multiply-add TwoProduct are exact, so the terms of levels 0..3 are
// carried exactly and only level 4 and beyond is summed in plain double.
// renorm5 then turns the five level sums into four components: error-free
// bottom-up TwoSum passes leave the rounded total in the first slot and the
// exact rest below it; the first slot is kept and the passes repeat on the
// rest.  Errors are of order u^4 relative to the operands.
#pragma once

#include <cuda_runtime.h>

namespace phc {

struct qd {
    double x0, x1, x2, x3;
};
struct cqd {
    qd re, im;
};

// s + e = a + b exactly (Knuth).  __dadd_rn keeps the compiler from
// reassociating the correction on the device.
__host__ __device__ __forceinline__ void qd_two_sum(double a, double b, double &s, double &e)
{
#ifdef __CUDA_ARCH__
    s = __dadd_rn(a, b);
    const double bb = __dsub_rn(s, a);
    e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
#else
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
#endif
}

// p + e = a b exactly (fused multiply-add).
__host__ __device__ __forceinline__ void qd_two_prod(double a, double b, double &p, double &e)
{
#ifdef __CUDA_ARCH__
    p = __dmul_rn(a, b);
#else
    p = a * b;
#endif
    e = fma(a, b, -p);
}

// One bottom-up pass over t[lo..M-1]: t[lo] receives the rounded sum, the
// rest the exact errors (the sum of the slots does not change).
template <int M>
__host__ __device__ __forceinline__ void qd_pass(double (&t)[M], int lo)
{
#pragma unroll
    for (int i = M - 1; i > lo; i--) {
        double s, e;
        qd_two_sum(t[i - 1], t[i], s, e);
        t[i - 1] = s;
        t[i] = e;
    }
}

// Four components of e0 + e1 + e2 + e3 + e4 (terms of levels 0..4).
__host__ __device__ __forceinline__ qd renorm5(double e0, double e1, double e2, double e3, double e4)
{
    double t[5] = {e0, e1, e2, e3, e4};
    qd_pass<5>(t, 0);
    qd_pass<5>(t, 0);
    qd_pass<5>(t, 1);
    qd_pass<5>(t, 1);
    qd_pass<5>(t, 2);
    qd_pass<5>(t, 2);
    return {t[0], t[1], t[2], t[3] + t[4]};
}

__host__ __device__ __forceinline__ qd qd_from(double a) { return {a, 0.0, 0.0, 0.0}; }
__host__ __device__ __forceinline__ qd qd_neg(qd a) { return {-a.x0, -a.x1, -a.x2, -a.x3}; }

__host__ __device__ __forceinline__ qd qd_add(qd a, qd b)
{
    double s0, c0, s1, c1, c2, s2, c3, c4, s3, c5;
    qd_two_sum(a.x0, b.x0, s0, c0);  // level 0, its error to level 1
    qd_two_sum(a.x1, b.x1, s1, c1);  // level 1
    qd_two_sum(s1, c0, s1, c2);
    qd_two_sum(a.x2, b.x2, s2, c3);  // level 2
    qd_two_sum(s2, c1, s2, c4);
    qd_two_sum(s2, c2, s2, c5);
    s3 = a.x3 + b.x3 + c3 + c4 + c5;  // level 3 (its rounding is of level 4)
    return renorm5(s0, s1, s2, s3, 0.0);
}

__host__ __device__ __forceinline__ qd qd_sub(qd a, qd b) { return qd_add(a, qd_neg(b)); }

__host__ __device__ __forceinline__ qd qd_mul(qd a, qd b)
{
    double p0, q0, p1, q1, p2, q2, p3, q3, p4, q4, p5, q5;
    qd_two_prod(a.x0, b.x0, p0, q0);  // level 0
    qd_two_prod(a.x0, b.x1, p1, q1);  // level 1
    qd_two_prod(a.x1, b.x0, p2, q2);
    qd_two_prod(a.x0, b.x2, p3, q3);  // level 2
    qd_two_prod(a.x1, b.x1, p4, q4);
    qd_two_prod(a.x2, b.x0, p5, q5);
    // level 1: p1 + p2 + q0, errors to level 2
    double s1, e1, e2;
    qd_two_sum(p1, p2, s1, e1);
    qd_two_sum(s1, q0, s1, e2);
    // level 2: p3 + p4 + p5 + q1 + q2 + e1 + e2, errors to level 3
    double s2, f1, f2, f3, f4, f5, f6;
    qd_two_sum(p3, p4, s2, f1);
    qd_two_sum(s2, p5, s2, f2);
    qd_two_sum(s2, q1, s2, f3);
    qd_two_sum(s2, q2, s2, f4);
    qd_two_sum(s2, e1, s2, f5);
    qd_two_sum(s2, e2, s2, f6);
    // level 3 (exact sum, its rounding error to level 4), level 4 in plain double
    double s3 = a.x0 * b.x3 + a.x1 * b.x2 + a.x2 * b.x1 + a.x3 * b.x0;
    double g1, g2, g3;
    qd_two_sum(s3, q3 + q4 + q5, s3, g1);
    qd_two_sum(s3, f1 + f2 + f3, s3, g2);
    qd_two_sum(s3, f4 + f5 + f6, s3, g3);
    const double s4 = a.x1 * b.x3 + a.x2 * b.x2 + a.x3 * b.x1 + g1 + g2 + g3;
    return renorm5(p0, s1, s2, s3, s4);
}

__host__ __device__ __forceinline__ qd qd_mul_d(qd a, double d)
{
    double p0, q0, p1, q1, p2, q2, p3, q3;
    qd_two_prod(a.x0, d, p0, q0);
    qd_two_prod(a.x1, d, p1, q1);
    qd_two_prod(a.x2, d, p2, q2);
    qd_two_prod(a.x3, d, p3, q3);
    double s1, e1, s2, e2, e3, s3, e4;
    qd_two_sum(p1, q0, s1, e1);  // level 1
    qd_two_sum(p2, q1, s2, e2);  // level 2
    qd_two_sum(s2, e1, s2, e3);
    qd_two_sum(p3, q2, s3, e4);  // level 3
    s3 += e2 + e3;
    return renorm5(p0, s1, s2, s3, q3 + e4);
}

// Long division: five quotient digits q_k = r_0 / b_0, r <- r - q_k b.
__host__ __device__ __forceinline__ qd qd_div(qd a, qd b)
{
    const double d0 = a.x0 / b.x0;
    qd r = qd_sub(a, qd_mul_d(b, d0));
    const double d1 = r.x0 / b.x0;
    r = qd_sub(r, qd_mul_d(b, d1));
    const double d2 = r.x0 / b.x0;
    r = qd_sub(r, qd_mul_d(b, d2));
    const double d3 = r.x0 / b.x0;
    r = qd_sub(r, qd_mul_d(b, d3));
    const double d4 = r.x0 / b.x0;
    // d0..d4 are of levels 0..4 (each the quotient of the exact rest)
    return renorm5(d0, d1, d2, d3, d4);
}

__host__ __device__ __forceinline__ cqd cqd_from(double re, double im) { return {qd_from(re), qd_from(im)}; }
__host__ __device__ __forceinline__ cqd cqd_add(cqd a, cqd b) { return {qd_add(a.re, b.re), qd_add(a.im, b.im)}; }
__host__ __device__ __forceinline__ cqd cqd_sub(cqd a, cqd b) { return {qd_sub(a.re, b.re), qd_sub(a.im, b.im)}; }
__host__ __device__ __forceinline__ cqd cqd_neg(cqd a) { return {qd_neg(a.re), qd_neg(a.im)}; }
__host__ __device__ __forceinline__ cqd cqd_mul(cqd a, cqd b)
{
    return {qd_sub(qd_mul(a.re, b.re), qd_mul(a.im, b.im)), qd_add(qd_mul(a.re, b.im), qd_mul(a.im, b.re))};
}
__host__ __device__ __forceinline__ cqd cqd_scale(double s, cqd a) { return {qd_mul_d(a.re, s), qd_mul_d(a.im, s)}; }
// a / b = a conj(b) / |b|^2
__host__ __device__ __forceinline__ cqd cqd_div(cqd a, cqd b)
{
    const qd d = qd_add(qd_mul(b.re, b.re), qd_mul(b.im, b.im));
    const qd nr = qd_add(qd_mul(a.re, b.re), qd_mul(a.im, b.im));
    const qd ni = qd_sub(qd_mul(a.im, b.re), qd_mul(a.re, b.im));
    return {qd_div(nr, d), qd_div(ni, d)};
}
// |.|_1 and max-norm of the leading parts (pivoting, step control)
__host__ __device__ __forceinline__ double cqd_abs1(cqd a) { return fabs(a.re.x0) + fabs(a.im.x0); }
__host__ __device__ __forceinline__ double cqd_absinf(cqd a)
{
    const double u = fabs(a.re.x0), v = fabs(a.im.x0);
    return u > v ? u : v;
}
__host__ __device__ __forceinline__ bool cqd_finite(cqd a)
{
    return isfinite(a.re.x0) && isfinite(a.re.x1) && isfinite(a.re.x2) && isfinite(a.re.x3) && isfinite(a.im.x0) &&
           isfinite(a.im.x1) && isfinite(a.im.x2) && isfinite(a.im.x3);
}

}  // namespace phc
