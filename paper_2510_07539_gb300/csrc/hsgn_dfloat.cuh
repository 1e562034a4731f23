// hsgn_dfloat.cuh -- double-float arithmetic for the FP64-class windowed stage.
//
// A value is the unevaluated sum hi + lo of two single-precision numbers with
// |lo| <= about one ulp of hi: a 48-bit significand with the exponent range of
// single precision. Every operation runs on the single-precision pipe, which
// on sm_103a issues 58 times as many operations per clock as the double-
// precision pipe; a double-float operation costs 4 to 14 of them.
//
// Building blocks, each a published error-free transformation:
//  * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e = a + b exactly, any order;
//  * FastTwoSum (Dekker 1971): s + e = a + b exactly when |a| >= |b|, used to
//    renormalise a pair;
//  * the product a*b = p + e exactly with one fused multiply-add
//    (e = fma(a, b, -p)).
// Sum: TwoSum of the high parts plus the low parts, renormalised (error about
// 2^-47 of |a| + |b|). Product: the exact product of the high parts plus the
// two cross terms (about 2^-46 relative), not renormalised. Reciprocal and
// quotient: one correction of the single-precision quotient by its exact
// residual, i.e. one Newton step from a 23-bit start (about 2^-46 relative).
//
// The helpers compile for the host too (plain C++, no contraction of a*b + c
// into a fused multiply-add: the operations are spelled with explicit
// rounding on the device and the host build must use -ffp-contract=off).
#pragma once

#include <cstdint>
#include <cmath>

#ifdef __CUDACC__
#define HSGN_HD __host__ __device__ __forceinline__
#else
#define HSGN_HD inline
#endif

namespace hsgn {

// Single-precision operations that the compiler may not fuse or reorder.
HSGN_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
HSGN_HD float f_sub(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fsub_rn(a, b);
#else
    return a - b;
#endif
}
HSGN_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
HSGN_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return std::fmaf(a, b, c);
#endif
}
// 1/x to about one ulp: the hardware approximation plus one Newton-Raphson
// step on the device (e = 1 - x r, r' = r + r e); the rounded quotient on the host.
HSGN_HD float f_rcp(float x) {
#ifdef __CUDA_ARCH__
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return __fmaf_rn(r, __fmaf_rn(-x, r, 1.f), r);
#else
    return 1.f / x;
#endif
}

struct dfl {
    float hi, lo;
    dfl() = default;
    // from one float (explicit, so that a double is never narrowed silently:
    // doubles go through dfl_of)
    HSGN_HD explicit constexpr dfl(float h) : hi(h), lo(0.f) {}
    HSGN_HD constexpr dfl(float h, float l) : hi(h), lo(l) {}
};

HSGN_HD dfl dfl_make(float hi, float lo) { return dfl(hi, lo); }

// x > 0 and finite, from the high part's bit pattern (false for +-0, negatives,
// +Inf and NaN).
HSGN_HD bool pos_finite_hi(float x) {
#ifdef __CUDA_ARCH__
    const unsigned b = __float_as_uint(x);
#else
    unsigned b;
    __builtin_memcpy(&b, &x, sizeof b);
#endif
    return (b - 1u) < 0x7F7FFFFFu;
}

// The pair nearest to a double (host constants and state conversion).
HSGN_HD dfl dfl_of(double x) {
    const float hi = (float)x;
    return dfl_make(hi, (float)(x - (double)hi));
}
HSGN_HD double dfl_to_double(dfl a) { return (double)a.hi + (double)a.lo; }

// s + e = a + b exactly (TwoSum).
HSGN_HD void two_sum_f(float a, float b, float& s, float& e) {
    s = f_add(a, b);
    const float bb = f_sub(s, a);
    e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
}

// (s, e) renormalised so that s = fl(s + e) (FastTwoSum, |s| >= |e|).
HSGN_HD dfl renorm(float s, float e) {
    const float h = f_add(s, e);
    return dfl_make(h, f_sub(e, f_sub(h, s)));
}

HSGN_HD dfl operator-(dfl a) { return dfl_make(-a.hi, -a.lo); }

HSGN_HD dfl operator+(dfl a, dfl b) {
    float s, e;
    two_sum_f(a.hi, b.hi, s, e);
    return renorm(s, f_add(e, f_add(a.lo, b.lo)));
}
HSGN_HD dfl operator-(dfl a, dfl b) { return a + (-b); }

// a + b left unrenormalised: the exact sum of the high parts (TwoSum) with the
// low parts added to its error term, three operations fewer than the sum
// above. The value carries the same error (about 2^-48 of |a| + |b|); the low
// part may reach a few ulps of the high part, or exceed it where the high
// parts cancel, and every operation here takes such a pair as an input
// (products, quotients, reciprocals and roots form the leading term from the
// high part and fold the low part into a correction; sums take both parts
// exactly). Values that are stored as a state, tested for sign or compared
// are formed with the renormalised operations.
HSGN_HD dfl add_u(dfl a, dfl b) {
    float s, e;
    two_sum_f(a.hi, b.hi, s, e);
    return dfl_make(s, f_add(e, f_add(a.lo, b.lo)));
}
HSGN_HD dfl sub_u(dfl a, dfl b) { return add_u(a, -b); }

// a + b with an error of about 2^-47 of |a + b| rather than of |a| + |b|:
// TwoSum of both the high and the low parts (for differences of close values,
// whose cancellation the plain sum would leave at the operands' rounding).
// The last low-part term is added without a final renormalisation (as add_u:
// the value is the same, the pair may carry a low part of a few ulps).
HSGN_HD dfl add_acc(dfl a, dfl b) {
    float s1, s2, t1, t2;
    two_sum_f(a.hi, b.hi, s1, s2);
    two_sum_f(a.lo, b.lo, t1, t2);
    const dfl u = renorm(s1, f_add(s2, t1));
    return dfl_make(u.hi, f_add(u.lo, t2));
}
HSGN_HD dfl sub_acc(dfl a, dfl b) { return add_acc(a, -b); }

// a + x for a single float x, unrenormalised (as add_u).
HSGN_HD dfl add_f(dfl a, float x) {
    float s, e;
    two_sum_f(a.hi, x, s, e);
    return dfl_make(s, f_add(e, a.lo));
}

// Products, reciprocals and quotients return the pair unrenormalised: the low
// part is the rounding error of the high part plus terms of relative size
// 2^-24 (|lo| <= about 2^-22 |hi|), which every operation here accepts as an
// input (they use hi for the leading products and lo only in correction
// terms); sums renormalise.
HSGN_HD dfl operator*(dfl a, dfl b) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    return dfl_make(p, e);
}

// a * x for a single float x (exact constants such as small integers).
HSGN_HD dfl mul_f(dfl a, float x) {
    const float p = f_mul(a.hi, x);
    float e = f_fma(a.hi, x, -p);
    e = f_fma(a.lo, x, e);
    return dfl_make(p, e);
}

// a * 2^k: exact.
HSGN_HD dfl scale(dfl a, float pow2) { return dfl_make(f_mul(a.hi, pow2), f_mul(a.lo, pow2)); }

// a * b + c with one renormalisation.
HSGN_HD dfl fma(dfl a, dfl b, dfl c) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    float s, t;
    two_sum_f(p, c.hi, s, t);
    return renorm(s, f_add(t, f_add(e, c.lo)));
}

// a * b + c without the final renormalisation (as add_u).
HSGN_HD dfl fma_u(dfl a, dfl b, dfl c) {
    const float p = f_mul(a.hi, b.hi);
    float e = f_fma(a.hi, b.hi, -p);
    e = f_fma(a.hi, b.lo, e);
    e = f_fma(a.lo, b.hi, e);
    float s, t;
    two_sum_f(p, c.hi, s, t);
    return dfl_make(s, f_add(t, f_add(e, c.lo)));
}

// 1/a: r = 1/a.hi to one ulp, then r + r (1 - a r) with the residual formed
// exactly from the high part (fma) and corrected by the low part.
HSGN_HD dfl rcp(dfl a) {
    const float r = f_rcp(a.hi);
    float e = f_fma(-a.hi, r, 1.f);
    e = f_fma(-a.lo, r, e);
    return dfl_make(r, f_mul(e, r));
}

// a / b: q0 = a.hi / b.hi to one ulp, corrected by the residual a - b q0.
HSGN_HD dfl operator/(dfl a, dfl b) {
    const float r = f_rcp(b.hi);
    const float q0 = f_mul(a.hi, r);
    const float p = f_mul(b.hi, q0);
    const float pe = f_fma(b.hi, q0, -p);
    float res = f_add(f_sub(f_sub(a.hi, p), pe), a.lo);
    res = f_fma(-b.lo, q0, res);
    return dfl_make(q0, f_mul(res, r));
}

// h^2 - m for h close to sqrt(m) (m/h^2 within a factor 2 of 1), with an
// error of about 2^-47 of the result: the exact square of h.hi (TwoProd), the
// exact product 2 h.hi h.lo, h.hi^2 - m.hi exact by Sterbenz's lemma, and the
// small terms summed with TwoSum.
HSGN_HD dfl sq_minus(dfl h, dfl m) {
    const float p = f_mul(h.hi, h.hi);
    const float pe = f_fma(h.hi, h.hi, -p);
    const float h2 = f_add(h.hi, h.hi);
    const float q = f_mul(h2, h.lo);
    const float qe = f_fma(h2, h.lo, -q);
    const float s1 = f_sub(p, m.hi);
    float a, b, c, d, s, t;
    two_sum_f(pe, q, a, b);
    two_sum_f(a, -m.lo, c, d);
    const float small = f_add(f_add(b, d), f_fma(h.lo, h.lo, qe));
    two_sum_f(s1, c, s, t);
    return renorm(s, f_add(t, small));
}

HSGN_HD dfl dabs(dfl a) { return a.hi < 0.f ? -a : a; }
HSGN_HD dfl dmax(dfl a, dfl b) {
    return (a.hi > b.hi || (a.hi == b.hi && a.lo >= b.lo)) ? a : b;
}

}  // namespace hsgn
