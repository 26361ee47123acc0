// ff.cuh -- float-float ("double-single") arithmetic for the contraction stages, with the conversions
// to and from binary64 done on the integer pipe.
//
// A value is an unevaluated pair hi + lo of binary32 numbers.  Products use the exact FMA-based
// TwoProduct and sums Knuth's TwoSum (error-free transformations, Dekker 1971; Knuth TAOCP vol. 2,
// 4.2.2), so a short dot product of pairs carries about 2^-46 relative error with respect to the sum of
// the absolute values of its terms -- far inside the 1e-12 gate, at a fraction of the FP64 pipe's cost
// on a part whose FP64 rate is 1/64 of its FP32 rate.  The binary64 <-> pair conversions touch no FP64
// unit: they re-pack exponent and significand bits with 32-bit integer operations.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace tl {

struct ff {
    float hi, lo;
};

// a + b = s + e exactly (any magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Split a binary64 value into hi (its leading 24 significant bits, truncated) and lo (the remaining 29
// bits rounded to binary32): hi + lo = x within 2^-48 |x| (the pair carries 48 significant bits).  Magnitudes below 2^-74 lose lo and below
// 2^-126 become zero (absolute error < 2^-97); `big` is set for |x| >= 2^63, infinities and NaN, which
// the caller must not feed to pair arithmetic (products of two values below 2^63 stay finite).
__device__ __forceinline__ ff split_ff(double x, uint32_t &big)
{
    const uint32_t hw = (uint32_t)__double2hiint(x), lw = (uint32_t)__double2loint(x);
    const uint32_t E = (hw >> 20) & 0x7ffu;
    const uint32_t sign = hw & 0x80000000u;
    // (hw:lw) << 3: the low 9 exponent bits and the leading 23 fraction bits; rebias 1023 -> 127 by
    // subtracting 896 << 23, taken modulo 2^32 (= 0xC0000000).
    const uint32_t t = __funnelshift_l(lw, hw, 3);
    const uint32_t hib = ((t - 0xC0000000u) & 0x7fffffffu) | sign;
    const uint32_t r = lw & 0x1fffffffu;               // the 29 fraction bits below hi
    // exact binary32 images of r >> 6 and r & 63 via the 2^23 magic constant, then one rounding
    const float rh = __fsub_rn(__uint_as_float(0x4b000000u | (r >> 6)), 8388608.0f);
    const float rl = __fsub_rn(__uint_as_float(0x4b000000u | (r & 63u)), 8388608.0f);
    const float rf = __fmaf_rn(rh, 64.0f, rl);
    const float scale = __uint_as_float(sign | ((E - 948u) << 23));   // +-2^(E - 1075)
    ff v;
    v.hi = (E >= 897u) ? __uint_as_float(hib) : __uint_as_float(sign);
    v.lo = (E >= 949u) ? __fmul_rn(rf, scale) : 0.0f;
    big |= (E > 1023u + 62u) ? 1u : 0u;
    return v;
}

// The range test of split_ff alone (1 when |x| >= 2^63, inf or nan).
__device__ __forceinline__ uint32_t out_of_ff_range(double x)
{
    return ((((uint32_t)__double2hiint(x)) >> 20) & 0x7ffu) > 1023u + 62u ? 1u : 0u;
}

// hi + lo -> binary64 (truncated below the 53rd bit; error < 1 ulp).  Requires a normalised pair,
// |lo| <= ulp(hi)/2, as produced by two_sum, and a finite hi (the callers' range checks guarantee it).
// Branch-free; a zero hi gives a signed zero.
__device__ __forceinline__ double merge_ff(ff v)
{
    const uint32_t hb = __float_as_uint(v.hi), lb = __float_as_uint(v.lo);
    const uint32_t sign = hb & 0x80000000u;
    const uint32_t Eh = (hb >> 23) & 0xffu, El = (lb >> 23) & 0xffu;
    const uint32_t Mh = (hb & 0x7fffffu) | 0x800000u;
    const uint32_t Ml = (El != 0u) ? ((lb & 0x7fffffu) | 0x800000u) : 0u;
    const uint32_t d = Eh - El;                            // >= 24 for a normalised pair
    // lo aligned to the 29 low bits of the 53-bit significand
    const uint32_t L = (d >= 53u) ? 0u : ((d <= 29u) ? (Ml << (29u - d)) : (Ml >> (d - 29u)));
    const bool borrow = (L != 0u) && ((hb ^ lb) & 0x80000000u);   // opposite signs: borrow from hi
    uint32_t hiM = borrow ? Mh - 1u : Mh;
    uint32_t loM = borrow ? (1u << 29) - L : L;
    uint32_t E = Eh + (1023u - 127u);
    const bool renorm = hiM < 0x800000u;                   // hi was a power of two
    hiM = renorm ? ((hiM << 1) | (loM >> 28)) : hiM;
    loM = renorm ? ((loM << 1) & 0x1fffffffu) : loM;
    E = renorm ? E - 1u : E;
    const uint32_t hw = (Eh == 0u) ? sign : (sign | (E << 20) | ((hiM & 0x7fffffu) >> 3));
    const uint32_t lw = (Eh == 0u) ? 0u : (((hiM & 7u) << 29) | loM);
    return __hiloint2double((int)hw, (int)lw);
}

// sum_{l<3} a_l b_l as a normalised pair.  Each product is hi*hi exactly (TwoProduct) plus the two
// cross terms; the lo*lo term (< 2^-48 |a b|) is dropped.  The three leading products are summed with
// TwoSum, and all low-order parts are accumulated in binary32.
__device__ __forceinline__ ff dot3_ff(const ff &a0, const ff &b0, const ff &a1, const ff &b1, const ff &a2,
                                      const ff &b2)
{
    const float p0 = __fmul_rn(a0.hi, b0.hi), p1 = __fmul_rn(a1.hi, b1.hi), p2 = __fmul_rn(a2.hi, b2.hi);
    float q0 = __fmaf_rn(a0.hi, b0.hi, -p0), q1 = __fmaf_rn(a1.hi, b1.hi, -p1), q2 = __fmaf_rn(a2.hi, b2.hi, -p2);
    q0 = __fmaf_rn(a0.hi, b0.lo, __fmaf_rn(a0.lo, b0.hi, q0));
    q1 = __fmaf_rn(a1.hi, b1.lo, __fmaf_rn(a1.lo, b1.hi, q1));
    q2 = __fmaf_rn(a2.hi, b2.lo, __fmaf_rn(a2.lo, b2.hi, q2));
    float s, t0, t1;
    two_sum(p0, p1, s, t0);
    two_sum(s, p2, s, t1);
    const float lo = __fadd_rn(__fadd_rn(__fadd_rn(q0, q1), __fadd_rn(q2, t0)), t1);
    // TwoSum rather than the cheaper FastTwoSum: when the leading products cancel, |lo| may exceed
    // |s|, and merge_ff needs |lo| <= ulp(hi) / 2, which TwoSum guarantees for any inputs.
    ff r;
    two_sum(s, lo, r.hi, r.lo);
    return r;
}

// Accumulator for sums of pair products: s collects the leading products with TwoSum, lo every
// low-order part (TwoProduct errors, cross terms, TwoSum errors) in binary32.
struct ffacc {
    float s, lo;
};

// The exact leading product a.hi*b.hi and the low-order part of a*b (TwoProduct error plus the two
// cross terms; the lo*lo term, below 2^-48 |a b|, is dropped).
__device__ __forceinline__ void ff_prod(const ff &a, const ff &b, float &p, float &q)
{
    p = __fmul_rn(a.hi, b.hi);
    q = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, __fmaf_rn(a.hi, b.hi, -p)));
}

__device__ __forceinline__ ffacc acc_from(const ff &c) { return ffacc{c.hi, c.lo}; }

__device__ __forceinline__ ffacc acc_prod(const ff &a, const ff &b)
{
    ffacc A;
    ff_prod(a, b, A.s, A.lo);
    return A;
}

// A += a * b
__device__ __forceinline__ void acc_add_prod(ffacc &A, const ff &a, const ff &b)
{
    float p, q, s, t;
    ff_prod(a, b, p, q);
    two_sum(A.s, p, s, t);
    A.s = s;
    A.lo = __fadd_rn(A.lo, __fadd_rn(q, t));
}

// A += c (a pair)
__device__ __forceinline__ void acc_add(ffacc &A, const ff &c)
{
    float s, t;
    two_sum(A.s, c.hi, s, t);
    A.s = s;
    A.lo = __fadd_rn(A.lo, __fadd_rn(c.lo, t));
}

// The accumulated sum as a normalised pair.
__device__ __forceinline__ ff acc_result(const ffacc &A)
{
    ff r;
    two_sum(A.s, A.lo, r.hi, r.lo);
    return r;
}

// Exact scalings of a pair by powers of two and its negation (binary32 operations that are exact away
// from the subnormal range, which the callers' range checks keep clear of).
__device__ __forceinline__ ff ff_scale(const ff &a, float pow2) { return ff{a.hi * pow2, a.lo * pow2}; }
__device__ __forceinline__ ff ff_neg(const ff &a) { return ff{-a.hi, -a.lo}; }

// a - b for pairs, normalised.
__device__ __forceinline__ ff sub_ff(const ff &a, const ff &b)
{
    float s, t;
    two_sum(a.hi, -b.hi, s, t);
    const float lo = __fadd_rn(t, __fsub_rn(a.lo, b.lo));
    ff r;
    two_sum(s, lo, r.hi, r.lo);
    return r;
}

// A pair with |lo| <= ulp(hi) / 2 (split_ff's pairs may have |lo| up to ulp(hi)).
__device__ __forceinline__ ff normalize_ff(const ff &a)
{
    ff r;
    two_sum(a.hi, a.lo, r.hi, r.lo);
    return r;
}

}  // namespace tl
