// tds_df.cuh -- float-pair ("double-float") arithmetic for the split-precision FP64 sweeps.
//
// GB300 issues FP64 arithmetic at 2 thread-operations per clock per SM against 128 for FP32, so a
// sweep that carries its recurrences as pairs of floats (value = h + l, |l| <= ulp(h) / 2, about
// 48 significant bits) on the FP32 pipes can outrun the native FP64 sweep, which is bound by the
// FP64 pipe (about 7.4 FP64 operations per point).  The building blocks are the error-free
// transformations of floating-point arithmetic (Knuth's two-sum, Dekker's fast two-sum, the
// FMA-based two-product), combined as in the double-word algorithms of Joldes, Muller and
// Popescu (ACM TOMS 2017) in their cheaper, "sloppy" forms: the error of a sum is bounded by
// about 2^-48 of the operands' magnitudes rather than of the result, which is what a recurrence
// whose terms have the size of its result needs.
//
// Every float operation here goes through the _rn intrinsics, so that the compiler never
// contracts a product and a sum into an FMA (that would break the error terms).
//
// Conversions between FP64 and float pairs use integer bit operations rather than the f64 <->
// f32 conversion instructions, which issue on the FP64 pipe on this part: the split keeps the
// top 24 bits of the significand in h and the next 24 in l; the join adds l to h's FP64
// encoding as an integer.  Values must lie in float's normal range with room for the low word:
// |x| in [2^-74, 2^126]; smaller magnitudes lose low-word bits (an absolute error below
// 2^-98), zero and subnormal floats map to zero.
#pragma once

#include <cstdint>

namespace tds {
namespace {

struct DF {
    float h, l;
    DF() = default;
    __device__ explicit DF(double x) {   // accurate split (FP64 arithmetic; constants, chunk ends)
        h = __double2float_rn(x);
        l = __double2float_rn(x - static_cast<double>(h));
    }
    __device__ explicit operator double() const { return static_cast<double>(h) + static_cast<double>(l); }
};

__device__ __forceinline__ DF df_make(float h, float l) {
    DF r;
    r.h = h;
    r.l = l;
    return r;
}

// |a| >= |b| (or a == 0): a + b = s + e exactly
__device__ __forceinline__ DF df_fast2(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// any a, b: a + b = s + e exactly
__device__ __forceinline__ DF df_two(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df_make(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ DF operator-(DF a) { return df_make(-a.h, -a.l); }

__device__ __forceinline__ DF operator+(DF x, DF y) {
    const DF s = df_two(x.h, y.h);
    return df_fast2(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ DF operator-(DF x, DF y) { return x + (-y); }

__device__ __forceinline__ DF &operator+=(DF &x, DF y) {
    x = x + y;
    return x;
}

__device__ __forceinline__ DF operator*(DF x, DF y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return df_fast2(p, e);
}

// a * b + c
__device__ __forceinline__ DF mad(DF a, DF b, DF c) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    const DF s = df_two(p, c.h);
    return df_fast2(s.h, __fadd_rn(s.l, __fadd_rn(e, c.l)));
}

// a1 * b1 + a2 * b2 + a3 * b3 with one renormalisation (the stencil products and the recurrence
// term of a forward row)
__device__ __forceinline__ DF dot3(DF a1, DF b1, DF a2, DF b2, DF a3, DF b3) {
    const float p1 = __fmul_rn(a1.h, b1.h), p2 = __fmul_rn(a2.h, b2.h), p3 = __fmul_rn(a3.h, b3.h);
    float e1 = __fmaf_rn(a1.h, b1.h, -p1);
    float e2 = __fmaf_rn(a2.h, b2.h, -p2);
    float e3 = __fmaf_rn(a3.h, b3.h, -p3);
    e1 = __fmaf_rn(a1.h, b1.l, e1);
    e2 = __fmaf_rn(a2.h, b2.l, e2);
    e3 = __fmaf_rn(a3.h, b3.l, e3);
    e1 = __fmaf_rn(a1.l, b1.h, e1);
    e2 = __fmaf_rn(a2.l, b2.h, e2);
    e3 = __fmaf_rn(a3.l, b3.h, e3);
    const DF s = df_two(p1, p2);
    const DF t = df_two(s.h, p3);
    const float err = __fadd_rn(__fadd_rn(s.l, t.l), __fadd_rn(__fadd_rn(e1, e2), e3));
    return df_fast2(t.h, err);
}

// a1 * b1 + a2 * b2 with one renormalisation
__device__ __forceinline__ DF dot2(DF a1, DF b1, DF a2, DF b2) {
    const float p1 = __fmul_rn(a1.h, b1.h), p2 = __fmul_rn(a2.h, b2.h);
    float e1 = __fmaf_rn(a1.h, b1.h, -p1);
    float e2 = __fmaf_rn(a2.h, b2.h, -p2);
    e1 = __fmaf_rn(a1.h, b1.l, e1);
    e2 = __fmaf_rn(a2.h, b2.l, e2);
    e1 = __fmaf_rn(a1.l, b1.h, e1);
    e2 = __fmaf_rn(a2.l, b2.h, e2);
    const DF s = df_two(p1, p2);
    return df_fast2(s.h, __fadd_rn(s.l, __fadd_rn(e1, e2)));
}

// FP64 -> float pair by bit operations: h is x with its significand cut to 24 bits (toward
// zero), l the remaining 29 bits rounded to 24 (one integer-to-float conversion, scaled by an
// exponent built from x's), so |x - (h + l)| <= 2^-48 |x|.  Exponents outside float's range give
// an infinite h (too large), a zero l (|x| below 2^-74) and a zero h (|x| below 2^-126).
__device__ __forceinline__ DF df_split(double x) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned hi = static_cast<unsigned>(b >> 32), lo = static_cast<unsigned>(b);
    const unsigned sign = hi & 0x80000000u;
    const int e = static_cast<int>((hi >> 20) & 0x7ffu);
    const unsigned mant = __funnelshift_l(lo, hi, 3) & 0x007fffffu;
    const int fe = e - 896;
    const float r = __uint2float_rn(lo & 0x1fffffffu);
    const int se = e - 948;
    const float scale = __uint_as_float(sign | (static_cast<unsigned>(se > 0 ? se : 0) << 23));
    DF o;
    o.h = (fe > 0) ? __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | mant) : __uint_as_float(sign);
    o.l = (fe > 0) ? __fmul_rn(r, scale) : 0.0f;
    if (fe > 254) o.h = __uint_as_float(sign | 0x7f800000u);
    return o;
}

// Exact FP64 image of a normal float (zero and subnormal floats give signed zero), by bit
// operations.
__device__ __forceinline__ double df_f2d(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned mag = u & 0x7fffffffu;
    unsigned hi = (u & 0x80000000u) | ((mag >> 3) + (896u << 20));
    unsigned lo = mag << 29;
    if (mag < 0x00800000u) { hi = u & 0x80000000u; lo = 0u; }
    return __hiloint2double(static_cast<int>(hi), static_cast<int>(lo));
}

// float pair -> FP64 by integer arithmetic on the FP64 encoding, without branches and without
// an FP64 instruction: the FP64 image of |h|, plus or minus l counted in units of the last
// place of that image (l's significand shifted left by 29 - (e_h - e_l); e_h - e_l >= 23, bits
// shifted out to the right are dropped, an error below 2^-52 of |h|).  When l has the opposite
// sign and h is a power of two the result lies in the binade below, whose last place is half as
// large, so l counts twice as many units there.  A zero h gives zero (in a normalised pair l is
// then zero too); subnormal words count as zero.
__device__ __forceinline__ double df_join(DF a) {
    const unsigned hb = __float_as_uint(a.h), lb = __float_as_uint(a.l);
    const unsigned hm = hb & 0x7fffffffu, lm = lb & 0x7fffffffu;
    const unsigned long long base = (static_cast<unsigned long long>((hm >> 3) + (896u << 20)) << 32) | (hm << 29);
    const int k = static_cast<int>(hm >> 23) - static_cast<int>(lm >> 23);
    const unsigned subm = static_cast<unsigned>(static_cast<int>(hb ^ lb) >> 31);
    const int sh = 29 - k + static_cast<int>(subm & ((hm & 0x007fffffu) == 0u ? 1u : 0u));
    const unsigned ml = (lm >= 0x00800000u) ? ((lm & 0x007fffffu) | 0x00800000u) : 0u;
    const unsigned u = (sh >= 0) ? (ml << sh) : __funnelshift_rc(ml, 0u, static_cast<unsigned>(-sh));
    const unsigned long long su = static_cast<unsigned long long>(static_cast<long long>(static_cast<int>(subm)));
    const unsigned long long r = base + ((static_cast<unsigned long long>(u) ^ su) - su);
    const unsigned long long bits = (hm < 0x00800000u) ? 0ull : r;
    return __longlong_as_double(static_cast<long long>(bits | (static_cast<unsigned long long>(hb & 0x80000000u) << 32)));
}

// The FP64 value's bits carried in a pair (input rows of the split sweeps, which take their
// differences in FP64 before splitting), and back.
__device__ __forceinline__ DF df_raw(double x) {
    return df_make(__int_as_float(__double2loint(x)), __int_as_float(__double2hiint(x)));
}
__device__ __forceinline__ double df_unraw(DF r) { return __hiloint2double(__float_as_int(r.l), __float_as_int(r.h)); }

} // namespace
} // namespace tds
