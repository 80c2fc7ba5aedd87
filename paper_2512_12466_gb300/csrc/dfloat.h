// Double-float arithmetic for the FP64 table march: a value is the unevaluated sum
// h + l of two floats (about 48 significant bits), carried on the FP32 pipe, which on
// GB300 is 64 times wider than the FP64 one. Built from error-free transformations:
// Knuth's two-sum (TAOCP vol. 2, 4.2.2), Dekker's fast two-sum for |a| >= |b| and
// Dekker's exact product (Dekker 1971), whose rounding error a fused multiply-add
// returns exactly. Every operation is an explicit round-to-nearest intrinsic, so
// nothing is contracted or reassociated by the compiler.
#pragma once

namespace nyx {

struct dflt {
    float h, l;
};

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dflt df_two_sum(const float a, const float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// s + e = a + b exactly when the exponent of a is at least that of b (Dekker)
__device__ __forceinline__ dflt df_fast_two_sum(const float a, const float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a b: the head product, its exact error and the two cross terms. The pair is left
// unnormalised (|l| up to about 2^-22 |h|), which the next product or sum absorbs;
// relative error below about 2^-45.
__device__ __forceinline__ dflt df_mul(const dflt a, const dflt b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return {p, e};
}

// a + b for any signs: heads by Knuth's two-sum, tails added to its error, renormalised
__device__ __forceinline__ dflt df_add(const dflt a, const dflt b)
{
    const dflt s = df_two_sum(a.h, b.h);
    return df_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}

// a 2^n, exactly while both parts stay normal
__device__ __forceinline__ dflt df_scale(const dflt a, const int n)
{
    const float m = __uint_as_float((unsigned)(127 + n) << 23);
    return {__fmul_rn(a.h, m), __fmul_rn(a.l, m)};
}

// a - b where 0 <= b <= 7/8 a (a budget less a segment's share of it): the heads by Dekker's fast
// two-sum, exact since |b.h| < |a.h|, the tails added to its error, renormalised
__device__ __forceinline__ dflt df_sub_part(const dflt a, const dflt b)
{
    const dflt s = df_fast_two_sum(a.h, -b.h);
    const float t = __fadd_rn(s.l, __fsub_rn(a.l, b.l));
    return df_fast_two_sum(s.h, t);
}

// 1 / x for x in [1, 2) as a double-float: the hardware's approximate reciprocal, one Newton step
// r + r (1 - x r) for the head, and the residual (1 - x r) r for the tail (relative error below
// about 2^-45)
__device__ __forceinline__ dflt df_rcp12(const dflt x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.h));
    r = __fmaf_rn(r, __fmaf_rn(-x.h, r, 1.0f), r);
    return {r, __fmul_rn(__fmaf_rn(-x.l, r, __fmaf_rn(-x.h, r, 1.0f)), r)};
}

// A positive normal double as a double-float mantissa in [1, 2) and its unbiased exponent:
// the head holds the leading 24 bits, the tail the remaining 29 rounded to 24 (error below
// 2^-48 of the value). Zero and subnormals are outside its domain (callers test x > 0).
__device__ __forceinline__ dflt df_mant(const double x, int& ex)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    ex = (int)(hw >> 20) - 1023;
    const float h = __uint_as_float(0x3f800000u | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const float l = __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), 2.220446049250313e-16f);   // 2^-52
    return {h, l};
}

// A non-negative double below 2^127 as a double-float, head = its leading 24 bits. Values
// below 2^-74 keep only the head (a relative error up to 2^-24 that the callers tolerate:
// they pass optical depths, whose error there only enters the rate factor, and segment
// lengths, which are never that short); values below 2^-126 read as 0.
__device__ __forceinline__ dflt df_of(const double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)(hw >> 20);
    if (e < 897) return {0.f, 0.f};
    const float h = __uint_as_float(((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    const float l = e >= 949 ? __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)(e - 948) << 23))
                             : 0.f;
    return {h, l};
}

// df_of for a positive double in [2^-74, 2^127), without the range tests (segment lengths: the
// integer traversal makes every segment longer than about 2^-46 cells)
__device__ __forceinline__ dflt df_of_len(const double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
    const int e = (int)(hw >> 20);
    return {__uint_as_float(((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29)),
            __fmul_rn(__uint2float_rn(lw & 0x1fffffffu), __uint_as_float((unsigned)(e - 948) << 23))};
}

// x 2^e2 as a double, exactly: float to double by re-biasing the exponent and shifting the
// mantissa (no FP64 instruction); zero and subnormal floats take the conversion.
__device__ __forceinline__ double widen_scaled(const float x, const int e2)
{
    const unsigned u = __float_as_uint(x);
    const unsigned mag = u & 0x7fffffffu;
    if (mag - 0x00800000u < 0x7f000000u) {              // normal and finite
        const unsigned hi = ((mag >> 3) + ((unsigned)(896 + e2) << 20)) | (u & 0x80000000u);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if (mag == 0u) return 0.0;
    const double d = (double)x;
    return __longlong_as_double(__double_as_longlong(d) + (long long)e2 * (1LL << 52));
}

// (h + l) 2^e2 rounded to double (one FP64 addition)
__device__ __forceinline__ double df_to_double(const dflt a, const int e2)
{
    return __dadd_rn(widen_scaled(a.h, e2), widen_scaled(a.l, e2));
}

// The same for h + l >= 0 without the FP64 unit: renormalise (|l| <= 2^-24 h), take h's double
// exactly, and add l counted in units of that double's last place, 2^(E_h - 52), as a 64-bit
// integer: l 2^(52 - E_h) is below 2^28 in magnitude and rounds to the nearest unit. The result is
// within one unit of the last place of h + l, except where the renormalised head is a power of two
// and the tail negative: the sum then lies in the binade below, whose last place is half as large,
// so only half the tail is subtracted (an error of at most 2^-26 of the value, for about one deposit
// in 10^7). Heads outside [2^-75, 2^127) (where the scale factor leaves the float range) take
// df_to_double.
__device__ __forceinline__ double df_to_double_pos(const dflt a, const int e2)
{
    const dflt n = df_fast_two_sum(a.h, a.l);
    const unsigned u = __float_as_uint(n.h);
    const int eh = (int)(u >> 23) - 127;
    if (eh < -75 || eh > 126 || (u >> 31)) return df_to_double(a, e2);
    const unsigned hi = (u >> 3) + ((unsigned)(896 + e2) << 20);
    const long long bits = (long long)(((unsigned long long)hi << 32) | (unsigned long long)(u << 29));
    const int units = __float2int_rn(__fmul_rn(n.l, __uint_as_float((unsigned)(179 - eh) << 23)));   // l 2^(52 - E_h)
    return __longlong_as_double(bits + (long long)units);
}

}  // namespace nyx
