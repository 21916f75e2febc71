// sgl_dfl.cuh -- double-float arithmetic on the FP32 pipe.
//
// A double-float number is the unevaluated sum h + l of two binary32 numbers with |l| <= ulp(h)/2.
// Sums by TwoSum (Knuth), products by TwoProduct (Dekker; exact with a fused multiply-add), each
// renormalized by Fast2Sum: a relative rounding of about 2^-44 per operation.  Quotients and square
// roots take one correction step (Newton) from the binary32 result, with the residual formed
// exactly.  The rounded intrinsics keep the compiler from fusing or reordering the error terms.
#pragma once

#include <cuda_runtime.h>

namespace sgl {

struct dfl {
    float h, l;
    dfl() = default;
    __host__ __device__ constexpr dfl(float hh, float ll) : h(hh), l(ll) {}
    __host__ __device__ constexpr dfl(int v) : h((float)v), l(0.f) {}
    __host__ __device__ constexpr dfl(float v) : h(v), l(0.f) {}
    __host__ __device__ constexpr dfl(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
};
struct dfl2 { dfl x, y; };

__device__ __forceinline__ dfl fast_two_sum(float a, float b) {       // |a| >= |b| (else a rounding of b's size)
    const float s = __fadd_rn(a, b);
    return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    const float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));   // a.h + b.h = s + e exactly
    return fast_two_sum(s, __fadd_rn(e, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = fmaf(a.h, b.h, -p);                                      // a.h b.h = p + e exactly
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return fast_two_sum(p, e);
}
// product by a binary32 number
__device__ __forceinline__ dfl df_mul(dfl a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = fmaf(a.h, b, -p);
    e = fmaf(a.l, b, e);
    return fast_two_sum(p, e);
}
// a / b, b != 0: q = a.h / b.h, then q + (a - q b) / b.h with the residual a - q b exact to the
// rounding of its low part
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
    const float q = __fdiv_rn(a.h, b.h);
    const float p = __fmul_rn(q, b.h);
    const float pe = fmaf(q, b.h, -p);                                 // q b.h = p + pe exactly
    float r = __fsub_rn(a.h, p);                                       // exact when q is near a.h / b.h
    r = __fsub_rn(r, pe);
    r = __fadd_rn(r, a.l);
    r = fmaf(-q, b.l, r);
    return fast_two_sum(q, __fdiv_rn(r, b.h));
}
// sqrt(a), a >= 0: s = sqrt(a.h), then s + (a - s^2) / 2s
__device__ __forceinline__ dfl df_sqrt(dfl a) {
    if (!(a.h > 0.f)) return dfl(0.f, 0.f);
    const float s = __fsqrt_rn(a.h);
    const float p = __fmul_rn(s, s);
    const float pe = fmaf(s, s, -p);                                   // s^2 = p + pe exactly
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.h, p), pe), a.l);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}
// multiplication by 2^k, -126 <= k <= 127 (exact while neither part leaves the normal range)
__device__ __forceinline__ dfl df_scale2(dfl a, int k) {
    const float p2 = __int_as_float((k + 127) << 23);
    return dfl(__fmul_rn(a.h, p2), __fmul_rn(a.l, p2));
}
__device__ __forceinline__ double df_to_double(dfl a) { return (double)a.h + (double)a.l; }

// x 2^-E as a double-float, from the bit pattern alone (integer operations, no FP64 pipe): the
// leading 24 significand bits give h, the other 29 (rounded to 24) give l.  Zero when x 2^-E lies
// below 2^-126 (subnormal doubles too); +-infinity (NaN for NaN) above the binary32 range.
__device__ __forceinline__ dfl df_split_bits(double x, int E = 0) {
    const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const int ex = (int)((bits >> 52) & 0x7ff);
    const int e = ex - 1023 - E;
    const unsigned sign = (unsigned)(bits >> 32) & 0x80000000u;
    const unsigned long long m = bits & 0xfffffffffffffull;
    if (ex == 0 || e < -126) return dfl(0.f, 0.f);
    if (e > 127) return dfl(__int_as_float((int)(sign | 0x7f800000u | (m ? 0x400000u : 0u))), 0.f);
    const float h = __int_as_float((int)(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29)));
    float l = 0.f;
    if (e >= -74) {
        const float v = __fmul_rn((float)(unsigned)(m & 0x1fffffffu), __int_as_float((e - 52 + 127) << 23));
        l = sign ? -v : v;
    }
    return dfl(h, l);
}

// a binary32 number as a binary64 one from its bit pattern (integer operations; subnormals -> 0)
__device__ __forceinline__ double f2d_bits(float f) {
    const unsigned u = (unsigned)__float_as_int(f);
    const unsigned ex = (u >> 23) & 0xff;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (ex == 0) return __longlong_as_double((long long)sign);
    const unsigned long long dex = ex == 0xff ? 0x7ffull : (unsigned long long)(ex - 127 + 1023);
    return __longlong_as_double((long long)(sign | (dex << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// h + l rounded to binary64 (one binary64 addition)
__device__ __forceinline__ double df_to_double_bits(dfl a) { return f2d_bits(a.h) + f2d_bits(a.l); }

// f 2^E as a binary64 number from the bit pattern (0 below the normal range, +-inf above it)
__device__ __forceinline__ double f2d_bits_scaled(float f, int E) {
    const unsigned u = (unsigned)__float_as_int(f);
    const int ex = (int)((u >> 23) & 0xff);
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    if (ex == 0) return __longlong_as_double((long long)sign);
    const int dex = ex == 0xff ? 0x7ff : ex - 127 + 1023 + E;
    if (dex <= 0) return __longlong_as_double((long long)sign);
    if (dex >= 0x7ff) return __longlong_as_double((long long)(sign | (0x7ffull << 52)));
    return __longlong_as_double((long long)(sign | ((unsigned long long)dex << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// (h + l) 2^E rounded to binary64
__device__ __forceinline__ double df_to_double_scaled(dfl a, int E) { return f2d_bits_scaled(a.h, E) + f2d_bits_scaled(a.l, E); }

// the exponent E with max 2^-E in [1, 2) from the bits of a non-negative binary64 max (0 when the
// max is zero, subnormal or not finite)
__device__ __forceinline__ int df_scale_exponent(const unsigned long long *bits) {
    if (!bits) return 0;
    const int ex = (int)((*bits >> 52) & 0x7ff);
    return (ex == 0 || ex == 0x7ff) ? 0 : ex - 1023;
}

}  // namespace sgl
