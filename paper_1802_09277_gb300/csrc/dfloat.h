// Double-float ("float-float") numbers: x = hi + lo with |lo| <= ulp(hi)/2,
// about 48 significant bits from FP32 arithmetic.  GB300 runs FP32 at ~60x
// its FP64 rate, so an FP64-accurate stencil in double-float is faster than
// one in FP64.  Error-free transformations: Knuth's TwoSum and the FMA-based
// TwoProduct (exact product error); the sums and products below are the
// classical double-float ("sloppy") add and multiply, each with a relative
// error of a few units of 2^-48.  Device arithmetic uses the _rn intrinsics
// so that no multiply and add are contracted into an FMA behind our back.
#pragma once

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ explicit operator double() const { return (double)hi + (double)lo; }
};

#ifdef __CUDACC__
__device__ __forceinline__ dfloat df_add(dfloat a, dfloat b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float hi = __fadd_rn(s, e);
    return dfloat(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

__device__ __forceinline__ dfloat df_mul(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact error of the leading product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float hi = __fadd_rn(p, e);
    return dfloat(hi, __fsub_rn(e, __fsub_rn(hi, p)));
}

// double -> (hi, lo) by bit manipulation (integer and FP32 operations only):
// hi = the sign, exponent and leading 23 fraction bits (truncated), lo = the
// remaining 29 fraction bits scaled by ulp(hi).  Outside |d| in
// [2^-100, 2^127) (and for zero) it falls back to the FP64 conversion.
__device__ __forceinline__ dfloat df_from_double(double d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int ef = e - 1023 + 127;  // float exponent field of hi
    if (ef < 24 || ef > 254) return dfloat(d);
    const unsigned sign = h32 & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)ef << 23) | ((h32 & 0xfffffu) << 3) | (l32 >> 29));
    // ulp(hi) * 2^-29 = 2^(ef - 127 - 23 - 29), built as a float (ef - 52 >= 1 is not
    // guaranteed, so scale in two steps)
    const float s1 = __uint_as_float((unsigned)(ef - 23) << 23);  // 2^(ef - 127 - 23)
    const float lo = __fmul_rn(__fmul_rn(__uint2float_rn(l32 & 0x1fffffffu), 0x1p-29f), s1);
    return dfloat(hi, sign ? -lo : lo);
}

// (hi, lo) -> double: each float widened exactly by bit manipulation, one FP64 add
__device__ __forceinline__ double df_widen(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned ex = (u >> 23) & 0xffu;
    if (ex == 0u && (u & 0x7fffffffu) == 0u)  // +-0
        return __longlong_as_double((long long)((unsigned long long)(u & 0x80000000u) << 32));
    if (ex == 0u || ex == 0xffu) return (double)x;  // subnormal, inf / nan
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(ex - 127u + 1023u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

__device__ __forceinline__ double df_to_double(dfloat a) {
    return __dadd_rn(df_widen(a.hi), df_widen(a.lo));
}

// acc + a * b in one step: the leading product's exact error by FMA, the
// cross terms added to it, one TwoSum with the accumulator, renormalisation
__device__ __forceinline__ dfloat df_fma(dfloat acc, dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    float t = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    t = __fadd_rn(t, __fadd_rn(acc.lo, e));
    const float hi = __fadd_rn(s, t);
    return dfloat(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = df_add(a, b); }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = df_add(a, -b); }
#endif
