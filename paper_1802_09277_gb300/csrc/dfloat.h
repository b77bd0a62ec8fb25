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

// Bit casts usable on the host too (the conversions below are checked there
// against FP64 arithmetic).
__host__ __device__ __forceinline__ unsigned df_f2u(float x) {
#ifdef __CUDA_ARCH__
    return __float_as_uint(x);
#else
    unsigned u;
    __builtin_memcpy(&u, &x, 4);
    return u;
#endif
}
__host__ __device__ __forceinline__ float df_u2f(unsigned u) {
#ifdef __CUDA_ARCH__
    return __uint_as_float(u);
#else
    float x;
    __builtin_memcpy(&x, &u, 4);
    return x;
#endif
}
__host__ __device__ __forceinline__ unsigned long long df_d2u(double x) {
#ifdef __CUDA_ARCH__
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long u;
    __builtin_memcpy(&u, &x, 8);
    return u;
#endif
}
__host__ __device__ __forceinline__ double df_u2d(unsigned long long u) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)u);
#else
    double x;
    __builtin_memcpy(&x, &u, 8);
    return x;
#endif
}
__host__ __device__ __forceinline__ int df_clz64(unsigned long long x) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)x);
#else
    return x ? __builtin_clzll(x) : 64;
#endif
}

// The conversions between FP64 data and double-float use integer and FP32
// operations only, in every branch: GB300 runs FP64 instructions (and the
// FP64 conversions) at 1/64 of the FP32 rate, and a compiler that predicates
// a rare branch into straight-line code would issue them for every element.

// double -> (hi, lo): hi = the sign, exponent and leading 23 fraction bits
// (truncated), lo = the remaining 29 fraction bits (rounded to 24 bits) scaled
// by ulp(hi): 48 significant bits (2^-48 relative).  Zero maps to (+-0, 0), inf and nan to
// (inf / nan, 0), |d| >= 2^128 to (+-inf, 0); below 2^-100 lo loses bits to
// FP32's subnormal range, below 2^-103 only hi is kept (below FP32's normal
// range: +-0): absolute errors under 2^-126.
__host__ __device__ __forceinline__ dfloat df_from_double(double d) {
    const unsigned long long b = df_d2u(d);
    const unsigned h32 = (unsigned)(b >> 32), l32 = (unsigned)b;
    const unsigned sign = h32 & 0x80000000u;
    const int e = (int)((h32 >> 20) & 0x7ffu);
    const int ef = e - 1023 + 127;  // float exponent field of hi
    const unsigned top = ((h32 & 0xfffffu) << 3) | (l32 >> 29);
    if (ef >= 24 && ef <= 254) {
        const float hi = df_u2f(sign | ((unsigned)ef << 23) | top);
        // float(m) of the 29 low bits, rounded once: its two parts are exact as
        // the fraction field of 2^23 + part, one FMA joins them
        const unsigned m = l32 & 0x1fffffffu;
        const float fh = df_u2f(0x4b000000u | (m >> 23)) - 8388608.f;
        const float fl = df_u2f(0x4b000000u | (m & 0x7fffffu)) - 8388608.f;
#ifdef __CUDA_ARCH__
        const float fm = __fmaf_rn(fh, 8388608.f, fl);
        // ulp(hi) * 2^-29 = 2^(ef - 127 - 23 - 29), applied in two exact steps
        const float lo = __fmul_rn(__fmul_rn(fm, 0x1p-29f), df_u2f((unsigned)(ef - 23) << 23));
#else
        const float fm = (float)((double)fh * 8388608.0 + (double)fl);
        const float lo = (fm * 0x1p-29f) * df_u2f((unsigned)(ef - 23) << 23);
#endif
        return dfloat(hi, sign ? -lo : lo);
    }
    if (e == 0x7ff)  // inf, nan
        return dfloat(df_u2f(sign | 0x7f800000u | (((h32 & 0xfffffu) | l32) ? 0x400000u : 0u)), 0.f);
    if (ef > 254) return dfloat(df_u2f(sign | 0x7f800000u), 0.f);
    if (ef >= 1) return dfloat(df_u2f(sign | ((unsigned)ef << 23) | top), 0.f);
    return dfloat(df_u2f(sign), 0.f);
}

// float -> double, exactly, from its bits
__host__ __device__ __forceinline__ double df_widen(float x) {
    const unsigned u = df_f2u(x);
    const unsigned long long s = (unsigned long long)(u & 0x80000000u) << 32;
    const unsigned ex = (u >> 23) & 0xffu;
    unsigned m = u & 0x7fffffu;
    if (ex == 0xffu) return df_u2d(s | 0x7ff0000000000000ull | ((unsigned long long)m << 29));
    if (ex != 0u)
        return df_u2d(s | ((unsigned long long)(ex + 896u) << 52) | ((unsigned long long)m << 29));
    if (m == 0u) return df_u2d(s);  // +-0
    // subnormal: m 2^-149, normalised (m < 2^23 has at least 9 leading zeros)
    const int k = df_clz64((unsigned long long)m) - 40;  // shift that brings bit 23 up
    m = (m << k) & 0x7fffffu;
    return df_u2d(s | ((unsigned long long)(897 - k) << 52) | ((unsigned long long)m << 29));
}

// (hi, lo) -> the double nearest to hi + lo (round to nearest, ties to even:
// what one FP64 add of the widened parts gives) from integer operations, for
// two normal floats; with a zero, subnormal, inf or nan part, hi alone is
// widened.
__host__ __device__ __forceinline__ double df_to_double(dfloat a) {
    unsigned uh = df_f2u(a.hi), ul = df_f2u(a.lo);
    int eh = (int)((uh >> 23) & 0xffu), el = (int)((ul >> 23) & 0xffu);
    if (eh == 0 || eh == 0xff || el == 0 || el == 0xff) return df_widen(a.hi);
    int d = eh - el;
    if (d <= -24) {  // lo is the larger part: the same sum with the roles swapped
        const unsigned t = uh;
        uh = ul;
        ul = t;
        eh = el;
        el = eh - (-d);
        d = -d;
    }
    if (d < 24) {  // not normalised: the exact sum (at most 49 bits) in units of the smaller ulp
        const long long mh = (long long)((uh & 0x7fffffu) | 0x800000u);
        const long long mlo = (long long)((ul & 0x7fffffu) | 0x800000u);
        const long long va = (d >= 0 ? (mh << d) : mh) * ((uh >> 31) ? -1 : 1);
        const long long vb = (d >= 0 ? mlo : (mlo << -d)) * ((ul >> 31) ? -1 : 1);
        const long long v = va + vb;
        if (v == 0) return 0.0;
        const unsigned long long mag = (unsigned long long)(v < 0 ? -v : v);
        const int L = 63 - df_clz64(mag);  // <= 48
        const int emin = d >= 0 ? el : eh;
        return df_u2d((v < 0 ? 0x8000000000000000ull : 0ull) |
                      (unsigned long long)(L + emin - 150 + 1023) << 52 |
                      ((mag << (52 - L)) & 0xfffffffffffffull));
    }
    // magnitudes in units of 2^(eh - 127 - 23 - 38): A = mh 2^38 (bit 61 set)
    const unsigned long long A = (unsigned long long)((uh & 0x7fffffu) | 0x800000u) << 38;
    const unsigned long long ml = (unsigned long long)((ul & 0x7fffffu) | 0x800000u);
    unsigned long long B;
    bool sticky;
    if (d <= 38) {
        B = ml << (38 - d);  // < 2^38
        sticky = false;
    } else if (d - 38 < 24) {
        B = ml >> (d - 38);
        sticky = (ml & ((1ull << (d - 38)) - 1ull)) != 0ull;
    } else {
        B = 0ull;
        sticky = true;
    }
    unsigned long long R;
    if (((uh ^ ul) >> 31) == 0u) {
        R = A + B;  // the true value is R (+ a fraction if sticky)
    } else {
        R = A - B;
        if (sticky) R -= 1ull;  // the true value is R + a fraction in (0, 1)
    }
    const int L = 63 - df_clz64(R);  // 60 .. 62
    const int sh = L - 52;           // 8 .. 10 bits below the double's last bit
    unsigned long long q = R >> sh;
    const unsigned long long rem = R & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (sticky || (q & 1ull)))) ++q;
    int E = (eh - 127) + (L - 61);  // unbiased exponent of the result
    if (q >> 53) {                  // rounding carried into a new bit
        q >>= 1;
        ++E;
    }
    return df_u2d((unsigned long long)(uh & 0x80000000u) << 32 |
                  (unsigned long long)(E + 1023) << 52 | (q & 0xfffffffffffffull));
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
