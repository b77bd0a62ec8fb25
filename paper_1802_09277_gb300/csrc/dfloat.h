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

__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) { return df_add(a, b); }
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return df_add(a, -b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) { return df_mul(a, b); }
__device__ __forceinline__ dfloat &operator+=(dfloat &a, dfloat b) { return a = df_add(a, b); }
__device__ __forceinline__ dfloat &operator-=(dfloat &a, dfloat b) { return a = df_add(a, -b); }
#endif
