// sg_df.cuh -- double-float arithmetic for the compensated FP32 plans
// (SG_F32X2): a value is the unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi) / 2, about 48 significant bits, computed on the FP32 pipes.
// The error-free transformations are the published ones: Knuth's TwoSum and
// Dekker's FastTwoSum for sums, the FMA form of Dekker's TwoProduct for
// products, combined as in Hida, Li and Bailey's double-double library
// (2001; the "sloppy" sum, whose error is bounded by about 2^-47 (|a| + |b|),
// which is the normwise bound an FFT's error analysis needs).  Every float
// operation is an explicitly rounded intrinsic, so that the compiler cannot
// contract a product and a sum of a transformation into one FMA.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

struct dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    // nearest double-float of a double (hi = fl(d), lo = fl(d - hi))
    __host__ __device__ constexpr dfloat(double d) : hi((float)d), lo((float)(d - (double)(float)d)) {}
    __host__ __device__ constexpr dfloat(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ constexpr dfloat(int i) : hi((float)i), lo((float)((double)i - (double)(float)i)) {}
};

struct dfloat2 {
    dfloat x, y;
};

__host__ __device__ inline double df_to_double(dfloat a) { return (double)a.hi + (double)a.lo; }

#ifdef __CUDACC__
// s + e = a + b exactly (Knuth's TwoSum)
__device__ __forceinline__ dfloat df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker's FastTwoSum)
__device__ __forceinline__ dfloat df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return dfloat(s, e);
}
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b)
{
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) { return a + (-b); }
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // p + e = a.hi b.hi exactly (TwoProduct)
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_two_sum(p, e);
}
// one Newton-type correction of the float quotient (long division by b.hi)
__device__ __forceinline__ dfloat operator/(dfloat a, dfloat b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const dfloat r = a - dfloat(q1, 0.0f) * b;
    const float q2 = __fdiv_rn(r.hi, b.hi);
    return df_fast_two_sum(q1, q2);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// loads and stores of 16-byte values (the read-only path and the cache-hint forms)
__device__ __forceinline__ dfloat2 sg_ldg(const dfloat2* p)
{
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    return dfloat2{dfloat(v.x, v.y), dfloat(v.z, v.w)};
}
__device__ __forceinline__ dfloat sg_ldg(const dfloat* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return dfloat(v.x, v.y);
}
__device__ __forceinline__ dfloat df_shfl_xor(dfloat v, int lane_mask)
{
    return dfloat(__shfl_xor_sync(0xffffffffu, v.hi, lane_mask), __shfl_xor_sync(0xffffffffu, v.lo, lane_mask));
}
#endif
