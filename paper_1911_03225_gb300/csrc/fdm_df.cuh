// fdm_df.cuh -- double-word ("double-float") arithmetic on FP32 hardware.
//
// A value is hi + lo with two floats, |lo| <= ulp(hi)/2, about 48 significant bits.  GB300
// executes FP32 at 58x the FP64 rate, so FP64-accurate kernels run faster on this type than
// on native doubles.  Building blocks, all from the published literature:
//   TwoSum (Knuth, TAOCP vol. 2), FastTwoSum (Dekker 1971), TwoProd with an FMA;
//   double-word + double-word (Joldes, Muller, Popescu, ACM TOMS 2017): the "sloppy"
//   version (their Algorithm 5, 11 flops), whose error is a few u^2 (|x| + |y|) (u = 2^-24)
//   -- relative when the signs agree, absolute under cancellation.  Every
//   value this library adds already carries a representation error of u^2 times its own
//   magnitude, so the 20-flop relative-error version buys no accuracy here;
//   double-word x double-word (same paper, Algorithm 12; <= 5 u^2) and
//   double-word x float (Algorithm 9);
//   reciprocal and reciprocal square root by one Newton step on the double word from a
//   float seed (relative error ~1e-14).
// Every float operation uses an explicitly rounded intrinsic so the compiler can neither
// contract nor reassociate the error-free transforms.
#pragma once
#include <cuda_runtime.h>

namespace fdm {

struct alignas(8) df {   // one 64-bit access per value
    float hi, lo;
    df() = default;
    __host__ __device__ __forceinline__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ __forceinline__ explicit df(int v) : hi((float)v), lo(0.f) {}
    __host__ __device__ __forceinline__ explicit df(float v) : hi(v), lo(0.f) {}
    __host__ __device__ __forceinline__ explicit df(double v) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    }
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

#if defined(__CUDA_ARCH__)
#define DF_ADD(a, b) __fadd_rn(a, b)
#define DF_SUB(a, b) __fsub_rn(a, b)
#define DF_MUL(a, b) __fmul_rn(a, b)
#define DF_FMA(a, b, c) __fmaf_rn(a, b, c)
#else
#define DF_ADD(a, b) df_host_add(a, b)
#define DF_SUB(a, b) df_host_sub(a, b)
#define DF_MUL(a, b) df_host_mul(a, b)
#define DF_FMA(a, b, c) df_host_fma(a, b, c)
float df_host_add(float a, float b);
float df_host_sub(float a, float b);
float df_host_mul(float a, float b);
float df_host_fma(float a, float b, float c);
#endif

// error-free transforms
__host__ __device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = DF_ADD(a, b);
    float bb = DF_SUB(s, a);
    e = DF_ADD(DF_SUB(a, DF_SUB(s, bb)), DF_SUB(b, bb));
}
__host__ __device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {  // |a| >= |b|
    s = DF_ADD(a, b);
    e = DF_SUB(b, DF_SUB(s, a));
}
__host__ __device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = DF_MUL(a, b);
    e = DF_FMA(a, b, -p);
}

__host__ __device__ __forceinline__ df operator+(df x, df y) {
    float sh, sl, zh, zl;
    two_sum(x.hi, y.hi, sh, sl);
    float v = DF_ADD(x.lo, y.lo);
    float w = DF_ADD(sl, v);
    fast_two_sum(sh, w, zh, zl);
    return df(zh, zl);
}
__host__ __device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo); }
__host__ __device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__host__ __device__ __forceinline__ df operator*(df x, df y) {
    float ch, cl1, zh, zl;
    two_prod(x.hi, y.hi, ch, cl1);
    float tl0 = DF_MUL(x.lo, y.lo);
    float tl1 = DF_FMA(x.hi, y.lo, tl0);
    float cl2 = DF_FMA(x.lo, y.hi, tl1);
    float cl3 = DF_ADD(cl1, cl2);
    fast_two_sum(ch, cl3, zh, zl);
    return df(zh, zl);
}
__host__ __device__ __forceinline__ df mul_f(df x, float y) {
    float ch, cl1, zh, zl;
    two_prod(x.hi, y, ch, cl1);
    float cl3 = DF_FMA(x.lo, y, cl1);
    fast_two_sum(ch, cl3, zh, zl);
    return df(zh, zl);
}
__host__ __device__ __forceinline__ df& operator+=(df& x, df y) { x = x + y; return x; }

__host__ __device__ __forceinline__ bool operator>(df x, df y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__host__ __device__ __forceinline__ bool operator<(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__host__ __device__ __forceinline__ bool operator==(df x, df y) { return x.hi == y.hi && x.lo == y.lo; }
__host__ __device__ __forceinline__ bool operator!=(df x, df y) { return !(x == y); }

// float seeds: IEEE-rounded on the host, special-function unit plus one FP32 Newton step
// on the device
__host__ __device__ __forceinline__ float rcp_seed(float a) {
#if defined(__CUDA_ARCH__)
    return __frcp_rn(a);
#else
    return 1.0f / a;
#endif
}
__host__ __device__ __forceinline__ float rsqrt_seed(float a) {
#if defined(__CUDA_ARCH__)
    float r = rsqrtf(a);
    return DF_MUL(r, DF_FMA(DF_MUL(-0.5f, a), DF_MUL(r, r), 1.5f));
#else
    return 1.0f / __builtin_sqrtf(a);
#endif
}

// 1/y for y != 0: r1 = r0 + r0 (1 - y r0)
__host__ __device__ __forceinline__ df df_rcp(df y) {
    float r0 = rcp_seed(y.hi);
    df p = mul_f(y, r0);
    float e = DF_SUB(DF_SUB(1.0f, p.hi), p.lo);  // 1 - p.hi is exact (p.hi ~ 1)
    float s, t;
    two_sum(r0, DF_MUL(r0, e), s, t);
    return df(s, t);
}
__host__ __device__ __forceinline__ df operator/(df x, df y) { return x * df_rcp(y); }

// 1/sqrt(x) for x > 0: r1 = r0 + r0 (1 - x r0^2) / 2
__host__ __device__ __forceinline__ df df_rsqrt(df x) {
    float r0 = rsqrt_seed(x.hi);
    float q, qe;
    two_prod(r0, r0, q, qe);
    df h = x * df(q, qe);
    float e = DF_SUB(DF_SUB(1.0f, h.hi), h.lo);
    float s, t;
    two_sum(r0, DF_MUL(DF_MUL(0.5f, r0), e), s, t);
    return df(s, t);
}

// exact scaling by a power of two (no rounding for normal values)
__host__ __device__ __forceinline__ df scale2(df x, float p2) { return df(DF_MUL(x.hi, p2), DF_MUL(x.lo, p2)); }

// precision-typed helpers used by the generic kernels
__host__ __device__ __forceinline__ df tmin(df a, df b) { return (b < a) ? b : a; }
__host__ __device__ __forceinline__ df tmax(df a, df b) { return (b > a) ? b : a; }
__host__ __device__ __forceinline__ df tabs(df a) { return (a.hi < 0.f) ? -a : a; }
__host__ __device__ __forceinline__ df trsqrt(df x) { return df_rsqrt(x); }
__host__ __device__ __forceinline__ df trcp(df x) { return df_rcp(x); }
__host__ __device__ __forceinline__ df thalf(df x) { return scale2(x, 0.5f); }

}  // namespace fdm
