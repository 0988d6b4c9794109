// Double-FP32 ("df32") arithmetic: a real number is carried as the unevaluated
// sum hi + lo of two floats, giving a 48-bit significand on the FP32 pipes.
//
// GB300 executes FP32 FMAs at 64 times the FP64 rate (128 vs 2 per SM and
// clock), so a stencil that is FP64-bound in native arithmetic can reach its
// memory roof in df32 with about 12 FP32 instructions per FP64 operation.
//
// Building blocks (published error-free transformations):
//   * Knuth's TwoSum: s = a + b, e = (a - (s - bb)) + (b - bb), bb = s - a,
//     with s + e == a + b exactly;
//   * TwoProduct with FMA: p = a * b, e = fma(a, b, -p), p + e == a * b exactly.
// Sums keep the TwoSum error of the high parts and add the low parts in FP32;
// products keep the exact high product and the two cross terms and drop
// lo * lo.  Results are not renormalised after each operation: hi + lo stays
// an exact-to-rounding representation and the low part only grows to a few
// ulps of the inputs, which bounds the absolute error of every result by
// about 2^-46 times the magnitude of its inputs.  The library's tests check
// the Dslash in this arithmetic against the FP64 oracle at the FP64 tolerance.
#pragma once
#include <cuda_runtime.h>

namespace wd {

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit df(double d) {
        hi = __double2float_rn(d);
        lo = __double2float_rn(d - (double)hi);
    }
    __device__ __forceinline__ explicit df(int i) : hi((float)i), lo(0.f) {}
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
    __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

__device__ __forceinline__ df operator+(df a, df b) {
    const float s = __fadd_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    return df(s, __fadd_rn(__fadd_rn(a.lo, b.lo), e));
}

__device__ __forceinline__ df operator-(df a) { return df(-a.hi, -a.lo); }
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator*(df a, df b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df(p, e);
}

}  // namespace wd
