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

// ------------------------------------------------------------------ packed pairs
// sm_100 and later execute two FP32 operations per instruction on a 64-bit register
// pair (add/sub/mul/fma .f32x2).  The FMA pipe does the same work per lane either way
// (a measured GB300 probe: 37 T lane-operations/s for both), but the instruction count
// halves, which is what bounds the issue-limited DF32 Dslash.  f2 holds (x, y) with x
// in the low 32 bits.
typedef unsigned long long f2;

__device__ __forceinline__ f2 f2_pack(float x, float y) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2 v, float &x, float &y) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v));
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
// sign flips and swaps are bit operations
__device__ __forceinline__ f2 neg2(f2 a) { return a ^ 0x8000000080000000ull; }
__device__ __forceinline__ f2 negx2(f2 a) { return a ^ 0x0000000080000000ull; }
__device__ __forceinline__ f2 negy2(f2 a) { return a ^ 0x8000000000000000ull; }
__device__ __forceinline__ f2 swap2(f2 a) { return (a >> 32) | (a << 32); }
__device__ __forceinline__ f2 bcastx(f2 a) {
    float x, y;
    f2_unpack(a, x, y);
    return f2_pack(x, x);
}
__device__ __forceinline__ f2 bcasty(f2 a) {
    float x, y;
    f2_unpack(a, x, y);
    return f2_pack(y, y);
}

// A complex df number with its parts packed: hi = (re.hi, im.hi), lo = (re.lo, im.lo)
// (the DF32 memory layout of one component, so a 128-bit load fills it directly).
struct cd2 {
    f2 hi, lo;
};

// a + b and a - b: Knuth's TwoSum on the two high parts at once, as for df
__device__ __forceinline__ cd2 cd_add(cd2 a, cd2 b) {
    const f2 s = add2(a.hi, b.hi);
    const f2 bb = sub2(s, a.hi);
    const f2 e = add2(sub2(a.hi, sub2(s, bb)), sub2(b.hi, bb));
    return cd2{s, add2(add2(a.lo, b.lo), e)};
}
__device__ __forceinline__ cd2 cd_sub(cd2 a, cd2 b) {
    const f2 s = sub2(a.hi, b.hi);
    const f2 bb = sub2(s, a.hi);
    const f2 e = sub2(sub2(a.hi, sub2(s, bb)), add2(b.hi, bb));
    return cd2{s, add2(sub2(a.lo, b.lo), e)};
}
__device__ __forceinline__ cd2 cd_neg_if(cd2 a, bool neg) {
    const f2 m = neg ? 0x8000000080000000ull : 0ull;
    return cd2{a.hi ^ m, a.lo ^ m};
}
// i a
__device__ __forceinline__ cd2 cd_muli(cd2 a) { return cd2{negx2(swap2(a.hi)), negx2(swap2(a.lo))}; }
__device__ __forceinline__ cd2 cd_conj(cd2 a) { return cd2{negy2(a.hi), negy2(a.lo)}; }
__device__ __forceinline__ cd2 cd_twice(cd2 a) { return cd2{add2(a.hi, a.hi), add2(a.lo, a.lo)}; }

// A real df number x broadcast to both halves, with the negated high part kept for
// the TwoProduct below.
struct bc2 {
    f2 hi, lo, nhi;
};
__device__ __forceinline__ bc2 bc_re(cd2 a) {
    const f2 h = bcastx(a.hi);
    return bc2{h, bcastx(a.lo), neg2(h)};
}
__device__ __forceinline__ bc2 bc_im(cd2 a) {
    const f2 h = bcasty(a.hi);
    return bc2{h, bcasty(a.lo), neg2(h)};
}

// s + x y for a broadcast real x and a complex y: per half the FMA TwoProduct of the
// high parts, q = -fl(x.hi y.hi) and its exact error, plus the cross terms, then the
// TwoSum of s.hi and -q (as a difference, so no negation is needed).
__device__ __forceinline__ cd2 cd_mac(cd2 s, const bc2 &x, cd2 y) {
    const f2 q = mul2(x.nhi, y.hi);
    f2 e = fma2(x.hi, y.hi, q);
    e = fma2(x.hi, y.lo, e);
    e = fma2(x.lo, y.hi, e);
    const f2 t = sub2(s.hi, q);
    const f2 bb = sub2(t, s.hi);
    const f2 err = sub2(sub2(s.hi, sub2(t, bb)), add2(q, bb));
    return cd2{t, add2(add2(s.lo, e), err)};
}
// x y alone
__device__ __forceinline__ cd2 cd_mul(const bc2 &x, cd2 y) {
    const f2 q = mul2(x.nhi, y.hi);
    f2 e = fma2(x.hi, y.hi, q);
    e = fma2(x.hi, y.lo, e);
    e = fma2(x.lo, y.hi, e);
    return cd2{neg2(q), e};
}

}  // namespace wd
