// Internal types, field layouts and device helpers of libwd (sm_103a).
//
// Field layouts are described in include/wd.h.  Gauge layouts (per direction mu,
// blocks of Vs sites, complex entries row-major A*3+B):
//   F64 recon-18: 9 arrays of Vs double2            recon-12: 6 arrays (rows 0, 1)
//   F32 recon-18: 4 arrays of Vs float4 (entries 0-7) + 1 array of Vs float2 (entry 8)
//   F32 recon-12: 3 arrays of Vs float4
//   F16 recon-18: 2 arrays of Vs uint4 (8 half2 entries 0-7) + 1 array of Vs half2
//   F16 recon-12: 1 array of Vs uint4 (entries 0-3) + 1 array of Vs uint2 (entries 4-5)
//   recon-8 (entries 1, 2, 3 and the phases th0 = arg u[0], th6 = arg u[6]):
//   F64  4 arrays of Vs double2: u[1], u[2], u[3], (th0, th6)
//   DF32 4 arrays of Vs float4:  u[1], u[2], u[3], (th0.hi, th6.hi, th0.lo, th6.lo)
//   F32  2 arrays of Vs float4:  (u[1], u[2]), (u[3], th0, th6)
//   F16  1 array of Vs uint4:    u[1], u[2], u[3], (th0 / pi, th6 / pi) as half2
// Link entries have modulus <= 1 (unitary matrices), so FP16 links need no scale.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <string>
#include <vector>
#include <map>

#include "../../include/wd.h"
#include "df32.cuh"

namespace wd {

enum Prec { F64 = 0, F32 = 1, F16 = 2, DF32 = 3 };
constexpr int kNumPrec = 4;

constexpr int kSiteAlign = 64;
constexpr float kPiF = 3.14159265358979f;
inline size_t round_up(size_t a, size_t b) { return (a + b - 1) / b * b; }

// ------------------------------------------------------------------ complex
template <class R> struct C { R re, im; };

template <class R> __device__ __forceinline__ C<R> cmk(R a, R b) { return C<R>{a, b}; }
template <class R> __device__ __forceinline__ C<R> cadd(C<R> a, C<R> b) { return C<R>{a.re + b.re, a.im + b.im}; }
template <class R> __device__ __forceinline__ C<R> csub(C<R> a, C<R> b) { return C<R>{a.re - b.re, a.im - b.im}; }
template <class R> __device__ __forceinline__ C<R> cneg(C<R> a) { return C<R>{-a.re, -a.im}; }
template <class R> __device__ __forceinline__ C<R> cconj(C<R> a) { return C<R>{a.re, -a.im}; }
// i * a
template <class R> __device__ __forceinline__ C<R> cmuli(C<R> a) { return C<R>{-a.im, a.re}; }
template <class R> __device__ __forceinline__ C<R> cmul(C<R> a, C<R> b) {
    return C<R>{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class R> __device__ __forceinline__ C<R> cmulc(C<R> a, C<R> b) {
    return C<R>{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class R> __device__ __forceinline__ C<R> cscale(R s, C<R> a) { return C<R>{s * a.re, s * a.im}; }

// a * b + c as one fused multiply-add where the type has one
template <class R> __device__ __forceinline__ R madd(R a, R b, R c) { return a * b + c; }
template <> __device__ __forceinline__ double madd<double>(double a, double b, double c) { return fma(a, b, c); }
template <> __device__ __forceinline__ float madd<float>(float a, float b, float c) { return fmaf(a, b, c); }
// s + a * b and s + conj(a) * b as chains of four multiply-adds
template <class R> __device__ __forceinline__ C<R> cmac(C<R> s, C<R> a, C<R> b) {
    const R re = madd(-a.im, b.im, madd(a.re, b.re, s.re));
    const R im = madd(a.im, b.re, madd(a.re, b.im, s.im));
    return C<R>{re, im};
}
template <class R> __device__ __forceinline__ C<R> cmacc(C<R> s, C<R> a, C<R> b) {
    const R re = madd(a.im, b.im, madd(a.re, b.re, s.re));
    const R im = madd(-a.im, b.re, madd(a.re, b.im, s.im));
    return C<R>{re, im};
}

// ------------------------------------------------------------------ geometry
struct Geom {
    int L[4];
    int V;           // output sites of a launch (V, or V/2 on one parity)
    int Vs;          // site stride of field arrays (V rounded up to kSiteAlign)
    int stride[4];   // 1, Lx, Lx*Ly, Lx*Ly*Lz (full-lattice strides)
    int antiperiodic;
    int eo_parity;   // -1: full lattice; 0 / 1: checkerboard fields, output on this parity
    unsigned *dbg;   // debug builds: the context's word for the first out-of-range index
    int split_t;     // 1: one sub-lattice of a lattice split along t; the t hops that leave it
                     // (from the first slice backward, from the last slice forward) are omitted
};

// Index checks of debug builds (compiled with -DWD_DEBUG, in place of a memory checker):
// an index outside [0, n) is recorded in the context's debug word, the first one only, as
// 0x80000000 | code << 24 | (index & 0xffffff), and replaced by 0, so that the access
// stays inside the field.  Release builds compile the check away.
#ifdef WD_DEBUG
__device__ __forceinline__ int checked_index(const Geom &g, int i, int n, unsigned code) {
    if (i >= 0 && i < n) return i;
    if (g.dbg) atomicCAS(g.dbg, 0u, 0x80000000u | (code << 24) | ((unsigned)i & 0xffffffu));
    return 0;
}
#define WD_IDX(g, i, n, code) ::wd::checked_index((g), (i), (n), (code))
#else
#define WD_IDX(g, i, n, code) (i)
#endif

// ------------------------------------------------------------------ field sizes
inline size_t spinor_bytes(Prec p, int Vs) {
    switch (p) {
    case F64:
    case DF32: return (size_t)12 * Vs * 16;
    case F32: return (size_t)6 * Vs * 16;
    default: return round_up((size_t)3 * Vs * 16 + (size_t)Vs * 4, 256);
    }
}
inline size_t link_dir_bytes(Prec p, int recon, int Vs) {
    if (recon == 8) return (size_t)(p == F64 || p == DF32 ? 4 : p == F32 ? 2 : 1) * Vs * 16;
    if (p == F64 || p == DF32) return (size_t)(recon == 12 ? 6 : 9) * Vs * 16;
    if (p == F32) return recon == 12 ? (size_t)3 * Vs * 16 : (size_t)4 * Vs * 16 + (size_t)Vs * 8;
    return recon == 12 ? (size_t)Vs * 16 + (size_t)Vs * 8 : (size_t)2 * Vs * 16 + (size_t)Vs * 4;
}
inline size_t gauge_bytes(Prec p, int recon, int Vs) { return 4 * round_up(link_dir_bytes(p, recon, Vs), 256); }

// ------------------------------------------------------------------ precision traits
template <int P> struct Real { using T = float; };
template <> struct Real<F64> { using T = double; };
template <> struct Real<DF32> { using T = df; };

// Global loads: the read-only path (ld.global.nc) for fields a launch only reads,
// plain coherent loads (NC = false) for fields that other blocks of the same
// persistent launch write between grid barriers.
template <bool NC, class T> __device__ __forceinline__ T ldx(const T *p) {
    if constexpr (NC) return __ldg(p);
    else return *p;
}

// Spinor load/store: v[spin*3 + colour]
template <int P> struct SpinorIO;

template <> struct SpinorIO<F64> {
    using R = double;
    template <bool NC = true>
    static __device__ __forceinline__ void load(const void *base, int Vs, int s, C<R> (&v)[12]) {
        const double2 *p = reinterpret_cast<const double2 *>(base) + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            double2 t = ldx<NC>(p + (size_t)c * Vs);
            v[c] = C<R>{t.x, t.y};
        }
    }
    static __device__ __forceinline__ void store(void *base, int Vs, int s, const C<R> (&v)[12]) {
        double2 *p = reinterpret_cast<double2 *>(base) + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) p[(size_t)c * Vs] = make_double2(v[c].re, v[c].im);
    }
};

template <> struct SpinorIO<F32> {
    using R = float;
    template <bool NC = true>
    static __device__ __forceinline__ void load(const void *base, int Vs, int s, C<R> (&v)[12]) {
        const float4 *p = reinterpret_cast<const float4 *>(base) + s;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            float4 t = ldx<NC>(p + (size_t)j * Vs);
            v[2 * j] = C<R>{t.x, t.y};
            v[2 * j + 1] = C<R>{t.z, t.w};
        }
    }
    static __device__ __forceinline__ void store(void *base, int Vs, int s, const C<R> (&v)[12]) {
        float4 *p = reinterpret_cast<float4 *>(base) + s;
#pragma unroll
        for (int j = 0; j < 6; ++j) p[(size_t)j * Vs] = make_float4(v[2 * j].re, v[2 * j].im, v[2 * j + 1].re, v[2 * j + 1].im);
    }
};

// DF32: one float4 (re.hi, im.hi, re.lo, im.lo) per complex component, 12 arrays: a
// 128-bit load gives the high parts and the low parts as two aligned float pairs.
template <> struct SpinorIO<DF32> {
    using R = df;
    template <bool NC = true>
    static __device__ __forceinline__ void load(const void *base, int Vs, int s, C<R> (&v)[12]) {
        const float4 *p = reinterpret_cast<const float4 *>(base) + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            float4 t = ldx<NC>(p + (size_t)c * Vs);
            v[c] = C<R>{df(t.x, t.z), df(t.y, t.w)};
        }
    }
    static __device__ __forceinline__ void store(void *base, int Vs, int s, const C<R> (&v)[12]) {
        float4 *p = reinterpret_cast<float4 *>(base) + s;
#pragma unroll
        for (int c = 0; c < 12; ++c) p[(size_t)c * Vs] = make_float4(v[c].re.hi, v[c].im.hi, v[c].re.lo, v[c].im.lo);
    }
};

__device__ __forceinline__ float2 h2f(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}
__device__ __forceinline__ uint32_t f2h(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

template <> struct SpinorIO<F16> {
    using R = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ const float *norms(const void *base, int Vs) {
        return reinterpret_cast<const float *>(reinterpret_cast<const char *>(base) + (size_t)3 * Vs * 16);
    }
    template <bool NC = true>
    static __device__ __forceinline__ void load(const void *base, int Vs, int s, C<R> (&v)[12]) {
        const uint4 *p = reinterpret_cast<const uint4 *>(base) + s;
        const float nrm = ldx<NC>(norms(base, Vs) + s);
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 t = ldx<NC>(p + (size_t)j * Vs);
            float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), d = h2f(t.w);
            v[4 * j + 0] = C<R>{a.x * nrm, a.y * nrm};
            v[4 * j + 1] = C<R>{b.x * nrm, b.y * nrm};
            v[4 * j + 2] = C<R>{c.x * nrm, c.y * nrm};
            v[4 * j + 3] = C<R>{d.x * nrm, d.y * nrm};
        }
    }
    static __device__ __forceinline__ void store(void *base, int Vs, int s, const C<R> (&v)[12]) {
        float m = 0.f;
#pragma unroll
        for (int c = 0; c < 12; ++c) m = fmaxf(m, fmaxf(fabsf(v[c].re), fabsf(v[c].im)));
        // sites whose largest component is below 1e-37 are stored as zero: the
        // reciprocal of a smaller scale would overflow FP32
        const float inv = m > 1e-37f ? 1.0f / m : 0.f;
        if (!(m > 1e-37f)) m = 0.f;
        uint4 *p = reinterpret_cast<uint4 *>(base) + s;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            uint4 t;
            t.x = f2h(v[4 * j + 0].re * inv, v[4 * j + 0].im * inv);
            t.y = f2h(v[4 * j + 1].re * inv, v[4 * j + 1].im * inv);
            t.z = f2h(v[4 * j + 2].re * inv, v[4 * j + 2].im * inv);
            t.w = f2h(v[4 * j + 3].re * inv, v[4 * j + 3].im * inv);
            p[(size_t)j * Vs] = t;
        }
        float *nrm = const_cast<float *>(norms(base, Vs));
        nrm[s] = m;
    }
};

// Link load: u[A*3+B] of U_mu(s); recon-12 rebuilds row 2 = conj(row0 x row1).
template <class R> __device__ __forceinline__ void rebuild_row2(C<R> (&u)[9]) {
    u[6] = cconj(csub(cmul(u[1], u[5]), cmul(u[2], u[4])));
    u[7] = cconj(csub(cmul(u[2], u[3]), cmul(u[0], u[5])));
    u[8] = cconj(csub(cmul(u[0], u[4]), cmul(u[1], u[3])));
}

// recon-8: the 8-real parametrisation of an SU(3) matrix by its entries u01, u02,
// u10 and the phases of u00 and u20 (the compression of Clark et al., "Solving
// lattice QCD systems of equations using mixed precision solvers on GPUs", 2010).
// With rows a, b, c and n = |a1|^2 + |a2|^2 > 0, unitarity and det U = 1 give
//   a0 = sqrt(1 - n) e^{i th0},   c0 = sqrt(n - |b0|^2) e^{i th6},
//   b1 = -(a1 conj(a0) b0 + conj(a2 c0)) / n,   b2 = (conj(a1 c0) - a2 conj(a0) b0) / n,
//   c1 = (conj(a2 b0) - a1 conj(a0) c0) / n,    c2 = -(conj(a1 b0) + a2 conj(a0) c0) / n,
// from the two linear conditions that row b (row c) is orthogonal to row a and that
// c = conj(a x b) (b = conj(c x a)).  CUDA's math library supplies the trig, roots and
// reciprocal: sincos / sqrt in FP64; in FP32 (the FP32 and FP16 links) the fast
// __sincosf (absolute error below 2^-21 on [-pi, pi], the range of the stored phases)
// and __fdividef, whose errors stay within a few FP32 roundings of the link entries.
// wd_set_gauge rejects gauge fields with n below 1e-6 on some link.
__device__ __forceinline__ void sincos_lib(double t, double *s, double *c) { sincos(t, s, c); }
__device__ __forceinline__ void sincos_lib(float t, float *s, float *c) { __sincosf(t, s, c); }
__device__ __forceinline__ double sqrt_lib(double x) { return sqrt(x); }
__device__ __forceinline__ float sqrt_lib(float x) { return sqrtf(x); }
__device__ __forceinline__ double recip_lib(double x) { return 1.0 / x; }
__device__ __forceinline__ float recip_lib(float x) { return __fdividef(1.0f, x); }

template <class R> __device__ __forceinline__ void rebuild_recon8(C<R> (&u)[9], R th0, R th6) {
    const C<R> a1 = u[1], a2 = u[2], b0 = u[3];
    const R n = a1.re * a1.re + a1.im * a1.im + a2.re * a2.re + a2.im * a2.im;
    const R m = n - (b0.re * b0.re + b0.im * b0.im);
    const R ra = sqrt_lib(R(1) - n > R(0) ? R(1) - n : R(0));
    const R rc = sqrt_lib(m > R(0) ? m : R(0));
    R sa, ca, sc, cc;
    sincos_lib(th0, &sa, &ca);
    sincos_lib(th6, &sc, &cc);
    const C<R> a0{ra * ca, ra * sa}, c0{rc * cc, rc * sc};
    const R inv = recip_lib(n);
    const C<R> p = cmulc(a0, b0), q = cmulc(a0, c0);  // conj(a0) b0, conj(a0) c0
    u[0] = a0;
    u[6] = c0;
    u[4] = cscale(-inv, cadd(cmul(a1, p), cconj(cmul(a2, c0))));
    u[5] = cscale(inv, csub(cconj(cmul(a1, c0)), cmul(a2, p)));
    u[7] = cscale(inv, csub(cconj(cmul(a2, b0)), cmul(a1, q)));
    u[8] = cscale(-inv, cadd(cconj(cmul(a1, b0)), cmul(a2, q)));
}

template <int P, int RECON> struct LinkIO;

template <int RECON> struct LinkIO<F64, RECON> {
    using R = double;
    static __device__ __forceinline__ void load(const void *dir_base, int Vs, int s, C<R> (&u)[9]) {
        const double2 *p = reinterpret_cast<const double2 *>(dir_base) + s;
        if constexpr (RECON == 8) {
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                double2 t = __ldg(p + (size_t)e * Vs);
                u[e + 1] = C<R>{t.x, t.y};
            }
            const double2 th = __ldg(p + (size_t)3 * Vs);
            rebuild_recon8(u, th.x, th.y);
            return;
        }
        constexpr int n = RECON == 12 ? 6 : 9;
#pragma unroll
        for (int e = 0; e < n; ++e) {
            double2 t = __ldg(p + (size_t)e * Vs);
            u[e] = C<R>{t.x, t.y};
        }
        if (RECON == 12) rebuild_row2(u);
    }
};

template <int RECON> struct LinkIO<F32, RECON> {
    using R = float;
    static __device__ __forceinline__ void load(const void *dir_base, int Vs, int s, C<R> (&u)[9]) {
        const float4 *p = reinterpret_cast<const float4 *>(dir_base) + s;
        if constexpr (RECON == 8) {
            const float4 t0 = __ldg(p), t1 = __ldg(p + Vs);
            u[1] = C<R>{t0.x, t0.y};
            u[2] = C<R>{t0.z, t0.w};
            u[3] = C<R>{t1.x, t1.y};
            rebuild_recon8(u, t1.z, t1.w);
            return;
        }
        constexpr int n4 = RECON == 12 ? 3 : 4;
#pragma unroll
        for (int j = 0; j < n4; ++j) {
            float4 t = __ldg(p + (size_t)j * Vs);
            u[2 * j] = C<R>{t.x, t.y};
            u[2 * j + 1] = C<R>{t.z, t.w};
        }
        if (RECON == 12) {
            rebuild_row2(u);
        } else {
            const float2 *q = reinterpret_cast<const float2 *>(reinterpret_cast<const float4 *>(dir_base) + (size_t)4 * Vs) + s;
            float2 t = __ldg(q);
            u[8] = C<R>{t.x, t.y};
        }
    }
};

template <int RECON> struct LinkIO<DF32, RECON> {
    using R = df;
    static __device__ __forceinline__ void load(const void *dir_base, int Vs, int s, C<R> (&u)[9]) {
        const float4 *p = reinterpret_cast<const float4 *>(dir_base) + s;
        if constexpr (RECON == 8) {
            // the trig and roots need FP64 accuracy: rebuild in double, split back
            C<double> w[9];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                float4 t = __ldg(p + (size_t)e * Vs);
                w[e + 1] = C<double>{(double)t.x + (double)t.z, (double)t.y + (double)t.w};
            }
            const float4 th = __ldg(p + (size_t)3 * Vs);
            rebuild_recon8(w, (double)th.x + (double)th.z, (double)th.y + (double)th.w);
#pragma unroll
            for (int e = 0; e < 9; ++e) u[e] = C<R>{df(w[e].re), df(w[e].im)};
            return;
        }
        constexpr int n = RECON == 12 ? 6 : 9;
#pragma unroll
        for (int e = 0; e < n; ++e) {
            float4 t = __ldg(p + (size_t)e * Vs);
            u[e] = C<R>{df(t.x, t.z), df(t.y, t.w)};
        }
        if (RECON == 12) rebuild_row2(u);
    }
};

template <int RECON> struct LinkIO<F16, RECON> {
    using R = float;
    static __device__ __forceinline__ void load(const void *dir_base, int Vs, int s, C<R> (&u)[9]) {
        const uint4 *p = reinterpret_cast<const uint4 *>(dir_base) + s;
        if constexpr (RECON == 8) {
            const uint4 t = __ldg(p);
            const float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), th = h2f(t.w);
            u[1] = C<R>{a.x, a.y};
            u[2] = C<R>{b.x, b.y};
            u[3] = C<R>{c.x, c.y};
            rebuild_recon8(u, th.x * kPiF, th.y * kPiF);
            return;
        }
        if (RECON == 12) {
            uint4 t = __ldg(p);
            float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), d = h2f(t.w);
            u[0] = C<R>{a.x, a.y}; u[1] = C<R>{b.x, b.y}; u[2] = C<R>{c.x, c.y}; u[3] = C<R>{d.x, d.y};
            const uint2 *q = reinterpret_cast<const uint2 *>(reinterpret_cast<const uint4 *>(dir_base) + Vs) + s;
            uint2 w = __ldg(q);
            float2 e = h2f(w.x), f = h2f(w.y);
            u[4] = C<R>{e.x, e.y}; u[5] = C<R>{f.x, f.y};
            rebuild_row2(u);
        } else {
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                uint4 t = __ldg(p + (size_t)j * Vs);
                float2 a = h2f(t.x), b = h2f(t.y), c = h2f(t.z), d = h2f(t.w);
                u[4 * j + 0] = C<R>{a.x, a.y}; u[4 * j + 1] = C<R>{b.x, b.y};
                u[4 * j + 2] = C<R>{c.x, c.y}; u[4 * j + 3] = C<R>{d.x, d.y};
            }
            const uint32_t *q = reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint4 *>(dir_base) + (size_t)2 * Vs) + s;
            float2 t = h2f(__ldg(q));
            u[8] = C<R>{t.x, t.y};
        }
    }
};

// ------------------------------------------------------------------ reductions
// Deterministic block reduction of NV doubles per row of a (SB x RT) block.  SB is a
// power of two (16 .. 256) and SB * RT a multiple of 32, so the shuffle groups of
// min(SB, 32) lanes never straddle two rows.  Result valid in threadIdx.x == 0.
// smem: at least RT * MAXW * NV doubles, MAXW >= ceil(SB / 32).
template <int NV, int MAXW = 8>
__device__ __forceinline__ void block_reduce_rows(double (&v)[NV], double *smem) {
    const int SB = blockDim.x;
    const int width = SB < 32 ? SB : 32;
#pragma unroll
    for (int k = 0; k < NV; ++k)
        for (int o = width >> 1; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (SB + 31) >> 5;
    double *row = smem + (size_t)threadIdx.y * MAXW * NV;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) row[w * NV + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0.0;
            for (int i = 0; i < nw; ++i) s += row[i * NV + k];
            v[k] = s;
        }
    }
}

// Last-block-done grid reduction.  Each block has written its per-row partials to
// partial[(rhs * NV + k) * nblk + blockIdx.x]; the block that finishes last sums
// them in block order (deterministic) and returns true in every thread of that
// block, with the totals in tot[rhs*NV + k] (shared memory, visible after the call).
__device__ __forceinline__ bool last_block(unsigned *counter) {
    __shared__ bool am_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        unsigned t = atomicAdd(counter, 1u);
        am_last = (t == gridDim.x * gridDim.y - 1);
    }
    __syncthreads();
    if (am_last) __threadfence();
    return am_last;
}

template <int NV>
__device__ __forceinline__ void sum_partials(const double *partial, int nblk, int nrows, double *tot) {
    // The block has a whole number of warps.  Many sums (rows x NV at least the
    // warps): one warp per sum, lanes stride over the blocks.  Few sums: every thread
    // strides over the partials of one sum, combined by a shuffle tree and then warp
    // by warp in order.  Either way the order is fixed: the same total on every run.
    __shared__ double wsum[32];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, nthr = blockDim.x * blockDim.y;
    const int lane = tid & 31, warp = tid >> 5, nwarp = nthr >> 5;
    if (nrows * NV >= nwarp) {
        for (int q = warp; q < nrows * NV; q += nwarp) {
            double s = 0.0;
            for (int b = lane; b < nblk; b += 32) s += __ldcg(partial + (size_t)q * nblk + b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (lane == 0) tot[q] = s;
        }
        __syncthreads();
        return;
    }
    for (int q = 0; q < nrows * NV; ++q) {
        double s = 0.0;
        for (int b = tid; b < nblk; b += nthr) s += __ldcg(partial + (size_t)q * nblk + b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) wsum[warp] = s;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < nwarp; ++w) t += wsum[w];
            tot[q] = t;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ solver scalars
// One record per right-hand side, resident in device memory.
struct Scalars {
    double rho;        // |r|^2 of the current residual
    double rho_new;
    double pAp;        // |D p|^2
    double alpha, beta;
    double rhs2;       // |D^dag b|^2
    double tol2;       // tol^2 * |D^dag b|^2
    double rmax2;      // max |r|^2 since the last reliable update
    double delta2;
    double true_n2;    // |D^dag (b - D x)|^2 at the end
    double true_b2;    // |b - D x|^2 at the end
    double b2;         // |b|^2
    int iter, max_iter;
    int active;        // still iterating
    int status;
    int reliable;      // number of reliable updates
    int do_update;     // reliable update requested for this iteration
    int pending;       // batched solver: a deferred reliable update is due (the CG step went on)
    int pending_since; // and the iteration at which it fell due
    double delta2_lo;  // FP16 inner iteration: FP32 correction threshold (0: none)
    double rmax2_lo;   // max |r|^2 since the last correction or reliable update
    int do_correct;    // FP32 correction requested for this iteration
    int corrections;   // FP32 corrections run
};

__device__ __forceinline__ bool row_on(const Scalars *sc, int mask, int r) {
    if (mask == 0 || sc == nullptr) return true;
    return mask == 1 ? sc[r].active != 0 : mask == 3 ? sc[r].do_correct != 0 : sc[r].do_update != 0;
}

// Launch shape of a Dslash: blocks of site_tile x rhs_tile (site, right-hand side) pairs; with
// rhs_per_thread = K > 1 (plain FP32 operator) each thread takes K of the block's right-hand
// sides, so the block has site_tile x rhs_tile / K threads and loads each link once for K.
struct DslashTiles { int site_tile = 128; int rhs_tile = 1; int rhs_per_thread = 1; };

}  // namespace wd
