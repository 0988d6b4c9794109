// Element-wise and layout kernels: pack/unpack, gauge upload, precision
// conversion and the CG vector updates (sm_103a).  One thread per (site,
// right-hand side); rows (right-hand sides) can be masked by the per-RHS solver
// state: mask 0 = every row, 1 = rows still iterating, 2 = rows with a reliable
// update pending.
#pragma once
#include "wd_internal.cuh"

namespace wd {

struct VecArgs {
    int V, Vs, nrhs;
    const void *a; size_t a_stride;
    void *b; size_t b_stride;
    const void *c; size_t c_stride;
    Scalars *sc;
    int mask;
    unsigned long long cond;   // while-loop handle to set (0 = none)
    int *state;                // [0] body iterations, [1] reliable-update bodies run, [2] x0 nonzero
};

template <class T> __device__ __forceinline__ const void *rp(const T *b, size_t st, int r) {
    return reinterpret_cast<const char *>(b) + st * (size_t)r;
}
template <class T> __device__ __forceinline__ void *rp(T *b, size_t st, int r) {
    return reinterpret_cast<char *>(b) + st * (size_t)r;
}

// canonical (nrhs x V x 12 complex128) -> field of precision P
template <int P> __global__ void k_pack(VecArgs v) {
    using R = typename Real<P>::T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (s >= v.V) return;
    const double2 *src = reinterpret_cast<const double2 *>(v.a) + ((size_t)r * v.V + s) * 12;
    C<R> x[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) { double2 t = src[c]; x[c] = C<R>{R(t.x), R(t.y)}; }
    SpinorIO<P>::store(rp(v.b, v.b_stride, r), v.Vs, s, x);
}

// field of precision P -> canonical
template <int P> __global__ void k_unpack(VecArgs v) {
    using R = typename Real<P>::T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (s >= v.V) return;
    C<R> x[12];
    SpinorIO<P>::load(rp(v.a, v.a_stride, r), v.Vs, s, x);
    double2 *dst = reinterpret_cast<double2 *>(v.b) + ((size_t)r * v.V + s) * 12;
#pragma unroll
    for (int c = 0; c < 12; ++c) dst[c] = make_double2((double)x[c].re, (double)x[c].im);
}

// b (precision PB) = a (precision PA), masked rows
template <int PA, int PB> __global__ void k_convert(VecArgs v) {
    using RA = typename Real<PA>::T;
    using RB = typename Real<PB>::T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (s >= v.V || !row_on(v.sc, v.mask, r)) return;
    C<RA> x[12];
    C<RB> y[12];
    SpinorIO<PA>::load(rp(v.a, v.a_stride, r), v.Vs, s, x);
#pragma unroll
    for (int c = 0; c < 12; ++c) y[c] = C<RB>{RB(x[c].re), RB(x[c].im)};
    SpinorIO<PB>::store(rp(v.b, v.b_stride, r), v.Vs, s, y);
}

// p = r + beta p   (p, r in precision P), rows still iterating.  Block (0, 0)
// thread 0 counts the iteration and sets the while-loop condition (any row active);
// thread 0 of every x-block-0 clears the row's pending reliable-update flag.
template <int P> __global__ void k_xpby(VecArgs v) {
    using R = typename Real<P>::T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (v.cond && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        int any = 0, cap = 0;
        for (int k = 0; k < v.nrhs; ++k) {
            any |= v.sc[k].active;
            cap = cap > v.sc[k].max_iter ? cap : v.sc[k].max_iter;
        }
        int body = 1;
        if (v.state) body = (v.state[0] += 1);
        if (body > cap + 2) any = 0;  // hard stop: the loop never outlives max_iter
        cudaGraphSetConditional((cudaGraphConditionalHandle)v.cond, any ? 1u : 0u);
    }
    if (v.sc && blockIdx.x == 0 && threadIdx.x == 0 && r < v.nrhs) v.sc[r].do_update = v.sc[r].do_correct = 0;
    if (s >= v.V || !row_on(v.sc, v.mask, r)) return;
    const R beta = R(v.sc[r].beta);
    C<R> x[12], y[12];
    SpinorIO<P>::load(rp(v.a, v.a_stride, r), v.Vs, s, x);  // r
    void *pb = rp(v.b, v.b_stride, r);
    SpinorIO<P>::load(pb, v.Vs, s, y);                       // p
#pragma unroll
    for (int c = 0; c < 12; ++c) y[c] = C<R>{x[c].re + beta * y[c].re, x[c].im + beta * y[c].im};
    SpinorIO<P>::store(pb, v.Vs, s, y);
}

// state[2] = 1 if the FP64 field a (the start vector x0) has a nonzero (or NaN)
// component at some site of some row; state[2] is cleared before the solve.
template <int DUMMY = 0> __global__ void k_any_nonzero(VecArgs v) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (s >= v.V) return;
    const double2 *p = reinterpret_cast<const double2 *>(rp(v.a, v.a_stride, r)) + s;
    bool nz = false;
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        const double2 t = p[(size_t)c * v.Vs];
        nz |= !(t.x == 0.0) || !(t.y == 0.0);
    }
    if (nz) v.state[2] = 1;
}

// x (F64) += xs (F32); xs = 0, rows with a pending reliable update.  Block (0, 0)
// thread 0 counts the reliable-update bodies run.
template <int DUMMY = 0> __global__ void k_reliable_x(VecArgs v) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (v.state && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        int any = 0;
        for (int k = 0; k < v.nrhs; ++k) any |= v.sc[k].do_update | v.sc[k].do_correct;
        if (any) v.state[1] += 1;  // runs of the update branch (a reliable update or a correction)
    }
    if (s >= v.V || !row_on(v.sc, v.mask, r)) return;
    C<double> x[12];
    C<float> xs[12];
    void *xb = rp(v.b, v.b_stride, r);
    void *sb = const_cast<void *>(rp(v.a, v.a_stride, r));
    SpinorIO<F64>::load(xb, v.Vs, s, x);
    SpinorIO<F32>::load(sb, v.Vs, s, xs);
#pragma unroll
    for (int c = 0; c < 12; ++c) {
        x[c] = C<double>{x[c].re + (double)xs[c].re, x[c].im + (double)xs[c].im};
        xs[c] = C<float>{0.f, 0.f};
    }
    SpinorIO<F64>::store(xb, v.Vs, s, x);
    SpinorIO<F32>::store(sb, v.Vs, s, xs);
}

// field = 0 (precision P), every row
template <int P> __global__ void k_zero(VecArgs v) {
    using R = typename Real<P>::T;
    const int s = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (s >= v.V) return;
    C<R> z[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) z[c] = C<R>{R(0), R(0)};
    SpinorIO<P>::store(rp(v.b, v.b_stride, r), v.Vs, s, z);
}

// One link, canonical complex128 u[9] -> the layout of precision P and recon R,
// at index idx of arrays with stride Vs starting at `base` (one direction).
template <int P, int RECON>
__device__ __forceinline__ void pack_link(const double2 *u, char *base, int Vs, int idx) {
    if constexpr (RECON == 8) {
        // entries 1, 2, 3 and the phases of entries 0 and 6
        const double th0 = atan2(u[0].y, u[0].x), th6 = atan2(u[6].y, u[6].x);
        if (P == F64) {
            double2 *d = reinterpret_cast<double2 *>(base) + idx;
            for (int e = 0; e < 3; ++e) d[(size_t)e * Vs] = u[e + 1];
            d[(size_t)3 * Vs] = make_double2(th0, th6);
        } else if (P == DF32) {
            float4 *d = reinterpret_cast<float4 *>(base) + idx;
            for (int e = 0; e < 3; ++e) {
                const df re(u[e + 1].x), im(u[e + 1].y);
                d[(size_t)e * Vs] = make_float4(re.hi, im.hi, re.lo, im.lo);
            }
            const df t0(th0), t6(th6);
            d[(size_t)3 * Vs] = make_float4(t0.hi, t6.hi, t0.lo, t6.lo);
        } else if (P == F32) {
            float4 *d = reinterpret_cast<float4 *>(base) + idx;
            d[0] = make_float4((float)u[1].x, (float)u[1].y, (float)u[2].x, (float)u[2].y);
            d[Vs] = make_float4((float)u[3].x, (float)u[3].y, (float)th0, (float)th6);
        } else {
            const double ipi = 0.31830988618379067;  // 1 / pi
            uint4 *d = reinterpret_cast<uint4 *>(base) + idx;
            *d = make_uint4(f2h((float)u[1].x, (float)u[1].y), f2h((float)u[2].x, (float)u[2].y),
                            f2h((float)u[3].x, (float)u[3].y), f2h((float)(th0 * ipi), (float)(th6 * ipi)));
        }
        return;
    }
    constexpr int n = RECON == 12 ? 6 : 9;
    if (P == F64) {
        double2 *d = reinterpret_cast<double2 *>(base) + idx;
        for (int e = 0; e < n; ++e) d[(size_t)e * Vs] = u[e];
    } else if (P == DF32) {
        float4 *d = reinterpret_cast<float4 *>(base) + idx;
        for (int e = 0; e < n; ++e) {
            const df re(u[e].x), im(u[e].y);
            d[(size_t)e * Vs] = make_float4(re.hi, im.hi, re.lo, im.lo);
        }
    } else if (P == F32) {
        float4 *d = reinterpret_cast<float4 *>(base) + idx;
        const int n4 = n / 2;
        for (int j = 0; j < n4; ++j)
            d[(size_t)j * Vs] = make_float4((float)u[2 * j].x, (float)u[2 * j].y, (float)u[2 * j + 1].x, (float)u[2 * j + 1].y);
        if (RECON == 18) {
            float2 *e = reinterpret_cast<float2 *>(reinterpret_cast<float4 *>(base) + (size_t)4 * Vs) + idx;
            *e = make_float2((float)u[8].x, (float)u[8].y);
        }
    } else {
        uint4 *d = reinterpret_cast<uint4 *>(base) + idx;
        auto h = [&](int e) { return f2h((float)u[e].x, (float)u[e].y); };
        if (RECON == 12) {
            *d = make_uint4(h(0), h(1), h(2), h(3));
            uint2 *e = reinterpret_cast<uint2 *>(reinterpret_cast<uint4 *>(base) + Vs) + idx;
            *e = make_uint2(h(4), h(5));
        } else {
            d[0] = make_uint4(h(0), h(1), h(2), h(3));
            d[Vs] = make_uint4(h(4), h(5), h(6), h(7));
            uint32_t *e = reinterpret_cast<uint32_t *>(reinterpret_cast<uint4 *>(base) + (size_t)2 * Vs) + idx;
            *e = h(8);
        }
    }
}

// gauge: canonical (4 x V x 9 complex128, device) -> field of precision P, recon R
template <int P, int RECON> __global__ void k_gauge_pack(const double2 *canon, void *dst, int V, int Vs,
                                                         size_t dir_bytes) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x, mu = blockIdx.y;
    if (s >= V) return;
    pack_link<P, RECON>(canon + ((size_t)mu * V + s) * 9, reinterpret_cast<char *>(dst) + (size_t)mu * dir_bytes, Vs, s);
}

// smallest n = |u01|^2 + |u02|^2 over all links (the recon-8 denominator), as the
// bits of a non-negative float (ordered like the floats); *out starts above any n
template <int DUMMY = 0> __global__ void k_gauge_min_offdiag(const double2 *canon, size_t nlinks, unsigned *out) {
    float m = 3.0e38f;
    for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < nlinks; l += (size_t)gridDim.x * blockDim.x) {
        const double2 a1 = canon[l * 9 + 1], a2 = canon[l * 9 + 2];
        m = fminf(m, (float)(a1.x * a1.x + a1.y * a1.y + a2.x * a2.x + a2.y * a2.y));
    }
    for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMin(out, __float_as_uint(m));
}

// gauge in checkerboard order: U_mu(n) -> parity of n, index n / 2 (arrays of stride Vhs)
template <int P, int RECON> __global__ void k_gauge_pack_eo(const double2 *canon, void *dst, Geom g, int Vhs,
                                                            size_t dir_bytes) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x, mu = blockIdx.y;
    if (n >= g.V) return;
    int rem = n;
    const int x = rem % g.L[0]; rem /= g.L[0];
    const int y = rem % g.L[1]; rem /= g.L[1];
    const int z = rem % g.L[2];
    const int t = rem / g.L[2];
    const int par = (x + y + z + t) & 1;
    char *base = reinterpret_cast<char *>(dst) + (size_t)(4 * par + mu) * dir_bytes;
    pack_link<P, RECON>(canon + ((size_t)mu * g.V + n) * 9, base, Vhs, n >> 1);
}

__device__ __forceinline__ int site_parity(const Geom &g, int n) {
    int rem = n;
    const int x = rem % g.L[0]; rem /= g.L[0];
    const int y = rem % g.L[1]; rem /= g.L[1];
    const int z = rem % g.L[2];
    const int t = rem / g.L[2];
    return (x + y + z + t) & 1;
}

struct EoVecArgs {
    VecArgs v;
    int Vhs;  // site stride of the half fields
    Geom g;   // full-lattice geometry
};

// FP64 full-lattice field (v.a, site stride v.Vs, RHS stride v.a_stride) -> even half
// (v.b) and odd half (v.c) in checkerboard order (site stride Vhs, RHS stride v.b_stride)
template <int DUMMY = 0> __global__ void k_split_eo(EoVecArgs e) {
    const VecArgs &v = e.v;
    const int n = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (n >= v.V) return;
    C<double> x[12];
    SpinorIO<F64>::load(rp(v.a, v.a_stride, r), v.Vs, n, x);
    void *dst = site_parity(e.g, n) ? const_cast<void *>(v.c) : v.b;
    SpinorIO<F64>::store(rp(dst, v.b_stride, r), e.Vhs, n >> 1, x);
}

// the inverse: even (v.a) and odd (v.c) halves (RHS stride v.a_stride) -> full field (v.b)
template <int DUMMY = 0> __global__ void k_join_eo(EoVecArgs e) {
    const VecArgs &v = e.v;
    const int n = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (n >= v.V) return;
    C<double> x[12];
    const void *src = site_parity(e.g, n) ? v.c : v.a;
    SpinorIO<F64>::load(rp(src, v.a_stride, r), e.Vhs, n >> 1, x);
    SpinorIO<F64>::store(rp(v.b, v.b_stride, r), v.Vs, n, x);
}

// A deterministic non-zero buffer (values in [-1, 1) from a hash of the index): the input of
// the autotuners, so that no candidate is timed on zeros.  For FP16 fields of reals it
// fills every 32-bit word with a float in [-1, 1), scales included.
template <class T> __global__ void k_fill_hash(T *p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        unsigned long long z = (i + 1) * 0x9E3779B97F4A7C15ull;
        z = (z ^ (z >> 31)) * 0xD6E8FEB86659FD93ull;
        z ^= z >> 32;
        p[i] = (T)((double)(z >> 11) * 0x1.0p-52 - 1.0);
    }
}

}  // namespace wd
