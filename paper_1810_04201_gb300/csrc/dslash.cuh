// Wilson-Dirac hopping term and the Dslash kernel template (sm_103a).
//
// One thread computes one output site of one right-hand side (FP32, FP16), or two
// lanes of a warp share it (FP64, DF32; see "two lanes per site" below).  A thread
// block is (site_tile x rhs_tile) threads: the rhs_tile right-hand sides of a block
// read the same links, which the L1 cache then serves once per block.
//
// Per hop (section 2.1, Eq. (1) and Eq. (3); section 2.1, half-spinor remark):
//   gamma_mu = [[0, A_mu], [A_mu^dag, 0]] in 2x2 spin blocks (Appendix A), with
//   A_0 = [[0, i], [i, 0]], A_1 = [[0, -1], [1, 0]], A_2 = [[i, 0], [0, -i]], A_3 = 1.
//   (1 + s gamma_mu) psi has upper half h = psi_up + s A_mu psi_dn and lower half
//   s A_mu^dag h, so only the two upper colour vectors are multiplied by the link:
//   spin projection -> SU(3) x 2 colour vectors -> reconstruction -> accumulation.
//   D: forward hop s = -1 with U_mu(n), backward hop s = +1 with U_mu(n-mu)^dag.
//   D^dag: the signs swap (gamma5 D gamma5 = D^dag, section 2.2).
//   Antiperiodic time boundary: the hop across t = T-1 <-> 0 is multiplied by -1.
#pragma once
#include "wd_internal.cuh"

namespace wd {

struct DslashArgs {
    Geom g;
    const void *in;
    size_t in_stride;   // bytes between right-hand sides
    void *out;
    size_t out_stride;
    const void *gauge;
    size_t gauge_dir;   // bytes between directions
    double kappa;
    int nrhs;
    // epilogue operands (meaning depends on the epilogue)
    const void *a0; size_t a0_stride;
    void *a1; size_t a1_stride;
    void *a2; size_t a2_stride;
    const void *a3; size_t a3_stride;
    Scalars *sc;               // per right-hand-side solver state (nullptr: plain operator)
    int mask;                  // rows to process: 0 all, 1 active, 2 reliable update, 3 FP32 correction
    double *partial;           // per-block partial sums
    unsigned *counter;         // last-block ticket
    unsigned long long cond;   // cudaGraphConditionalHandle to set (0 = none)
    int *state;                // solver-wide counters
    const int *run_flag;       // when set and zero, the whole launch returns at once
    const void *xsrc;          // field added by the xpay epilogues (nullptr: the hopping input)
    size_t xsrc_stride;
    const int *in_nonzero;     // when set and zero, the input fields are zero: not read, hopping sum 0
};

template <class R> __device__ __forceinline__ const void *rhs_ptr(const void *b, size_t stride, int r) {
    return reinterpret_cast<const char *>(b) + stride * (size_t)r;
}
template <class R> __device__ __forceinline__ void *rhs_ptr(void *b, size_t stride, int r) {
    return reinterpret_cast<char *>(b) + stride * (size_t)r;
}

// h = psi_up + s A_mu psi_dn, h[sp*3 + colour], sp = 0, 1
template <int MU, int S, class R>
__device__ __forceinline__ void project(const C<R> (&p)[12], C<R> (&h)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C<R> d2 = p[6 + c], d3 = p[9 + c];
        C<R> a0, a1;
        if (MU == 0) { a0 = cmuli(d3); a1 = cmuli(d2); }
        else if (MU == 1) { a0 = cneg(d3); a1 = d2; }
        else if (MU == 2) { a0 = cmuli(d2); a1 = cneg(cmuli(d3)); }
        else { a0 = d2; a1 = d3; }
        if (S > 0) { h[c] = cadd(p[c], a0); h[3 + c] = cadd(p[3 + c], a1); }
        else { h[c] = csub(p[c], a0); h[3 + c] = csub(p[3 + c], a1); }
    }
}

// acc_up += w, acc_dn += s A_mu^dag w
template <int MU, int S, class R>
__device__ __forceinline__ void accumulate(C<R> (&acc)[12], const C<R> (&w)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C<R> w0 = w[c], w1 = w[3 + c];
        acc[c] = cadd(acc[c], w0);
        acc[3 + c] = cadd(acc[3 + c], w1);
        C<R> b0, b1;  // A^dag (w0, w1)
        if (MU == 0) { b0 = cneg(cmuli(w1)); b1 = cneg(cmuli(w0)); }
        else if (MU == 1) { b0 = w1; b1 = cneg(w0); }
        else if (MU == 2) { b0 = cneg(cmuli(w0)); b1 = cmuli(w1); }
        else { b0 = w0; b1 = w1; }
        if (S > 0) { acc[6 + c] = cadd(acc[6 + c], b0); acc[9 + c] = cadd(acc[9 + c], b1); }
        else { acc[6 + c] = csub(acc[6 + c], b0); acc[9 + c] = csub(acc[9 + c], b1); }
    }
}

template <int P> struct HasScale { static constexpr bool value = false; };
template <> struct HasScale<F16> { static constexpr bool value = true; };

// w = U h (forward) or U^dag h (backward), two colour vectors; optional sign flip
template <class R> __device__ __forceinline__ void zero6(C<R> (&w)[6]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) w[k] = C<R>{R(0), R(0)};
}

template <bool ADJ, class R>
__device__ __forceinline__ void su3_mult(const C<R> (&u)[9], const C<R> (&h)[6], C<R> (&w)[6], bool flip) {
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C<R> s;
            if (!ADJ) {
                s = cmul(u[3 * a + 0], h[3 * sp + 0]);
                s = cmac(s, u[3 * a + 1], h[3 * sp + 1]);
                s = cmac(s, u[3 * a + 2], h[3 * sp + 2]);
            } else {
                s = cmulc(u[0 + a], h[3 * sp + 0]);
                s = cmacc(s, u[3 + a], h[3 * sp + 1]);
                s = cmacc(s, u[6 + a], h[3 * sp + 2]);
            }
            w[3 * sp + a] = flip ? cneg(s) : s;
        }
}

template <int P, int RECON, bool DAG, int MU, bool NC = true>
__device__ __forceinline__ void hop_dir(const Geom &g, const void *in, const char *gdir, int s, int c,
                                        C<typename Real<P>::T> (&acc)[12]) {
    using R = typename Real<P>::T;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma
    const int L = g.L[MU], st = g.stride[MU];
    {
        const int sf = WD_IDX(g, (c == L - 1) ? s - (L - 1) * st : s + st, g.V, 1);
        C<R> p[12], h[6], w[6], u[9];
        SpinorIO<P>::template load<NC>(in, g.Vs, sf, p);
        project<MU, SF>(p, h);
        LinkIO<P, RECON>::load(gdir, g.Vs, s, u);
        su3_mult<false>(u, h, w, MU == 3 && g.antiperiodic && c == L - 1);
        if (MU == 3 && g.split_t && c == L - 1) zero6(w);  // the neighbour lives on the next sub-lattice
        accumulate<MU, SF>(acc, w);
    }
    {
        const int sb = WD_IDX(g, (c == 0) ? s + (L - 1) * st : s - st, g.V, 2);
        C<R> p[12], h[6], w[6], u[9];
        SpinorIO<P>::template load<NC>(in, g.Vs, sb, p);
        project<MU, -SF>(p, h);
        LinkIO<P, RECON>::load(gdir, g.Vs, sb, u);
        su3_mult<true>(u, h, w, MU == 3 && g.antiperiodic && c == 0);
        if (MU == 3 && g.split_t && c == 0) zero6(w);  // the neighbour lives on the previous sub-lattice
        accumulate<MU, -SF>(acc, w);
    }
}

// ---------------------------------------------------------------- FP16 on half operands
// FP16 spinors (scaled to the site maximum) and links stay in half precision up to
// the SU(3) product: the projection adds the two half values of each pair (HADD2,
// one rounding to half, the size of the storage rounding), and U h is formed by FMAs
// with half multiplicands and FP32 accumulators (fma.rn.f32.f16 of sm_100+: a product
// of two halves is exact in FP32).  No half value is converted on the way.  The site
// scale and the boundary sign enter once, in the FP32 multiply-adds that accumulate
// U h.  (GB300 probe: 33 T such FMAs/s against 20 T/s for two conversions and an FFMA.)
typedef uint32_t h2;  // a half2, real part in the low half, as its bits

__device__ __forceinline__ h2 h2_add(h2 a, h2 b) {
    const __half2 r = __hadd2(*reinterpret_cast<const __half2 *>(&a), *reinterpret_cast<const __half2 *>(&b));
    return *reinterpret_cast<const h2 *>(&r);
}
__device__ __forceinline__ h2 h2_sub(h2 a, h2 b) {
    const __half2 r = __hsub2(*reinterpret_cast<const __half2 *>(&a), *reinterpret_cast<const __half2 *>(&b));
    return *reinterpret_cast<const h2 *>(&r);
}
__device__ __forceinline__ h2 h2_neg(h2 a) { return a ^ 0x80008000u; }
__device__ __forceinline__ h2 h2_muli(h2 a) { return ((a >> 16) | (a << 16)) ^ 0x00008000u; }  // i (x + iy) = -y + ix

// s + u h: re += ur hr - ui hi, im += ur hi + ui hr (hn: h with its imaginary half negated)
__device__ __forceinline__ void cmac_h(C<float> &s, h2 u, h2 h, h2 hn) {
    asm("{\n\t.reg .f16 ur, ui, hr, hi, nr, ni;\n\t"
        "mov.b32 {ur, ui}, %2;\n\tmov.b32 {hr, hi}, %3;\n\tmov.b32 {nr, ni}, %4;\n\t"
        "fma.rn.f32.f16 %0, ur, hr, %0;\n\tfma.rn.f32.f16 %0, ui, ni, %0;\n\t"
        "fma.rn.f32.f16 %1, ur, hi, %1;\n\tfma.rn.f32.f16 %1, ui, hr, %1;\n\t}"
        : "+f"(s.re), "+f"(s.im) : "r"(u), "r"(h), "r"(hn));
}
// s + conj(u) h: re += ur hr + ui hi, im += ur hi - ui hr (hn: h with its real half negated)
__device__ __forceinline__ void cmacc_h(C<float> &s, h2 u, h2 h, h2 hn) {
    asm("{\n\t.reg .f16 ur, ui, hr, hi, nr, ni;\n\t"
        "mov.b32 {ur, ui}, %2;\n\tmov.b32 {hr, hi}, %3;\n\tmov.b32 {nr, ni}, %4;\n\t"
        "fma.rn.f32.f16 %0, ur, hr, %0;\n\tfma.rn.f32.f16 %0, ui, hi, %0;\n\t"
        "fma.rn.f32.f16 %1, ur, hi, %1;\n\tfma.rn.f32.f16 %1, ui, nr, %1;\n\t}"
        : "+f"(s.re), "+f"(s.im) : "r"(u), "r"(h), "r"(hn));
}

// the 12 raw half2 components of site s and its scale
template <bool NC>
__device__ __forceinline__ float load_raw_h2(const void *base, int Vs, int s, h2 (&v)[12]) {
    const uint4 *p = reinterpret_cast<const uint4 *>(base) + s;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const uint4 t = ldx<NC>(p + (size_t)j * Vs);
        v[4 * j + 0] = t.x; v[4 * j + 1] = t.y; v[4 * j + 2] = t.z; v[4 * j + 3] = t.w;
    }
    return ldx<NC>(SpinorIO<F16>::norms(base, Vs) + s);
}

// the 9 link entries as half2 (recon-12/8 rows are rebuilt in FP32 and rounded to half)
template <int RECON>
__device__ __forceinline__ void load_link_h2(const char *gdir, int Vs, int s, h2 (&u)[9]) {
    if constexpr (RECON == 18) {
        const uint4 *p = reinterpret_cast<const uint4 *>(gdir) + s;
        const uint4 a = __ldg(p), b = __ldg(p + Vs);
        u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
        u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
        u[8] = __ldg(reinterpret_cast<const uint32_t *>(reinterpret_cast<const uint4 *>(gdir) + (size_t)2 * Vs) + s);
    } else {
        C<float> w[9];
        LinkIO<F16, RECON>::load(gdir, Vs, s, w);
#pragma unroll
        for (int e = 0; e < 9; ++e) u[e] = f2h(w[e].re, w[e].im);
    }
}

// h = psi_up + S A_mu psi_dn on half2 values (the half-precision projection)
template <int MU, int S>
__device__ __forceinline__ void project_h2(const h2 (&p)[12], h2 (&h)[6]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const h2 d2 = p[6 + c], d3 = p[9 + c];
        h2 a0, a1;
        if (MU == 0) { a0 = h2_muli(d3); a1 = h2_muli(d2); }
        else if (MU == 1) { a0 = h2_neg(d3); a1 = d2; }
        else if (MU == 2) { a0 = h2_muli(d2); a1 = h2_neg(h2_muli(d3)); }
        else { a0 = d2; a1 = d3; }
        h[c] = S > 0 ? h2_add(p[c], a0) : h2_sub(p[c], a0);
        h[3 + c] = S > 0 ? h2_add(p[3 + c], a1) : h2_sub(p[3 + c], a1);
    }
}

// acc_up += sc w, acc_dn += S sc A_mu^dag w (FP32 multiply-adds; sc: scale and sign)
template <int MU, int S>
__device__ __forceinline__ void accumulate_scaled(C<float> (&acc)[12], const C<float> (&w)[6], float sc) {
    const float ss = S > 0 ? sc : -sc;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C<float> w0 = w[c], w1 = w[3 + c];
        acc[c] = C<float>{fmaf(sc, w0.re, acc[c].re), fmaf(sc, w0.im, acc[c].im)};
        acc[3 + c] = C<float>{fmaf(sc, w1.re, acc[3 + c].re), fmaf(sc, w1.im, acc[3 + c].im)};
        C<float> b0, b1;  // A^dag (w0, w1)
        if (MU == 0) { b0 = cneg(cmuli(w1)); b1 = cneg(cmuli(w0)); }
        else if (MU == 1) { b0 = w1; b1 = cneg(w0); }
        else if (MU == 2) { b0 = cneg(cmuli(w0)); b1 = cmuli(w1); }
        else { b0 = w0; b1 = w1; }
        acc[6 + c] = C<float>{fmaf(ss, b0.re, acc[6 + c].re), fmaf(ss, b0.im, acc[6 + c].im)};
        acc[9 + c] = C<float>{fmaf(ss, b1.re, acc[9 + c].re), fmaf(ss, b1.im, acc[9 + c].im)};
    }
}

// one FP16 hop: neighbour spinor at index sn, link at index sl of gdir (its adjoint for
// ADJ), projector sign S, boundary sign flip; the links' site stride is Vl (0: Vs, the
// spinor's, except for spinors staged in shared memory)
template <int RECON, bool ADJ, int MU, int S, bool NC>
__device__ __forceinline__ void hop_f16(const void *in, int Vs, int sn, const char *gdir, int sl, bool flip,
                                        C<float> (&acc)[12], int Vl = 0) {
    h2 p[12], h[6], hn[6], u[9];
    const float scale = load_raw_h2<NC>(in, Vs, sn, p);
    project_h2<MU, S>(p, h);
#pragma unroll
    for (int k = 0; k < 6; ++k) hn[k] = h[k] ^ (ADJ ? 0x00008000u : 0x80000000u);
    load_link_h2<RECON>(gdir, Vl ? Vl : Vs, sl, u);
    C<float> w[6];
#pragma unroll
    for (int sp = 0; sp < 2; ++sp)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C<float> t{0.f, 0.f};
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (!ADJ) cmac_h(t, u[3 * a + b], h[3 * sp + b], hn[3 * sp + b]);
                else cmacc_h(t, u[3 * b + a], h[3 * sp + b], hn[3 * sp + b]);
            }
            w[3 * sp + a] = t;
        }
    accumulate_scaled<MU, S>(acc, w, flip ? -scale : scale);
}

template <int P, int RECON, bool DAG, int MU, bool NC = true>
__device__ __forceinline__ void hop_dir_scaled(const Geom &g, const void *in, const char *gdir, int s, int c,
                                               C<typename Real<P>::T> (&acc)[12]) {
    static_assert(P == F16, "FP16 hop");
    constexpr int SF = DAG ? +1 : -1;
    const int L = g.L[MU], st = g.stride[MU];
    const int sf = WD_IDX(g, (c == L - 1) ? s - (L - 1) * st : s + st, g.V, 1);
    hop_f16<RECON, false, MU, SF, NC>(in, g.Vs, sf, gdir, s, MU == 3 && g.antiperiodic && c == L - 1, acc);
    const int sb = WD_IDX(g, (c == 0) ? s + (L - 1) * st : s - st, g.V, 2);
    hop_f16<RECON, true, MU, -SF, NC>(in, g.Vs, sb, gdir, sb, MU == 3 && g.antiperiodic && c == 0, acc);
}

// acc = sum over the 8 hops (the bracket of Eq. (1)) at site s of field `in`.
template <int P, int RECON, bool DAG, bool NC = true>
__device__ __forceinline__ void hopping(const Geom &g, const void *in, const void *gauge, size_t gdir_bytes, int s,
                                        C<typename Real<P>::T> (&acc)[12]) {
    using R = typename Real<P>::T;
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = C<R>{R(0), R(0)};
    int rem = s;
    const int x = rem % g.L[0]; rem /= g.L[0];
    const int y = rem % g.L[1]; rem /= g.L[1];
    const int z = rem % g.L[2];
    const int t = rem / g.L[2];
    const char *gb = reinterpret_cast<const char *>(gauge);
    if constexpr (HasScale<P>::value) {
        hop_dir_scaled<P, RECON, DAG, 0, NC>(g, in, gb, s, x, acc);
        hop_dir_scaled<P, RECON, DAG, 1, NC>(g, in, gb + gdir_bytes, s, y, acc);
        hop_dir_scaled<P, RECON, DAG, 2, NC>(g, in, gb + 2 * gdir_bytes, s, z, acc);
        hop_dir_scaled<P, RECON, DAG, 3, NC>(g, in, gb + 3 * gdir_bytes, s, t, acc);
    } else {
        hop_dir<P, RECON, DAG, 0, NC>(g, in, gb, s, x, acc);
        hop_dir<P, RECON, DAG, 1, NC>(g, in, gb + gdir_bytes, s, y, acc);
        hop_dir<P, RECON, DAG, 2, NC>(g, in, gb + 2 * gdir_bytes, s, z, acc);
        hop_dir<P, RECON, DAG, 3, NC>(g, in, gb + 3 * gdir_bytes, s, t, acc);
    }
}

// ---------------------------------------------------------------- checkerboard
// Even-odd fields hold one parity of the lattice: the site with full index n
// (parity (x+y+z+t) mod 2) sits at n / 2 of its parity's arrays (all extents
// even).  Links are stored the same way, per parity: U_mu(n) at n / 2 of the
// parity of n, so the forward hop reads the output site's own parity and the
// backward hop reads U_mu(n - mu) at the neighbour's index.  gauge points to
// parity 0; parity 1 follows 4 * gdir_bytes later.
__device__ __forceinline__ int eo_full_index(const Geom &g, int k, int &x, int &y, int &z, int &t) {
    const int lxh = g.L[0] >> 1;
    int r = k / lxh;
    const int xh = k - r * lxh;
    y = r % g.L[1];
    r /= g.L[1];
    z = r % g.L[2];
    t = r / g.L[2];
    x = 2 * xh + ((g.eo_parity + y + z + t) & 1);
    return WD_IDX(g, x + g.stride[1] * y + g.stride[2] * z + g.stride[3] * t, 2 * g.V, 5);
}

template <int P, int RECON, bool DAG, int MU, bool NC = true>
__device__ __forceinline__ void hop_dir_eo(const Geom &g, const void *in, const char *gp, const char *gq, int k, int n,
                                           int c, C<typename Real<P>::T> (&acc)[12]) {
    using R = typename Real<P>::T;
    constexpr int SF = DAG ? +1 : -1;
    const int L = g.L[MU], st = g.stride[MU];
    if constexpr (P == F16) {
        const int nf = WD_IDX(g, (c == L - 1) ? n - (L - 1) * st : n + st, 2 * g.V, 3);
        hop_f16<RECON, false, MU, SF, NC>(in, g.Vs, nf >> 1, gp, k, MU == 3 && g.antiperiodic && c == L - 1, acc);
        const int nb = WD_IDX(g, (c == 0) ? n + (L - 1) * st : n - st, 2 * g.V, 4);
        hop_f16<RECON, true, MU, -SF, NC>(in, g.Vs, nb >> 1, gq, nb >> 1, MU == 3 && g.antiperiodic && c == 0, acc);
    } else {
        {
            const int nf = WD_IDX(g, (c == L - 1) ? n - (L - 1) * st : n + st, 2 * g.V, 3);
            C<R> p[12], h[6], w[6], u[9];
            SpinorIO<P>::template load<NC>(in, g.Vs, nf >> 1, p);
            project<MU, SF>(p, h);
            LinkIO<P, RECON>::load(gp, g.Vs, k, u);
            su3_mult<false>(u, h, w, MU == 3 && g.antiperiodic && c == L - 1);
            accumulate<MU, SF>(acc, w);
        }
        {
            const int nb = WD_IDX(g, (c == 0) ? n + (L - 1) * st : n - st, 2 * g.V, 4);
            C<R> p[12], h[6], w[6], u[9];
            SpinorIO<P>::template load<NC>(in, g.Vs, nb >> 1, p);
            project<MU, -SF>(p, h);
            LinkIO<P, RECON>::load(gq, g.Vs, nb >> 1, u);
            su3_mult<true>(u, h, w, MU == 3 && g.antiperiodic && c == 0);
            accumulate<MU, -SF>(acc, w);
        }
    }
}

template <int P, int RECON, bool DAG, bool NC = true>
__device__ __forceinline__ void hopping_eo(const Geom &g, const void *in, const void *gauge, size_t gdir_bytes, int k,
                                           C<typename Real<P>::T> (&acc)[12]) {
    using R = typename Real<P>::T;
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = C<R>{R(0), R(0)};
    int x, y, z, t;
    const int n = eo_full_index(g, k, x, y, z, t);
    const char *gp = reinterpret_cast<const char *>(gauge) + (size_t)(4 * g.eo_parity) * gdir_bytes;
    const char *gq = reinterpret_cast<const char *>(gauge) + (size_t)(4 * (1 - g.eo_parity)) * gdir_bytes;
    hop_dir_eo<P, RECON, DAG, 0, NC>(g, in, gp, gq, k, n, x, acc);
    hop_dir_eo<P, RECON, DAG, 1, NC>(g, in, gp + gdir_bytes, gq + gdir_bytes, k, n, y, acc);
    hop_dir_eo<P, RECON, DAG, 2, NC>(g, in, gp + 2 * gdir_bytes, gq + 2 * gdir_bytes, k, n, z, acc);
    hop_dir_eo<P, RECON, DAG, 3, NC>(g, in, gp + 3 * gdir_bytes, gq + 3 * gdir_bytes, k, n, t, acc);
}

// ---------------------------------------------------------------- two lanes per site
// FP64 is bound by the FP64 units, which belong to the four schedulers of an SM:
// a scheduler without warps leaves its unit idle, as in the partial last wave of a
// launch.  So FP64 sites run on two lanes of a warp, lane l and l ^ 16, and twice
// as many warps share the work.  DF32 (bound by instruction issue) does the same:
// half the work per lane needs 128 instead of 255 registers, so twice the warps
// hide the latencies.  Lane half hh computes spin component hh of every
// projected half spinor.  Row hh of A_mu has one entry f, in column ps - 2, where
// ps = 3 - hh for mu = 0, 1 and ps = 2 + hh for mu = 2, 3, so
//   h_hh = psi_hh + s f psi_ps,   upper spin hh += (U h)_hh,   lower spin ps += s conj(f) (U h)_hh,
// with f = i (mu = 0), -1 / +1 (mu = 1, hh = 0 / 1), i / -i (mu = 2), 1 (mu = 3).
// The two halves do exactly the arithmetic of one site between them.  The lane's
// accumulator holds spin hh [0..2], spin 3 - hh [3..5] (from mu = 0, 1) and spin
// 2 + hh [6..8] (from mu = 2, 3); after the last hop the last block is exchanged
// with the partner lane, and the lane owns spins hh and 3 - hh.
template <int P> constexpr bool split_site() { return P == F64 || P == DF32; }
template <int P> constexpr int threads_per_site() { return split_site<P>() ? 2 : 1; }
inline int threads_per_site(Prec p) {
    return p == F64 ? threads_per_site<F64>() : p == DF32 ? threads_per_site<DF32>()
         : p == F32 ? threads_per_site<F32>() : threads_per_site<F16>();
}
// blocks along the sites for a (site_tile x rhs_tile) block: site_tile / threads_per_site sites each
template <int P> inline int site_blocks(int V, int site_tile) {
    const int spb = site_tile / threads_per_site<P>();
    return (V + spb - 1) / spb;
}

// sign flips as bit operations (no floating-point instruction)
__device__ __forceinline__ double xsign(double x, bool neg) {
    return __longlong_as_double(__double_as_longlong(x) ^ ((unsigned long long)neg << 63));
}
__device__ __forceinline__ float xsign(float x, bool neg) { return __uint_as_float(__float_as_uint(x) ^ ((unsigned)neg << 31)); }
__device__ __forceinline__ df xsign(df x, bool neg) { return df(xsign(x.hi, neg), xsign(x.lo, neg)); }
template <class R> __device__ __forceinline__ C<R> cxsign(C<R> a, bool neg) { return C<R>{xsign(a.re, neg), xsign(a.im, neg)}; }
// f d with f = +-1 (im = false) or +-i (im = true), the sign given by neg
template <class R> __device__ __forceinline__ C<R> times_f(C<R> d, bool im, bool neg) {
    const C<R> t = im ? C<R>{xsign(d.im, true), d.re} : d;
    return cxsign(t, neg);
}

// the 3 colour components of spin sp of site s (FP64 layout: one array per component;
// DF32 has its packed form, load_spin_cd)
template <int P, bool NC, class R>
__device__ __forceinline__ void load_spin(const void *base, int Vs, int s, int sp, C<R> (&v)[3]) {
    static_assert(P == F64, "per-component FP64 spinor arrays");
    const double2 *q = reinterpret_cast<const double2 *>(base) + (size_t)(3 * sp) * Vs + s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 t = ldx<NC>(q + (size_t)c * Vs);
        v[c] = C<R>{t.x, t.y};
    }
}

// w = U h (ADJ = false) or U^dag h (ADJ = true) for one colour vector
template <bool ADJ, class R>
__device__ __forceinline__ void su3_mult1(const C<R> (&u)[9], const C<R> (&h)[3], C<R> (&w)[3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        C<R> s;
        if (!ADJ) {
            s = cmul(u[3 * a + 0], h[0]);
            s = cmac(s, u[3 * a + 1], h[1]);
            s = cmac(s, u[3 * a + 2], h[2]);
        } else {
            s = cmulc(u[0 + a], h[0]);
            s = cmacc(s, u[3 + a], h[1]);
            s = cmacc(s, u[6 + a], h[2]);
        }
        w[a] = s;
    }
}

// Both hops of direction mu for lane half hh.  The forward and backward products
// enter the upper spin as a sum and the lower spin ps as a difference (the two
// projectors differ in the sign of s), so the backward product is accumulated onto
// the forward one (w_f + w_b as one chain of multiply-adds) and the difference
// is formed as 2 w_f - (w_f + w_b): 6 fewer FP64 operations per lane and direction
// than two separate hops.  Neighbours: forward spinor index nf with link gf[kf],
// backward spinor index nb with link gb[kb]; flip_f / flip_b are the boundary signs.
// mu is a run-time value (constant-folded where the caller unrolls the directions);
// LO = 3 for mu = 0, 1 and 6 for mu = 2, 3 selects the accumulator block of spin ps.

template <int P, int RECON, bool DAG, int LO, bool NC, class R>
__device__ __forceinline__ void half_pair(int mu, const void *in, int Vs, int nf, const char *gf, int kf, bool flip_f,
                                          int nb, const char *gb, int kb, bool flip_b, int hh, C<R> (&acc)[9],
                                          bool zero_f = false, bool zero_b = false) {
    constexpr int SF = DAG ? +1 : -1;
    const bool IM = mu == 0 || mu == 2;
    const bool neg = mu == 1 ? hh == 0 : mu == 2 ? hh != 0 : false;
    const int ps = mu < 2 ? 3 - hh : 2 + hh;
    C<R> wf[3], sum[3];
    {
        C<R> ph[3], pd[3], h[3], u[9];
        load_spin<P, NC>(in, Vs, nf, hh, ph);
        load_spin<P, NC>(in, Vs, nf, ps, pd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C<R> fd = times_f(pd[c], IM, neg);
            h[c] = cxsign(SF > 0 ? cadd(ph[c], fd) : csub(ph[c], fd), flip_f);
            if (zero_f) h[c] = C<R>{R(0), R(0)};
        }
        LinkIO<P, RECON>::load(gf, Vs, kf, u);
        su3_mult1<false>(u, h, wf);
    }
    {
        C<R> ph[3], pd[3], h[3], u[9];
        load_spin<P, NC>(in, Vs, nb, hh, ph);
        load_spin<P, NC>(in, Vs, nb, ps, pd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const C<R> fd = times_f(pd[c], IM, neg);
            h[c] = cxsign(SF > 0 ? csub(ph[c], fd) : cadd(ph[c], fd), flip_b);
            if (zero_b) h[c] = C<R>{R(0), R(0)};
        }
        LinkIO<P, RECON>::load(gb, Vs, kb, u);
        // sum = w_f + U^dag h
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            C<R> t = cmacc(wf[a], u[0 + a], h[0]);
            t = cmacc(t, u[3 + a], h[1]);
            sum[a] = cmacc(t, u[6 + a], h[2]);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cadd(acc[c], sum[c]);
        const C<R> d{madd(R(2), wf[c].re, -sum[c].re), madd(R(2), wf[c].im, -sum[c].im)};  // w_f - w_b
        const C<R> gw = times_f(d, IM, IM ? !neg : neg);                      // conj(f) (w_f - w_b)
        acc[LO + c] = SF > 0 ? cadd(acc[LO + c], gw) : csub(acc[LO + c], gw);
    }
}

template <int P, int RECON, bool DAG, int MU, bool NC, class R>
__device__ __forceinline__ void half_dir(const Geom &g, const void *in, const char *gdir, int s, int c, int hh,
                                         C<R> (&acc)[9]) {
    const int L = g.L[MU], st = g.stride[MU];
    const int sf = WD_IDX(g, (c == L - 1) ? s - (L - 1) * st : s + st, g.V, 1);
    const int sb = WD_IDX(g, (c == 0) ? s + (L - 1) * st : s - st, g.V, 2);
    half_pair<P, RECON, DAG, MU < 2 ? 3 : 6, NC>(MU, in, g.Vs, sf, gdir, s, MU == 3 && g.antiperiodic && c == L - 1,
                                                sb, gdir, sb, MU == 3 && g.antiperiodic && c == 0, hh, acc,
                                                MU == 3 && g.split_t && c == L - 1, MU == 3 && g.split_t && c == 0);
}

template <int P, int RECON, bool DAG, int MU, bool NC, class R>
__device__ __forceinline__ void half_dir_eo(const Geom &g, const void *in, const char *gp, const char *gq, int k,
                                            int n, int c, int hh, C<R> (&acc)[9]) {
    const int L = g.L[MU], st = g.stride[MU];
    const int nf = WD_IDX(g, (c == L - 1) ? n - (L - 1) * st : n + st, 2 * g.V, 3);
    const int nb = WD_IDX(g, (c == 0) ? n + (L - 1) * st : n - st, 2 * g.V, 4);
    half_pair<P, RECON, DAG, MU < 2 ? 3 : 6, NC>(MU, in, g.Vs, nf >> 1, gp, k, MU == 3 && g.antiperiodic && c == L - 1,
                                                nb >> 1, gq, nb >> 1, MU == 3 && g.antiperiodic && c == 0, hh, acc);
}

// ------------------------------------------------------------ DF32 on packed pairs
// The DF32 form of half_pair: every complex df value is a cd2 (high parts and low
// parts packed), so each add, product and TwoSum step handles the real and the
// imaginary part in one f32x2 instruction.  Complex products are written as
// h u = h.re u + h.im (i u) and conj(u) h = h.re conj(u) + h.im (i conj(u)), with the
// parts of h broadcast once and reused by the three rows of the link.
template <bool NC>
__device__ __forceinline__ void load_spin_cd(const void *base, int Vs, int s, int sp, cd2 (&v)[3]) {
    const ulonglong2 *q = reinterpret_cast<const ulonglong2 *>(base) + (size_t)(3 * sp) * Vs + s;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const ulonglong2 t = ldx<NC>(q + (size_t)c * Vs);
        v[c] = cd2{t.x, t.y};
    }
}

template <int RECON>
__device__ __forceinline__ void load_link_cd(const char *gdir, int Vs, int s, cd2 (&u)[9]) {
    if constexpr (RECON == 18) {
        const ulonglong2 *p = reinterpret_cast<const ulonglong2 *>(gdir) + s;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const ulonglong2 t = __ldg(p + (size_t)e * Vs);
            u[e] = cd2{t.x, t.y};
        }
    } else {
        C<df> w[9];
        LinkIO<DF32, RECON>::load(gdir, Vs, s, w);
#pragma unroll
        for (int e = 0; e < 9; ++e)
            u[e] = cd2{f2_pack(w[e].re.hi, w[e].im.hi), f2_pack(w[e].re.lo, w[e].im.lo)};
    }
}

// f z for f = +-1 or +-i
__device__ __forceinline__ cd2 cd_times_f(cd2 z, bool im, bool neg) { return cd_neg_if(im ? cd_muli(z) : z, neg); }

template <int RECON, bool DAG, int LO, bool NC>
__device__ __forceinline__ void half_pair_cd(int mu, const void *in, int Vs, int nf, const char *gf, int kf,
                                             bool flip_f, int nb, const char *gb, int kb, bool flip_b, int hh,
                                             cd2 (&acc)[9]) {
    constexpr int SF = DAG ? +1 : -1;
    const bool IM = mu == 0 || mu == 2;
    const bool neg = mu == 1 ? hh == 0 : mu == 2 ? hh != 0 : false;
    const int ps = mu < 2 ? 3 - hh : 2 + hh;
    cd2 wf[3], sum[3];
    {
        cd2 ph[3], pd[3], u[9];
        bc2 hr[3], hi[3];
        load_spin_cd<NC>(in, Vs, nf, hh, ph);
        load_spin_cd<NC>(in, Vs, nf, ps, pd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cd2 fd = cd_times_f(pd[c], IM, neg);
            const cd2 h = cd_neg_if(SF > 0 ? cd_add(ph[c], fd) : cd_sub(ph[c], fd), flip_f);
            hr[c] = bc_re(h);
            hi[c] = bc_im(h);
        }
        load_link_cd<RECON>(gf, Vs, kf, u);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cd2 t = cd_mul(hr[0], u[3 * a]);
            t = cd_mac(t, hi[0], cd_muli(u[3 * a]));
#pragma unroll
            for (int b = 1; b < 3; ++b) {
                t = cd_mac(t, hr[b], u[3 * a + b]);
                t = cd_mac(t, hi[b], cd_muli(u[3 * a + b]));
            }
            wf[a] = t;
        }
    }
    {
        cd2 ph[3], pd[3], u[9];
        bc2 hr[3], hi[3];
        load_spin_cd<NC>(in, Vs, nb, hh, ph);
        load_spin_cd<NC>(in, Vs, nb, ps, pd);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const cd2 fd = cd_times_f(pd[c], IM, neg);
            const cd2 h = cd_neg_if(SF > 0 ? cd_sub(ph[c], fd) : cd_add(ph[c], fd), flip_b);
            hr[c] = bc_re(h);
            hi[c] = bc_im(h);
        }
        load_link_cd<RECON>(gb, Vs, kb, u);
        // sum = w_f + U^dag h
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            cd2 t = wf[a];
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cd2 cu = cd_conj(u[3 * b + a]);
                t = cd_mac(t, hr[b], cu);
                t = cd_mac(t, hi[b], cd_muli(cu));
            }
            sum[a] = t;
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = cd_add(acc[c], sum[c]);
        const cd2 d = cd_sub(cd_twice(wf[c]), sum[c]);      // w_f - w_b
        const cd2 gw = cd_times_f(d, IM, IM ? !neg : neg);  // conj(f) (w_f - w_b)
        acc[LO + c] = SF > 0 ? cd_add(acc[LO + c], gw) : cd_sub(acc[LO + c], gw);
    }
}

// Directions mu0 and mu0 + 1 as a loop that is not unrolled (DF32: the unrolled
// code of all directions would miss in the instruction cache).
template <int RECON, bool DAG, bool EO, int LO, bool NC>
__device__ __forceinline__ void half_rolled(const Geom &g, const void *in, const char *gp, const char *gq,
                                            size_t gdir_bytes, int s, int n, const int (&xc)[4], int hh,
                                            cd2 (&acc)[9]) {
    const int mu0 = LO == 3 ? 0 : 2;
#pragma unroll 1
    for (int mu = mu0; mu < mu0 + 2; ++mu) {
        const int L = g.L[mu], st = g.stride[mu];
        const int c = mu == 0 ? xc[0] : mu == 1 ? xc[1] : mu == 2 ? xc[2] : xc[3];  // no indexed register array
        const int m = EO ? n : s;
        const int nf = WD_IDX(g, (c == L - 1) ? m - (L - 1) * st : m + st, EO ? 2 * g.V : g.V, EO ? 3 : 1);
        const int nb = WD_IDX(g, (c == 0) ? m + (L - 1) * st : m - st, EO ? 2 * g.V : g.V, EO ? 4 : 2);
        const bool ff = mu == 3 && g.antiperiodic && c == L - 1, fb = mu == 3 && g.antiperiodic && c == 0;
        const char *gf = gp + (size_t)mu * gdir_bytes, *gb = gq + (size_t)mu * gdir_bytes;
        if (EO) half_pair_cd<RECON, DAG, LO, NC>(mu, in, g.Vs, nf >> 1, gf, s, ff, nb >> 1, gb, nb >> 1, fb, hh, acc);
        else half_pair_cd<RECON, DAG, LO, NC>(mu, in, g.Vs, nf, gf, s, ff, nb, gb, nb, fb, hh, acc);
    }
}

// the hopping sum of lane half hh at site s (full lattice) or checkerboard index s (EO)
template <int P, int RECON, bool DAG, bool EO, bool NC = true>
__device__ __forceinline__ void hopping_half(const Geom &g, const void *in, const void *gauge, size_t gdir_bytes, int s,
                                             int hh, C<typename Real<P>::T> (&acc)[9]) {
    using R = typename Real<P>::T;
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] = C<R>{R(0), R(0)};
    if constexpr (P == DF32) {
        int xc[4], n = s;
        const char *gp = reinterpret_cast<const char *>(gauge), *gq = gp;
        if constexpr (EO) {
            n = eo_full_index(g, s, xc[0], xc[1], xc[2], xc[3]);
            gp += (size_t)(4 * g.eo_parity) * gdir_bytes;
            gq += (size_t)(4 * (1 - g.eo_parity)) * gdir_bytes;
        } else {
            int rem = s;
            xc[0] = rem % g.L[0]; rem /= g.L[0];
            xc[1] = rem % g.L[1]; rem /= g.L[1];
            xc[2] = rem % g.L[2];
            xc[3] = rem / g.L[2];
        }
        cd2 a9[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) a9[k] = cd2{0ull, 0ull};
        half_rolled<RECON, DAG, EO, 3, NC>(g, in, gp, gq, gdir_bytes, s, n, xc, hh, a9);
        half_rolled<RECON, DAG, EO, 6, NC>(g, in, gp, gq, gdir_bytes, s, n, xc, hh, a9);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float rh, ih, rl, il;
            f2_unpack(a9[k].hi, rh, ih);
            f2_unpack(a9[k].lo, rl, il);
            acc[k] = C<R>{df(rh, rl), df(ih, il)};
        }
    } else if constexpr (EO) {
        int x, y, z, t;
        const int n = eo_full_index(g, s, x, y, z, t);
        const char *gp = reinterpret_cast<const char *>(gauge) + (size_t)(4 * g.eo_parity) * gdir_bytes;
        const char *gq = reinterpret_cast<const char *>(gauge) + (size_t)(4 * (1 - g.eo_parity)) * gdir_bytes;
        half_dir_eo<P, RECON, DAG, 0, NC>(g, in, gp, gq, s, n, x, hh, acc);
        half_dir_eo<P, RECON, DAG, 1, NC>(g, in, gp + gdir_bytes, gq + gdir_bytes, s, n, y, hh, acc);
        half_dir_eo<P, RECON, DAG, 2, NC>(g, in, gp + 2 * gdir_bytes, gq + 2 * gdir_bytes, s, n, z, hh, acc);
        half_dir_eo<P, RECON, DAG, 3, NC>(g, in, gp + 3 * gdir_bytes, gq + 3 * gdir_bytes, s, n, t, hh, acc);
    } else {
        int rem = s;
        const int x = rem % g.L[0]; rem /= g.L[0];
        const int y = rem % g.L[1]; rem /= g.L[1];
        const int z = rem % g.L[2];
        const int t = rem / g.L[2];
        const char *gb = reinterpret_cast<const char *>(gauge);
        half_dir<P, RECON, DAG, 0, NC>(g, in, gb, s, x, hh, acc);
        half_dir<P, RECON, DAG, 1, NC>(g, in, gb + gdir_bytes, s, y, hh, acc);
        half_dir<P, RECON, DAG, 2, NC>(g, in, gb + 2 * gdir_bytes, s, z, hh, acc);
        half_dir<P, RECON, DAG, 3, NC>(g, in, gb + 3 * gdir_bytes, s, t, hh, acc);
    }
}

__device__ __forceinline__ double shfl16(double v) { return __shfl_xor_sync(0xffffffffu, v, 16); }
__device__ __forceinline__ df shfl16(df v) {
    return df(__shfl_xor_sync(0xffffffffu, v.hi, 16), __shfl_xor_sync(0xffffffffu, v.lo, 16));
}
// spin 2 + hh of this lane's accumulator completes the partner's spin 3 - hh';
// called by all 32 lanes of the warp
template <class R> __device__ __forceinline__ void exchange_halves(C<R> (&acc)[9]) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const C<R> o{shfl16(acc[6 + c].re), shfl16(acc[6 + c].im)};
        acc[3 + c] = cadd(acc[3 + c], o);
    }
}

// The components of a site one thread owns in an epilogue: all 12, or the 6 of
// spins hh and 3 - hh (two lanes per site).  comp(k) is the global component of
// local component k.
struct SiteAll {
    static constexpr int N = 12;
    __device__ __forceinline__ int comp(int k) const { return k; }
};
struct SiteHalf {
    static constexpr int N = 6;
    int hh;
    __device__ __forceinline__ int comp(int k) const { return k < 3 ? 3 * hh + k : 3 * (3 - hh) + k - 3; }
};

template <int P, class Pt, bool NC = true, class R>
__device__ __forceinline__ void load_part(const Pt &pt, const void *base, int Vs, int s, C<R> (&v)[Pt::N]) {
    if constexpr (Pt::N == 12) {
        SpinorIO<P>::template load<NC>(base, Vs, s, v);
    } else if constexpr (P == F64) {
#pragma unroll
        for (int k = 0; k < Pt::N; ++k) {
            const double2 t = ldx<NC>(reinterpret_cast<const double2 *>(base) + (size_t)pt.comp(k) * Vs + s);
            v[k] = C<R>{t.x, t.y};
        }
    } else if constexpr (P == DF32) {
#pragma unroll
        for (int k = 0; k < Pt::N; ++k) {
            const float4 t = ldx<NC>(reinterpret_cast<const float4 *>(base) + (size_t)pt.comp(k) * Vs + s);
            v[k] = C<R>{df(t.x, t.z), df(t.y, t.w)};
        }
    } else {
        static_assert(P == F32, "partial sites: F64, DF32 and F32 layouts");
        // component c: half c % 2 of float4 array c / 2
#pragma unroll
        for (int k = 0; k < Pt::N; ++k) {
            const int c = pt.comp(k);
            const float2 t = ldx<NC>(reinterpret_cast<const float2 *>(base) + 2 * ((size_t)(c >> 1) * Vs + s) + (c & 1));
            v[k] = C<R>{t.x, t.y};
        }
    }
}

template <int P, class Pt, class R>
__device__ __forceinline__ void store_part(const Pt &pt, void *base, int Vs, int s, const C<R> (&v)[Pt::N]) {
    if constexpr (Pt::N == 12) {
        SpinorIO<P>::store(base, Vs, s, v);
    } else if constexpr (P == F64) {
#pragma unroll
        for (int k = 0; k < Pt::N; ++k)
            reinterpret_cast<double2 *>(base)[(size_t)pt.comp(k) * Vs + s] = make_double2(v[k].re, v[k].im);
    } else if constexpr (P == DF32) {
#pragma unroll
        for (int k = 0; k < Pt::N; ++k)
            reinterpret_cast<float4 *>(base)[(size_t)pt.comp(k) * Vs + s] =
                make_float4(v[k].re.hi, v[k].im.hi, v[k].re.lo, v[k].im.lo);
    } else {
        static_assert(P == F32, "partial sites: F64, DF32 and F32 layouts");
#pragma unroll
        for (int k = 0; k < Pt::N; ++k) {
            const int c = pt.comp(k);
            reinterpret_cast<float2 *>(base)[2 * ((size_t)(c >> 1) * Vs + s) + (c & 1)] = make_float2(v[k].re, v[k].im);
        }
    }
}

// Register budget: the FP32 and FP16 kernels are memory-bound and want many
// resident warps, so they are held to 3 blocks of 256 threads per SM (at most 85
// registers); FP64 and DF32 are arithmetic-bound and keep the compiler's choice.
template <int P> constexpr int dslash_min_blocks() { return (P == F32 || P == F16) ? 3 : 0; }

// Site tile (tile_x, in [0, gridDim.x)) and right-hand-side group (tile_y, in
// [0, gridDim.y)) of this block.  Blocks start in linear order (x fastest); numbering
// them with the RHS group fastest makes the blocks that share a site tile, and so its
// links, start together: a link then comes from DRAM once and the other RHS groups find
// it in L2, also when the gauge field is larger than L2.
__device__ __forceinline__ int tile_x() {
    return gridDim.y == 1 ? (int)blockIdx.x : (int)((blockIdx.y * gridDim.x + blockIdx.x) / gridDim.y);
}
__device__ __forceinline__ int tile_y() {
    return gridDim.y == 1 ? (int)blockIdx.y : (int)((blockIdx.y * gridDim.x + blockIdx.x) % gridDim.y);
}

// Generic Dslash kernel.  Block (bx, by) = (tile_x, tile_y) of (site_tile x rhs_tile) threads walks
// the site tiles bx, bx + gridDim.x, ... (grid-stride, so a grid smaller than the
// lattice bounds the number of reduction partials); thread (x, y) handles right-hand
// side by * rhs_tile + y, and one site (FP32, FP16) or half a site (FP64, DF32: tiles
// of site_tile / 2 sites).  Ep::site consumes the hopping sum of one site (or of the
// lane's two spins); Ep::finish runs once per thread after the loop (block and grid
// reductions, solver scalars).
template <int P, int RECON, bool DAG, class Ep, bool EO = false>
__global__ void __launch_bounds__(256, dslash_min_blocks<P>()) dslash_kernel(DslashArgs a) {
    using R = typename Real<P>::T;
    if (a.run_flag && *a.run_flag == 0) return;
    const int r = tile_y() * blockDim.y + threadIdx.y;
    const bool row = r < a.nrhs && row_on(a.sc, a.mask, r);
    const int rr = r < a.nrhs ? r : 0;
    const void *in = rhs_ptr<R>(a.in, a.in_stride, rr);
    // the field the xpay epilogues add: the hopping input unless another is given
    const void *xin = a.xsrc ? rhs_ptr<R>(a.xsrc, a.xsrc_stride, rr) : in;
    const bool zin = a.in_nonzero && *a.in_nonzero == 0;
    typename Ep::State st{};
    if constexpr (split_site<P>()) {
        // two lanes per site (blockDim.x a multiple of 32): lane l of warp w of the
        // block takes site 16 w + (l mod 16), half l / 16
        const int hh = (threadIdx.x >> 4) & 1;
        const int sl = ((threadIdx.x >> 5) << 4) | (threadIdx.x & 15);
        const int spb = blockDim.x >> 1;
        const SiteHalf pt{hh};
        for (int s0 = tile_x() * spb; s0 < a.g.V; s0 += gridDim.x * spb) {
            const int s = s0 + sl;
            const bool on = row && s < a.g.V;
            C<R> acc[9];
            if (on && !zin) hopping_half<P, RECON, DAG, EO>(a.g, in, a.gauge, a.gauge_dir, s, hh, acc);
            else
#pragma unroll
                for (int k = 0; k < 9; ++k) acc[k] = C<R>{R(0), R(0)};
            exchange_halves(acc);  // warp-uniform: row and s0 are the same for all 32 lanes
            if (on) {
                C<R> own[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) own[k] = acc[k];
                Ep::template site<P>(a, s, r, xin, own, st, pt);
            }
        }
    } else {
        const SiteAll pt{};
        for (int s0 = tile_x() * blockDim.x; s0 < a.g.V; s0 += gridDim.x * blockDim.x) {
            const int s = s0 + threadIdx.x;
            if (row && s < a.g.V) {
                C<R> acc[12];
                if (zin)
#pragma unroll
                    for (int k = 0; k < 12; ++k) acc[k] = C<R>{R(0), R(0)};
                else if constexpr (EO) hopping_eo<P, RECON, DAG>(a.g, in, a.gauge, a.gauge_dir, s, acc);
                else hopping<P, RECON, DAG>(a.g, in, a.gauge, a.gauge_dir, s, acc);
                Ep::template site<P>(a, s, r, xin, acc, st, pt);
            }
        }
    }
    Ep::template finish<P>(a, r, row, st);
}

// ---------------------------------------------------------------- epilogues
// out = in - kappa * hop     (D or D^dag applied to in)
struct EpXpay {
    struct State {};
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &, const Pt &pt) {
        C<R> p[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, p);
        const R k = R(a.kappa);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) p[c] = C<R>{p[c].re - k * acc[c].re, p[c].im - k * acc[c].im};
        store_part<P>(pt, rhs_ptr<R>(a.out, a.out_stride, r), a.g.Vs, s, p);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &, int, bool, State &) {}
};

// out = -kappa * hop (no added field); kappa = -1 gives the bare hopping term
struct EpHop {
    struct State {};
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *, C<R> (&acc)[Pt::N],
                                                State &, const Pt &pt) {
        const R k = R(-a.kappa);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) acc[c] = C<R>{k * acc[c].re, k * acc[c].im};
        store_part<P>(pt, rhs_ptr<R>(a.out, a.out_stride, r), a.g.Vs, s, acc);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &, int, bool, State &) {}
};

template <class R, int N> __device__ __forceinline__ double norm2_of(const C<R> (&v)[N]) {
    double n = 0.0;
#pragma unroll
    for (int c = 0; c < N; ++c) n += (double)v[c].re * (double)v[c].re + (double)v[c].im * (double)v[c].im;
    return n;
}

// ---------------------------------------------------------------- K right-hand sides per thread
// The plain FP32 operator with each thread applying its site's links to K right-hand sides:
// a link is loaded once and multiplies K projected half spinors, so per site and right-hand
// side the loads of links (288 bytes, 40 instructions) fall K-fold; the spinor loads are the
// same.  Rows past nrhs (a partial last group) read a valid row and store nothing.
template <int RECON, bool DAG, int MU, int K>
__device__ __forceinline__ void hop_dir_k(const DslashArgs &a, const char *gdir, const int (&row)[K], int s, int c,
                                          C<float> (&acc)[K][12]) {
    constexpr int SF = DAG ? +1 : -1;
    const Geom &g = a.g;
    const int L = g.L[MU], st = g.stride[MU];
    {
        const int sf = WD_IDX(g, (c == L - 1) ? s - (L - 1) * st : s + st, g.V, 1);
        C<float> u[9];
        LinkIO<F32, RECON>::load(gdir, g.Vs, s, u);
        const bool flip = MU == 3 && g.antiperiodic && c == L - 1;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            C<float> p[12], h[6], w[6];
            SpinorIO<F32>::load(rhs_ptr<float>(a.in, a.in_stride, row[k]), g.Vs, sf, p);
            project<MU, SF>(p, h);
            su3_mult<false>(u, h, w, flip);
            accumulate<MU, SF>(acc[k], w);
        }
    }
    {
        const int sb = WD_IDX(g, (c == 0) ? s + (L - 1) * st : s - st, g.V, 2);
        C<float> u[9];
        LinkIO<F32, RECON>::load(gdir, g.Vs, sb, u);
        const bool flip = MU == 3 && g.antiperiodic && c == 0;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            C<float> p[12], h[6], w[6];
            SpinorIO<F32>::load(rhs_ptr<float>(a.in, a.in_stride, row[k]), g.Vs, sb, p);
            project<MU, -SF>(p, h);
            su3_mult<true>(u, h, w, flip);
            accumulate<MU, -SF>(acc[k], w);
        }
    }
}

// K = 2 is held to 128 registers (two blocks of 256 per SM; the compiler's choice is 152, and
// the cap costs 32 bytes of spills): 4 % faster at 12 right-hand sides.  K = 3, 4 keep theirs.
template <int RECON, bool DAG, int K>
__global__ void __launch_bounds__(256, K == 2 ? 2 : 1) dslash_multi_kernel(DslashArgs a) {
    const int r0 = (tile_y() * blockDim.y + threadIdx.y) * K;
    if (r0 >= a.nrhs) return;  // no block-wide step follows
    int row[K];
#pragma unroll
    for (int k = 0; k < K; ++k) row[k] = r0 + k < a.nrhs ? r0 + k : a.nrhs - 1;
    const char *gb = reinterpret_cast<const char *>(a.gauge);
    for (int s0 = tile_x() * blockDim.x; s0 < a.g.V; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        if (s >= a.g.V) continue;
        int rem = s;
        const int x = rem % a.g.L[0]; rem /= a.g.L[0];
        const int y = rem % a.g.L[1]; rem /= a.g.L[1];
        const int z = rem % a.g.L[2];
        const int t = rem / a.g.L[2];
        C<float> acc[K][12];
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[k][c] = C<float>{0.f, 0.f};
        hop_dir_k<RECON, DAG, 0, K>(a, gb, row, s, x, acc);
        hop_dir_k<RECON, DAG, 1, K>(a, gb + a.gauge_dir, row, s, y, acc);
        hop_dir_k<RECON, DAG, 2, K>(a, gb + 2 * a.gauge_dir, row, s, z, acc);
        hop_dir_k<RECON, DAG, 3, K>(a, gb + 3 * a.gauge_dir, row, s, t, acc);
        const float kap = (float)a.kappa;
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (r0 + k >= a.nrhs) break;
            C<float> p[12];
            SpinorIO<F32>::load(a.xsrc ? rhs_ptr<float>(a.xsrc, a.xsrc_stride, row[k]) : rhs_ptr<float>(a.in, a.in_stride, row[k]),
                                a.g.Vs, s, p);
#pragma unroll
            for (int c = 0; c < 12; ++c) p[c] = C<float>{p[c].re - kap * acc[k][c].re, p[c].im - kap * acc[k][c].im};
            SpinorIO<F32>::store(rhs_ptr<float>(a.out, a.out_stride, row[k]), a.g.Vs, s, p);
        }
    }
}

}  // namespace wd
