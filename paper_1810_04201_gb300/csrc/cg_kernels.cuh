// Dslash epilogues of the CG solvers: the vector updates and reductions of one CG
// step are fused into the operator kernel that produces their input, and the
// scalar recursion (alpha, beta, stopping test) runs in the last block to finish.
//
// CG on the normal equations (section 2.2; Hestenes-Stiefel with squared norms):
//   setup  db = D^dag b, t = D x0, r = db - D^dag t, p = r, rho = |r|^2
//   step   t = D p;            alpha = rho / |t|^2              (EpCG1)
//          q = D^dag t; r -= alpha q; x += alpha p; rho' = |r|^2 (EpCG2 / EpCG2Mixed)
//          beta = rho' / rho; p = r + beta p                     (k_xpby)
//   stop   |r|^2 <= tol^2 |D^dag b|^2
// Mixed precision: the step runs on low-precision fields (p, t, r in the inner
// precision, the partial solution xs in FP32); when |r|^2 drops below delta^2
// times its value at the last update (or below the tolerance), a reliable update
// runs in FP64: x += xs, xs = 0, r = D^dag (b - D x), rho = |r|^2, and r is
// copied back to the inner precision.  An FP16 iteration is also corrected in FP32
// in between (EpCorrect): r = r64 - A xs from the last FP64 residual r64.
#pragma once
#include "dslash.cuh"
#include "blas.cuh"

namespace wd {

// |v|^2 of one site (or the lane's half site) of an FP32 or FP16-storage field of the
// inner iteration: the at most 24 squares are summed in FP32 (relative error below
// 24 u = 1.4e-6, far below what an FP32 recursion resolves) and only the site's total
// goes on in FP64.  Squaring in FP64 takes 24 FP64 multiply-adds per site and
// right-hand side on a part with 2 FP64 FMA per SM and clock: 40 us of FP64 pipe per
// half-lattice pass at 32^3 x 64, and 0.3 ms per pass with 12 right-hand sides at
// 24^3 x 48.  FP64 and DF32 fields keep the generic FP64 sum.
template <int N> __device__ __forceinline__ double norm2_of(const C<float> (&v)[N]) {
    float n = 0.f;
#pragma unroll
    for (int c = 0; c < N; ++c) n = fmaf(v[c].re, v[c].re, fmaf(v[c].im, v[c].im, n));
    return (double)n;
}

// Block + grid reduction of NV doubles per row; `fin(row, tot)` runs once per
// enabled row, in thread (0, 0) of the last block, rows in order.
template <int NV, class F>
__device__ __forceinline__ bool reduce_finish(const DslashArgs &a, double (&v)[NV], F &&fin) {
    __shared__ double smem[WD_MAX_RHS * 8 * NV];
    __shared__ double tot[WD_MAX_RHS * NV];
    block_reduce_rows<NV>(v, smem);
    const int r = tile_y() * blockDim.y + threadIdx.y;
    if (threadIdx.x == 0 && r < a.nrhs)
#pragma unroll
        for (int k = 0; k < NV; ++k) a.partial[((size_t)r * NV + k) * gridDim.x + tile_x()] = v[k];
    const bool last = last_block(a.counter);
    if (last) {
        sum_partials<NV>(a.partial, gridDim.x, a.nrhs, tot);
        if (threadIdx.x == 0 && threadIdx.y == 0) {
            for (int row = 0; row < a.nrhs; ++row)
                if (row_on(a.sc, a.mask, row)) fin(row, tot + row * NV);
            *a.counter = 0;
        }
    }
    return last;
}

__device__ __forceinline__ bool is_fin(double x) { return isfinite(x); }

template <class R, int N> __device__ __forceinline__ void xpay_site(C<R> (&p)[N], const C<R> (&acc)[N], R k) {
#pragma unroll
    for (int c = 0; c < N; ++c) p[c] = C<R>{p[c].re - k * acc[c].re, p[c].im - k * acc[c].im};
}

// db = D^dag b (out); |db|^2 -> rhs2, |b|^2 -> b2, tol2 *= rhs2
struct EpSetupDb {
    struct State { double v[2]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> p[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, p);
        st.v[1] += norm2_of(p);
        xpay_site(p, acc, R(a.kappa));
        st.v[0] += norm2_of(p);
        store_part<P>(pt, rhs_ptr<R>(a.out, a.out_stride, r), a.g.Vs, s, p);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<2>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            c.rhs2 = t[0];
            c.b2 = t[1];
            c.tol2 *= t[0];
        });
    }
};

// q = D^dag t; r = db - q (a1), p = r (a2); rho = |r|^2; rows already converged stop.
// With a zero start vector (in_nonzero flag 0) t was never formed: q = 0, r = db.
struct EpSetupR {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> q[Pt::N], d[Pt::N];
        if (a.in_nonzero && *a.in_nonzero == 0) {
#pragma unroll
            for (int c = 0; c < Pt::N; ++c) q[c] = C<R>{R(0), R(0)};
        } else {
            load_part<P>(pt, in, a.g.Vs, s, q);
            xpay_site(q, acc, R(a.kappa));
        }
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, d);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) d[c] = csub(d[c], q[c]);
        st.v[0] += norm2_of(d);
        store_part<P>(pt, rhs_ptr<R>(a.a1, a.a1_stride, r), a.g.Vs, s, d);
        store_part<P>(pt, rhs_ptr<R>(a.a2, a.a2_stride, r), a.g.Vs, s, d);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            c.rho = t[0];
            c.rmax2 = t[0];
            c.rmax2_lo = t[0];
            c.iter = 0;
            if (!is_fin(t[0])) { c.status = WD_ERR_NONFINITE; c.active = 0; }
            else if (t[0] <= c.tol2) { c.status = WD_OK; c.active = 0; }
            else if (c.max_iter <= 0) { c.status = WD_ERR_NOT_CONVERGED; c.active = 0; }
        });
    }
};

// t = D p (out); pAp = |t|^2; alpha = rho / pAp
struct EpCG1 {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> p[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, p);
        xpay_site(p, acc, R(a.kappa));
        st.v[0] += norm2_of(p);
        store_part<P>(pt, rhs_ptr<R>(a.out, a.out_stride, r), a.g.Vs, s, p);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            c.pAp = t[0];
            if (!is_fin(t[0])) { c.status = WD_ERR_NONFINITE; c.active = 0; c.alpha = 0.0; }
            else if (!(t[0] > 0.0)) { c.status = WD_ERR_BREAKDOWN; c.active = 0; c.alpha = 0.0; }
            else c.alpha = c.rho / t[0];
        });
    }
};

// FP64 step: q = D^dag t; r -= alpha q (a1); x += alpha p (a2, p = a0); rho' = |r|^2
struct EpCG2 {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        const R alpha = R(a.sc[r].alpha);
        C<R> q[Pt::N], v[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, q);
        xpay_site(q, acc, R(a.kappa));
        void *rr = rhs_ptr<R>(a.a1, a.a1_stride, r);
        load_part<P>(pt, rr, a.g.Vs, s, v);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) v[c] = C<R>{v[c].re - alpha * q[c].re, v[c].im - alpha * q[c].im};
        st.v[0] += norm2_of(v);
        store_part<P>(pt, rr, a.g.Vs, s, v);
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, q);
        void *xr = rhs_ptr<R>(a.a2, a.a2_stride, r);
        load_part<P>(pt, xr, a.g.Vs, s, v);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) v[c] = C<R>{v[c].re + alpha * q[c].re, v[c].im + alpha * q[c].im};
        store_part<P>(pt, xr, a.g.Vs, s, v);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            const double rn = t[0];
            c.iter += 1;
            c.rho_new = rn;
            if (!is_fin(rn)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
            c.beta = rn / c.rho;
            c.rho = rn;
            if (rn <= c.tol2) { c.status = WD_OK; c.active = 0; }
            else if (c.iter >= c.max_iter) { c.status = WD_ERR_NOT_CONVERGED; c.active = 0; }
        });
    }
};

// Mixed step (inner precision P): q = D^dag t; r -= alpha q (a1, P); xs += alpha p
// (a2, FP32; p = a0, P); rho' = |r|^2.  Decides the reliable update and sets the
// if-condition (cond) when any row needs one.
struct EpCG2Mixed {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        const R alpha = R(a.sc[r].alpha);
        C<R> q[Pt::N], v[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, q);
        xpay_site(q, acc, R(a.kappa));
        void *rr = rhs_ptr<R>(a.a1, a.a1_stride, r);
        load_part<P>(pt, rr, a.g.Vs, s, v);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) v[c] = C<R>{v[c].re - alpha * q[c].re, v[c].im - alpha * q[c].im};
        st.v[0] += norm2_of(v);
        store_part<P>(pt, rr, a.g.Vs, s, v);
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, q);
        C<float> xs[Pt::N];
        void *xr = rhs_ptr<R>(a.a2, a.a2_stride, r);
        load_part<F32>(pt, xr, a.g.Vs, s, xs);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c)
            xs[c] = C<float>{xs[c].re + float(alpha * q[c].re), xs[c].im + float(alpha * q[c].im)};
        store_part<F32>(pt, xr, a.g.Vs, s, xs);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        __shared__ int any;
        if (threadIdx.x == 0 && threadIdx.y == 0) any = 0;
        const bool last = reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            const double rn = t[0];
            c.iter += 1;
            c.rho_new = rn;
            if (!is_fin(rn)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
            if (c.iter > c.max_iter) { c.status = WD_ERR_NOT_CONVERGED; c.active = 0; return; }
            if (rn <= c.tol2 || rn < c.delta2 * c.rmax2 || c.iter >= c.max_iter) {
                c.do_update = 1;
                any = 1;
            } else if (rn < c.delta2_lo * c.rmax2_lo) {
                c.do_correct = 1;  // beta and rho follow from the corrected residual
                any = 1;
            } else {
                c.beta = rn / c.rho;
                c.rho = rn;
                c.rmax2 = fmax(c.rmax2, rn);
                c.rmax2_lo = fmax(c.rmax2_lo, rn);
            }
        });
        // the if-condition keeps its value across loop iterations: set it every time
        if (last && a.cond && threadIdx.x == 0 && threadIdx.y == 0)
            cudaGraphSetConditional((cudaGraphConditionalHandle)a.cond, any ? 1u : 0u);
    }
};

// Reliable update, FP64: q = D^dag t (t = D x); r = db - q (a1, db = a0); rho = |r|^2
struct EpReliable {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> q[Pt::N], d[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, q);
        xpay_site(q, acc, R(a.kappa));
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, d);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) d[c] = csub(d[c], q[c]);
        st.v[0] += norm2_of(d);
        store_part<P>(pt, rhs_ptr<R>(a.a1, a.a1_stride, r), a.g.Vs, s, d);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            const double rt = t[0];
            c.reliable += 1;
            if (!is_fin(rt)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
            c.beta = rt / c.rho;
            c.rho = rt;
            c.rmax2 = rt;
            c.rmax2_lo = rt;
            if (rt <= c.tol2) { c.status = WD_OK; c.active = 0; }
            else if (c.iter >= c.max_iter) { c.status = WD_ERR_NOT_CONVERGED; c.active = 0; }
            if (!c.active && a.state) {
                // this update checked the x the row returns: state[3] counts such rows, and
                // state[4] (the final check's run flag where a plan allows) drops to 0
                // once every row has stopped this way
                c.true_n2 = rt;
                a.state[3] += 1;
                a.state[4] = a.state[3] < a.nrhs;
            }
        });
    }
};

// FP32 correction of an FP16 inner iteration (a P = FP32 kernel): with x = x64 + xs and
// r64 = b' - A x64 the FP64 residual of the last reliable update (a0), the residual of x
// is r64 - A xs; here q = (A xs) from the second operator pass, r = r64 - q goes to the
// inner field (a1, FP16 storage) and rho = |r|^2.  Its error, about 2^-24 |r64|, stays
// below the FP16 recursion's as long as |r| > 2^-24 |r64| / 1e-2, which the FP64
// threshold delta keeps.  No counterpart in the paper (a three-level reliable update).
template <int SP>
struct EpCorrect {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        static_assert(P == F32, "the correction runs in FP32");
        C<R> q[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, q);
        xpay_site(q, acc, R(a.kappa));
        C<double> b[Pt::N];
        load_part<F64>(pt, rhs_ptr<double>(a.a0, a.a0_stride, r), a.g.Vs, s, b);
        C<float> d[Pt::N];
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) d[c] = C<float>{float(b[c].re) - q[c].re, float(b[c].im) - q[c].im};
        st.v[0] += norm2_of(d);
        store_part<SP>(pt, rhs_ptr<float>(a.a1, a.a1_stride, r), a.g.Vs, s, d);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) {
            Scalars &c = a.sc[row];
            const double rt = t[0];
            c.corrections += 1;
            if (!is_fin(rt)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
            c.beta = rt / c.rho;
            c.rho = rt;
            c.rmax2 = fmax(c.rmax2, rt);
            c.rmax2_lo = rt;
        });
    }
};

// Final check, pass 1: t = D x (out); |b - t|^2 -> true_b2 (b = a0)
struct EpTrue1 {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> p[Pt::N], b[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, p);
        xpay_site(p, acc, R(a.kappa));
        store_part<P>(pt, rhs_ptr<R>(a.out, a.out_stride, r), a.g.Vs, s, p);
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, b);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) b[c] = csub(b[c], p[c]);
        st.v[0] += norm2_of(b);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) { a.sc[row].true_b2 = t[0]; });
    }
};

// Final check, pass 2: q = D^dag t; |db - q|^2 -> true_n2 (db = a0)
struct EpTrue2 {
    struct State { double v[1]; };
    template <int P, class R, class Pt>
    static __device__ __forceinline__ void site(const DslashArgs &a, int s, int r, const void *in, C<R> (&acc)[Pt::N],
                                                State &st, const Pt &pt) {
        C<R> q[Pt::N], d[Pt::N];
        load_part<P>(pt, in, a.g.Vs, s, q);
        xpay_site(q, acc, R(a.kappa));
        load_part<P>(pt, rhs_ptr<R>(a.a0, a.a0_stride, r), a.g.Vs, s, d);
#pragma unroll
        for (int c = 0; c < Pt::N; ++c) d[c] = csub(d[c], q[c]);
        st.v[0] += norm2_of(d);
    }
    template <int P>
    static __device__ __forceinline__ void finish(const DslashArgs &a, int, bool, State &st) {
        reduce_finish<1>(a, st.v, [&](int row, const double *t) { a.sc[row].true_n2 = t[0]; });
    }
};

}  // namespace wd
