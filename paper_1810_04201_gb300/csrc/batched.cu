// Batched solver: many independent lattices (own dims, links, kappa, source) in
// one persistent cooperative kernel, mixed-precision CG with FP64 reliable
// updates (section 2.3: a new U and eta per solve; section 2.2: CG on the normal
// equations).
//
// Work list: every lattice is cut into tiles of kTile sites; the tiles of all
// lattices form one list that the resident blocks walk (block b takes tiles b,
// b + grid, ...).  A CG step is a sequence of phases separated by grid barriers;
// per-lattice reductions use one partial per tile and the block that finishes a
// lattice's last tile sums them in tile order (deterministic) and advances that
// lattice's scalar recursion, so every phase needs exactly one barrier.
// Converged lattices drop out of the list; the kernel ends when none is left.
// The FP64 phases (setup, reliable updates, final check) run two lanes per site
// with paired hops, like the FP64 Dslash kernel; a zero start vector skips the
// setup's D x0 and D^dag D x0; a reliable update that stops a lattice doubles as
// its final check.
//
// Grid barriers spin on a generation counter with a cycle limit: when it runs
// out the waiting block raises an error flag, every block leaves the kernel at
// its next barrier, and the host reports WD_ERR_TIMEOUT for every lattice.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "cg_kernels.cuh"
#include "plan.cuh"
#include "wd_host.h"

using namespace wd;

namespace wd {

constexpr int kTile = 128;
constexpr int kHalfTile = kTile / 2;  // sites of one pass of the two-lane FP64 phases
constexpr int kPart = 4;              // partial sums per tile
// A reliable update that delta triggers waits up to this many iterations, while the
// lattice's CG steps go on, so that the updates of many lattices share one update phase
// (three grid barriers and a walk over every tile).  Convergence and the iteration limit
// still update at once.
constexpr int kDeferIters = 4;

struct LatDesc {
    Geom g;
    double kappa;
    const void *g64, *gs;
    size_t gdir64, gdirs;
    void *b, *x, *db, *r, *t, *rs, *ps, *ts, *xs;
    int tile0, ntiles;
};

struct BatchArgs {
    const LatDesc *lat;
    Scalars *sc;         // per lattice
    unsigned *lcount;    // per lattice tile tickets
    double *tpart;       // per tile partials (2 values)
    const int *tile_lat; // lattice of each tile
    int ntiles, nlat, max_iter;
    unsigned *bar_count, *bar_gen;
    int *flags;          // [0] error, [1] any reliable update pending, [2] iterations run, [3] never set
    int *lstate;         // per lattice: [0] start vector nonzero, [1] the last reliable update was the final check
    long long spin_limit;
    int stall_test;      // block 0 first waits on flags[3], which nothing sets
};

// Bounded grid barrier (all blocks are co-resident: cooperative launch).
__device__ bool grid_barrier(const BatchArgs &a) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = a.bar_gen;
        volatile int *err = a.flags;
        const unsigned my = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            *a.bar_count = 0;
            __threadfence();
            atomicAdd(a.bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == my) {
                if (*err) break;
                if (clock64() - t0 > a.spin_limit) {
                    atomicExch(a.flags, 1);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok = *err == 0;
    }
    __syncthreads();
    return ok;
}

// Block reduction of NV values, one partial per tile, and the per-lattice finish
// in the block that completes the lattice's last tile (`fin(l, totals)`, thread 0).
template <int NV, class F>
__device__ void tile_reduce(const BatchArgs &a, const LatDesc &L, int g, int l, double (&v)[NV], F &&fin) {
    __shared__ double red[8 * NV];
    __shared__ int last;
    block_reduce_rows<NV>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) a.tpart[(size_t)g * kPart + k] = v[k];
        __threadfence();
        last = atomicAdd(a.lcount + l, 1u) == (unsigned)L.ntiles - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) s[k] = 0.0;
    for (int i = threadIdx.x; i < L.ntiles; i += blockDim.x)
#pragma unroll
        for (int k = 0; k < NV; ++k) s[k] += __ldcg(a.tpart + (size_t)(L.tile0 + i) * kPart + k);
    __syncthreads();
    block_reduce_rows<NV>(s, red);
    if (threadIdx.x == 0) {
        a.lcount[l] = 0;
        fin(l, s);
    }
    __syncthreads();
}

// One phase: walk the tiles of the lattices selected by `want(sc, lattice)`, one
// thread per site.
template <class W, class F>
__device__ void for_tiles(const BatchArgs &a, W &&want, F &&body) {
    __shared__ LatDesc L;
    __shared__ int run;
    for (int g = blockIdx.x; g < a.ntiles; g += gridDim.x) {
        const int l = a.tile_lat[g];
        if (threadIdx.x == 0) {
            run = want(a.sc[l], l);
            if (run) L = a.lat[l];
        }
        __syncthreads();
        if (run) {
            const int s = (g - L.tile0) * kTile + threadIdx.x;
            body(L, g, l, s, s < L.g.V);
        }
        __syncthreads();
    }
}

// The FP64 phases run two lanes per site like the FP64 Dslash kernel: lanes l and
// l ^ 16 of a warp share a site (lane half hh), so a tile takes two passes of
// kHalfTile sites; `body(L, g, l, sl, hh)` gets the lane's site offset sl within a pass.
template <class W, class F>
__device__ void for_tiles_half(const BatchArgs &a, W &&want, F &&body) {
    __shared__ LatDesc L;
    __shared__ int run;
    const int hh = (threadIdx.x >> 4) & 1;
    const int sl = ((threadIdx.x >> 5) << 4) | (threadIdx.x & 15);
    for (int g = blockIdx.x; g < a.ntiles; g += gridDim.x) {
        const int l = a.tile_lat[g];
        if (threadIdx.x == 0) {
            run = want(a.sc[l], l);
            if (run) L = a.lat[l];
        }
        __syncthreads();
        if (run) body(L, g, l, sl, hh);
        __syncthreads();
    }
}

// The hopping sum of lane half hh at site s (zero where `on` is false), exchanged
// with the partner lane: the lane's two spins (SiteHalf).  Every lane of the warp
// calls it.  Plain loads: the fields change between the phases of one launch.
template <int RECON, bool DAG>
__device__ __forceinline__ void hop64_half(const LatDesc &L, const void *in, int s, int hh, bool on,
                                           C<double> (&own)[6]) {
    C<double> acc[9];
    if (on) hopping_half<F64, RECON, DAG, false, false>(L.g, in, L.g64, L.gdir64, s, hh, acc);
    else
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] = C<double>{0.0, 0.0};
    exchange_halves(acc);
#pragma unroll
    for (int k = 0; k < 6; ++k) own[k] = acc[k];
}

// Five blocks of 128 threads per SM (96 registers): the inner FP32 phases, which wait on
// loads, gain more from the extra warps than the FP64 phases lose to spills (C5: 54.0 ms
// at four blocks, 52.7 at five).
template <int SP, int RECON, int RIN>
__global__ void __launch_bounds__(kTile, 5) k_batched_cg(BatchArgs a) {
    using RS = typename Real<SP>::T;
    auto all = [](const Scalars &, int) { return 1; };
    auto active = [](const Scalars &c, int) { return c.active; };
    auto updating = [](const Scalars &c, int) { return c.active && (c.do_update || c.pending); };
    auto x0_nonzero = [&](const Scalars &, int l) { return a.lstate[2 * l]; };
    auto unchecked = [&](const Scalars &, int l) { return 1 - a.lstate[2 * l + 1]; };

    if (a.stall_test && blockIdx.x == 0 && threadIdx.x == 0) {
        // a wait that runs out: nothing ever sets flags[3]
        const long long t0 = clock64();
        volatile int *never = a.flags + 3;
        while (*never == 0 && clock64() - t0 <= a.spin_limit) __nanosleep(64);
        if (*never == 0) atomicExch(a.flags, 1);
    }

    // ---- setup (FP64, two lanes per site)
    // S1: db = D^dag b ; |db|^2, |b|^2, |x0|^2 (a zero start vector skips S2 and the hop of S3)
    for_tiles_half(a, all, [&](const LatDesc &L, int g, int l, int sl, int hh) {
        const SiteHalf pt{hh};
        double v[3] = {0.0, 0.0, 0.0};
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
            const bool on = s < L.g.V;
            C<double> acc[6], p[6];
            hop64_half<RECON, true>(L, L.b, s, hh, on, acc);
            if (on) {
                load_part<F64, SiteHalf, false>(pt, L.b, L.g.Vs, s, p);
                v[1] += norm2_of(p);
                xpay_site(p, acc, L.kappa);
                v[0] += norm2_of(p);
                store_part<F64>(pt, L.db, L.g.Vs, s, p);
                load_part<F64, SiteHalf, false>(pt, L.x, L.g.Vs, s, p);
                v[2] += norm2_of(p);
            }
        }
        tile_reduce<3>(a, L, g, l, v, [&](int l2, const double *t) {
            Scalars &c = a.sc[l2];
            c.rhs2 = t[0];
            c.b2 = t[1];
            c.tol2 *= t[0];
            a.lstate[2 * l2] = !(t[2] == 0.0);  // NaN counts as nonzero
        });
    });
    if (!grid_barrier(a)) return;
    // S2: t = D x0
    for_tiles_half(a, x0_nonzero, [&](const LatDesc &L, int g, int, int sl, int hh) {
        const SiteHalf pt{hh};
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
            const bool on = s < L.g.V;
            C<double> acc[6], p[6];
            hop64_half<RECON, false>(L, L.x, s, hh, on, acc);
            if (on) {
                load_part<F64, SiteHalf, false>(pt, L.x, L.g.Vs, s, p);
                xpay_site(p, acc, L.kappa);
                store_part<F64>(pt, L.t, L.g.Vs, s, p);
            }
        }
    });
    if (!grid_barrier(a)) return;
    // S3: r = db - D^dag t (r = db for x0 = 0) ; rho = |r|^2
    for_tiles_half(a, all, [&](const LatDesc &L, int g, int l, int sl, int hh) {
        const SiteHalf pt{hh};
        const bool nz = a.lstate[2 * l] != 0;
        double v[1] = {0.0};
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
            const bool on = s < L.g.V;
            C<double> acc[6], q[6], d[6];
            hop64_half<RECON, true>(L, L.t, s, hh, on && nz, acc);
            if (on) {
                if (nz) {
                    load_part<F64, SiteHalf, false>(pt, L.t, L.g.Vs, s, q);
                    xpay_site(q, acc, L.kappa);
                } else {
#pragma unroll
                    for (int k = 0; k < 6; ++k) q[k] = C<double>{0.0, 0.0};
                }
                load_part<F64, SiteHalf, false>(pt, L.db, L.g.Vs, s, d);
#pragma unroll
                for (int k = 0; k < 6; ++k) d[k] = csub(d[k], q[k]);
                v[0] += norm2_of(d);
                store_part<F64>(pt, L.r, L.g.Vs, s, d);
            }
        }
        tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) {
            Scalars &c = a.sc[l2];
            c.rho = t[0];
            c.rmax2 = t[0];
            a.lstate[2 * l2 + 1] = 0;
            if (!isfinite(t[0])) { c.status = WD_ERR_NONFINITE; c.active = 0; }
            else if (t[0] <= c.tol2) { c.status = WD_OK; c.active = 0; }
        });
    });
    if (!grid_barrier(a)) return;
    // S4: rs = ps = r (inner precision) ; xs = 0
    for_tiles(a, all, [&](const LatDesc &L, int, int, int s, bool valid) {
        if (!valid) return;
        C<double> d[12];
        SpinorIO<F64>::template load<false>(L.r, L.g.Vs, s, d);
        C<RS> w[12];
        C<float> z[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            w[c] = C<RS>{RS(d[c].re), RS(d[c].im)};
            z[c] = C<float>{0.f, 0.f};
        }
        SpinorIO<SP>::store(L.rs, L.g.Vs, s, w);
        SpinorIO<SP>::store(L.ps, L.g.Vs, s, w);
        SpinorIO<F32>::store(L.xs, L.g.Vs, s, z);
    });
    if (!grid_barrier(a)) return;

    for (int it = 0; it < a.max_iter + 2; ++it) {
        int any = 0;
        for (int l = 0; l < a.nlat; ++l) any |= a.sc[l].active;
        if (!any) break;
        if (threadIdx.x == 0 && blockIdx.x == 0) a.flags[2] = it + 1;
        // A: ts = D ps ; pAp = |ts|^2 ; alpha
        for_tiles(a, active, [&](const LatDesc &L, int g, int l, int s, bool valid) {
            double v[1] = {0.0};
            if (valid) {
                C<RS> acc[12], p[12];
                hopping<SP, RIN, false, false>(L.g, L.ps, L.gs, L.gdirs, s, acc);
                SpinorIO<SP>::template load<false>(L.ps, L.g.Vs, s, p);
                xpay_site(p, acc, RS(L.kappa));
                v[0] = norm2_of(p);
                SpinorIO<SP>::store(L.ts, L.g.Vs, s, p);
            }
            tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) {
                Scalars &c = a.sc[l2];
                c.pAp = t[0];
                if (!isfinite(t[0])) { c.status = WD_ERR_NONFINITE; c.active = 0; }
                else if (!(t[0] > 0.0)) { c.status = WD_ERR_BREAKDOWN; c.active = 0; }
                else c.alpha = c.rho / t[0];
            });
        });
        if (!grid_barrier(a)) return;
        // B: q = D^dag ts ; rs -= alpha q ; xs += alpha ps ; rho' = |rs|^2 ; decide
        for_tiles(a, active, [&](const LatDesc &L, int g, int l, int s, bool valid) {
            double v[1] = {0.0};
            if (valid) {
                const RS alpha = RS(a.sc[l].alpha);
                C<RS> acc[12], q[12], w[12];
                hopping<SP, RIN, true, false>(L.g, L.ts, L.gs, L.gdirs, s, acc);
                SpinorIO<SP>::template load<false>(L.ts, L.g.Vs, s, q);
                xpay_site(q, acc, RS(L.kappa));
                SpinorIO<SP>::template load<false>(L.rs, L.g.Vs, s, w);
#pragma unroll
                for (int c = 0; c < 12; ++c) w[c] = C<RS>{w[c].re - alpha * q[c].re, w[c].im - alpha * q[c].im};
                v[0] = norm2_of(w);
                SpinorIO<SP>::store(L.rs, L.g.Vs, s, w);
                SpinorIO<SP>::template load<false>(L.ps, L.g.Vs, s, q);
                C<float> xs[12];
                SpinorIO<F32>::template load<false>(L.xs, L.g.Vs, s, xs);
#pragma unroll
                for (int c = 0; c < 12; ++c)
                    xs[c] = C<float>{xs[c].re + float(alpha * q[c].re), xs[c].im + float(alpha * q[c].im)};
                SpinorIO<F32>::store(L.xs, L.g.Vs, s, xs);
            }
            tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) {
                Scalars &c = a.sc[l2];
                const double rn = t[0];
                c.iter += 1;
                if (!isfinite(rn)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
                if (rn <= c.tol2 || c.iter >= c.max_iter) {
                    // stopping: update now, in place of this step
                    c.do_update = 1;
                    atomicExch(a.flags + 1, 1);
                } else {
                    c.beta = rn / c.rho;
                    c.rho = rn;
                    c.rmax2 = fmax(c.rmax2, rn);
                    if (!c.pending && rn < c.delta2 * c.rmax2) {
                        c.pending = 1;
                        c.pending_since = c.iter;
                    }
                    if (c.pending && c.iter - c.pending_since >= kDeferIters) atomicExch(a.flags + 1, 1);
                }
            });
        });
        if (!grid_barrier(a)) return;
        if (*(volatile int *)(a.flags + 1)) {
            // C1: x += xs ; xs = 0  (FP64 solution accumulation)
            for_tiles(a, updating, [&](const LatDesc &L, int, int, int s, bool valid) {
                if (!valid) return;
                C<double> x[12];
                C<float> xs[12];
                SpinorIO<F64>::template load<false>(L.x, L.g.Vs, s, x);
                SpinorIO<F32>::template load<false>(L.xs, L.g.Vs, s, xs);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    x[c] = C<double>{x[c].re + (double)xs[c].re, x[c].im + (double)xs[c].im};
                    xs[c] = C<float>{0.f, 0.f};
                }
                SpinorIO<F64>::store(L.x, L.g.Vs, s, x);
                SpinorIO<F32>::store(L.xs, L.g.Vs, s, xs);
            });
            if (!grid_barrier(a)) return;
            // C2: t = D x (FP64) ; |b - t|^2 (the final check's first norm, should x stay)
            for_tiles_half(a, updating, [&](const LatDesc &L, int g, int l, int sl, int hh) {
                const SiteHalf pt{hh};
                double v[1] = {0.0};
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
                    const bool on = s < L.g.V;
                    C<double> acc[6], p[6], bb[6];
                    hop64_half<RECON, false>(L, L.x, s, hh, on, acc);
                    if (on) {
                        load_part<F64, SiteHalf, false>(pt, L.x, L.g.Vs, s, p);
                        xpay_site(p, acc, L.kappa);
                        store_part<F64>(pt, L.t, L.g.Vs, s, p);
                        load_part<F64, SiteHalf, false>(pt, L.b, L.g.Vs, s, bb);
#pragma unroll
                        for (int k = 0; k < 6; ++k) bb[k] = csub(bb[k], p[k]);
                        v[0] += norm2_of(bb);
                    }
                }
                tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) { a.sc[l2].true_b2 = t[0]; });
            });
            if (!grid_barrier(a)) return;
            // C3: r = db - D^dag t ; rho = |r|^2 (the true residual of the normal equations)
            for_tiles_half(a, updating, [&](const LatDesc &L, int g, int l, int sl, int hh) {
                const SiteHalf pt{hh};
                double v[1] = {0.0};
                for (int h2 = 0; h2 < 2; ++h2) {
                    const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
                    const bool on = s < L.g.V;
                    C<double> acc[6], q[6], d[6];
                    hop64_half<RECON, true>(L, L.t, s, hh, on, acc);
                    if (on) {
                        load_part<F64, SiteHalf, false>(pt, L.t, L.g.Vs, s, q);
                        xpay_site(q, acc, L.kappa);
                        load_part<F64, SiteHalf, false>(pt, L.db, L.g.Vs, s, d);
#pragma unroll
                        for (int k = 0; k < 6; ++k) d[k] = csub(d[k], q[k]);
                        v[0] += norm2_of(d);
                        store_part<F64>(pt, L.r, L.g.Vs, s, d);
                    }
                }
                tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) {
                    Scalars &c = a.sc[l2];
                    const double rt = t[0];
                    c.reliable += 1;
                    if (!isfinite(rt)) { c.status = WD_ERR_NONFINITE; c.active = 0; return; }
                    // beta = |r_true|^2 / |r|^2 of the previous step; a deferred update comes after
                    // this iteration's step, which set beta = rho / rho_prev and rho = |r|^2
                    c.beta = c.do_update ? rt / c.rho : rt * c.beta / c.rho;
                    c.rho = rt;
                    c.rmax2 = rt;
                    if (rt <= c.tol2) { c.status = WD_OK; c.active = 0; }
                    else if (c.iter >= c.max_iter) { c.status = WD_ERR_NOT_CONVERGED; c.active = 0; }
                    if (!c.active) {
                        // x stays as it is: this update was the final check
                        c.true_n2 = rt;
                        a.lstate[2 * l2 + 1] = 1;
                    }
                });
            });
            if (!grid_barrier(a)) return;
        }
        // D: rs = r (after a reliable update) ; ps = rs + beta ps
        for_tiles(a, active, [&](const LatDesc &L, int, int l, int s, bool valid) {
            if (!valid) return;
            const Scalars &c = a.sc[l];
            const RS beta = RS(c.beta);
            C<RS> w[12], p[12];
            if (c.do_update || (c.pending && *(volatile int *)(a.flags + 1))) {
                C<double> d[12];
                SpinorIO<F64>::template load<false>(L.r, L.g.Vs, s, d);
#pragma unroll
                for (int k = 0; k < 12; ++k) w[k] = C<RS>{RS(d[k].re), RS(d[k].im)};
                SpinorIO<SP>::store(L.rs, L.g.Vs, s, w);
            } else {
                SpinorIO<SP>::template load<false>(L.rs, L.g.Vs, s, w);
            }
            SpinorIO<SP>::template load<false>(L.ps, L.g.Vs, s, p);
#pragma unroll
            for (int k = 0; k < 12; ++k) p[k] = C<RS>{w[k].re + beta * p[k].re, w[k].im + beta * p[k].im};
            SpinorIO<SP>::store(L.ps, L.g.Vs, s, p);
        });
        if (!grid_barrier(a)) return;
        // clear the pending flags (one block owns them), then a barrier before the next step
        if (blockIdx.x == 0) {
            const bool updated = *(volatile int *)(a.flags + 1) != 0;
            __syncthreads();  // every thread has read the flag before thread 0 clears it
            for (int l = threadIdx.x; l < a.nlat; l += blockDim.x) {
                a.sc[l].do_update = 0;
                if (updated) a.sc[l].pending = 0;
            }
            if (threadIdx.x == 0) a.flags[1] = 0;
        }
        if (!grid_barrier(a)) return;
    }

    // ---- final FP64 check, for lattices whose last step was not a reliable update that
    // stopped them: t = D x, |b - t|^2 ; |db - D^dag t|^2
    for_tiles_half(a, unchecked, [&](const LatDesc &L, int g, int l, int sl, int hh) {
        const SiteHalf pt{hh};
        double v[1] = {0.0};
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
            const bool on = s < L.g.V;
            C<double> acc[6], p[6], bb[6];
            hop64_half<RECON, false>(L, L.x, s, hh, on, acc);
            if (on) {
                load_part<F64, SiteHalf, false>(pt, L.x, L.g.Vs, s, p);
                xpay_site(p, acc, L.kappa);
                store_part<F64>(pt, L.t, L.g.Vs, s, p);
                load_part<F64, SiteHalf, false>(pt, L.b, L.g.Vs, s, bb);
#pragma unroll
                for (int k = 0; k < 6; ++k) bb[k] = csub(bb[k], p[k]);
                v[0] += norm2_of(bb);
            }
        }
        tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) { a.sc[l2].true_b2 = t[0]; });
    });
    if (!grid_barrier(a)) return;
    for_tiles_half(a, unchecked, [&](const LatDesc &L, int g, int l, int sl, int hh) {
        const SiteHalf pt{hh};
        double v[1] = {0.0};
        for (int h2 = 0; h2 < 2; ++h2) {
            const int s = (g - L.tile0) * kTile + h2 * kHalfTile + sl;
            const bool on = s < L.g.V;
            C<double> acc[6], q[6], d[6];
            hop64_half<RECON, true>(L, L.t, s, hh, on, acc);
            if (on) {
                load_part<F64, SiteHalf, false>(pt, L.t, L.g.Vs, s, q);
                xpay_site(q, acc, L.kappa);
                load_part<F64, SiteHalf, false>(pt, L.db, L.g.Vs, s, d);
#pragma unroll
                for (int k = 0; k < 6; ++k) d[k] = csub(d[k], q[k]);
                v[0] += norm2_of(d);
            }
        }
        tile_reduce<1>(a, L, g, l, v, [&](int l2, const double *t) { a.sc[l2].true_n2 = t[0]; });
    });
}

// One persistent cooperative launch, captured once into a CUDA graph per argument
// set (the arguments are pointers into context workspace, stable across calls).
template <int SP, int RECON, int RIN>
static cudaError_t build_batched(BatchArgs &a, cudaGraphExec_t *exec) {
    auto k = k_batched_cg<SP, RECON, RIN>;
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kTile, 0);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int grid = per_sm * sms;
    if (grid > a.ntiles) grid = a.ntiles;
    if (grid < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kTile);
    cfg.dynamicSmemBytes = 0;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    // the legacy default stream cannot be captured: capture on a private stream
    cudaStream_t cap;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    cfg.stream = cap;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t el = cudaLaunchKernelEx(&cfg, k, a);
        e = cudaStreamEndCapture(cap, &graph);
        if (el != cudaSuccess) e = el;
    }
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    return e;
}

}  // namespace wd

extern "C" wd_status wd_cg_solve_batched(wd_ctx *const *ctxs, const double *kappas, const void *const *b,
                                         void *const *x, int n, const wd_cg_params *prm, wd_cg_result *res) {
    wd::NvtxRange nvtx_("wd_cg_solve_batched");
    if (!ctxs || n < 1 || !ctxs[0]) return WD_ERR_ARG;
    wd_ctx *c0 = ctxs[0];
    c0->launches = 0;
    if (!kappas || !b || !x || !prm || !res) return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: null argument");
    if (prm->inner_prec != WD_F32 && prm->inner_prec != WD_F16)
        return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: inner_prec must be WD_F32 or WD_F16");
    if ((prm->nrhs > 1) || !(prm->tol > 0)) return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: bad nrhs or tol");
    if (prm->normal_eq) return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: solves D^dag D only (normal_eq = 0)");
    if (prm->stop_rule != WD_STOP_NORMAL)
        return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: stops on the normal residual only");
    const Prec sp = (Prec)prm->inner_prec;
    std::vector<LatDesc> lat(n);
    std::vector<int> tile_lat;
    int ntiles = 0;
    for (int i = 0; i < n; ++i) {
        wd_ctx *c = ctxs[i];
        if (!c || !b[i] || !x[i] || !std::isfinite(kappas[i]))
            return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: null context, field or bad kappa");
        if (c->device != c0->device) return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: contexts on different devices");
        if (c->split) return fail(c0, WD_ERR_STATE, "wd_cg_solve_batched: a split sub-lattice (use wd_cg_solve_split)");
        if (link_recon(c, F64) != link_recon(c0, F64) || link_recon(c, sp) != link_recon(c0, sp))
            return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: every context needs the same link compressions");
        wd_status s;
        const void *g64, *gs;
        if ((s = gauge_get(c, F64, &g64)) != WD_OK) return fail(c0, s, c->last_error);
        if ((s = gauge_get(c, sp, &gs)) != WD_OK) return fail(c0, s, c->last_error);
        LatDesc &L = lat[i];
        L.g = c->g;
        L.kappa = kappas[i];
        L.g64 = g64;
        L.gs = gs;
        L.gdir64 = gauge_dir_bytes(c, F64);
        L.gdirs = gauge_dir_bytes(c, sp);
        const size_t f64 = spinor_bytes(F64, c->g.Vs), fsp = spinor_bytes(sp, c->g.Vs),
                     f32 = spinor_bytes(F32, c->g.Vs);
        void **p64[4] = {&L.x, &L.db, &L.r, &L.t};
        const char *n64[4] = {"bt_x", "bt_db", "bt_r", "bt_t"};
        for (int k = 0; k < 4; ++k)
            if ((s = ws_get(c, n64[k], f64, p64[k])) != WD_OK) return fail(c0, s, c->last_error);
        void **psp[3] = {&L.rs, &L.ps, &L.ts};
        const char *nsp[3] = {"bt_rs", "bt_ps", "bt_ts"};
        for (int k = 0; k < 3; ++k)
            if ((s = ws_get(c, std::string(nsp[k]) + (sp == F32 ? "32" : "16"), fsp, psp[k])) != WD_OK)
                return fail(c0, s, c->last_error);
        if ((s = ws_get(c, "bt_xs", f32, &L.xs)) != WD_OK) return fail(c0, s, c->last_error);
        L.b = const_cast<void *>(b[i]);
        L.tile0 = ntiles;
        L.ntiles = (c->g.V + kTile - 1) / kTile;
        ntiles += L.ntiles;
        tile_lat.insert(tile_lat.end(), L.ntiles, i);
    }
    // batch-wide buffers live in the first context
    cudaStream_t st = c0->stream;
    void *d_lat, *d_sc, *d_cnt, *d_part, *d_tl, *d_bar, *d_lst;
    wd_status s;
    if ((s = ws_get(c0, "bt_lat", sizeof(LatDesc) * n, &d_lat)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_sc", sizeof(Scalars) * n, &d_sc)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_cnt", sizeof(unsigned) * n, &d_cnt)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_part", sizeof(double) * kPart * ntiles, &d_part)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_lstate", sizeof(int) * 2 * n, &d_lst)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_tl", sizeof(int) * ntiles, &d_tl)) != WD_OK) return s;
    if ((s = ws_get(c0, "bt_bar", 256, &d_bar)) != WD_OK) return s;
    std::vector<Scalars> h(n);
    const double delta = prm->delta > 0 ? prm->delta : default_delta((Prec)prm->inner_prec, false);
    for (int i = 0; i < n; ++i) {
        std::memset(&h[i], 0, sizeof(Scalars));
        h[i].tol2 = prm->tol * prm->tol;
        h[i].max_iter = prm->max_iter;
        h[i].delta2 = delta * delta;
        h[i].active = 1;
        h[i].status = WD_ERR_NOT_CONVERGED;
    }
    WD_CUDA(c0, cudaMemcpyAsync(d_lat, lat.data(), sizeof(LatDesc) * n, cudaMemcpyHostToDevice, st));
    WD_CUDA(c0, cudaMemcpyAsync(d_sc, h.data(), sizeof(Scalars) * n, cudaMemcpyHostToDevice, st));
    WD_CUDA(c0, cudaMemcpyAsync(d_tl, tile_lat.data(), sizeof(int) * ntiles, cudaMemcpyHostToDevice, st));
    WD_CUDA(c0, cudaMemsetAsync(d_cnt, 0, sizeof(unsigned) * n, st));
    WD_CUDA(c0, cudaMemsetAsync(d_bar, 0, 256, st));
    for (int i = 0; i < n; ++i)
        WD_CUDA(c0, cudaMemcpyAsync(lat[i].x, x[i], spinor_bytes(F64, lat[i].g.Vs), cudaMemcpyDeviceToDevice, st));

    BatchArgs a{};
    a.lat = (const LatDesc *)d_lat;
    a.sc = (Scalars *)d_sc;
    a.lcount = (unsigned *)d_cnt;
    a.tpart = (double *)d_part;
    a.tile_lat = (const int *)d_tl;
    a.ntiles = ntiles;
    a.nlat = n;
    a.max_iter = prm->max_iter;
    a.bar_count = (unsigned *)d_bar;
    a.bar_gen = (unsigned *)d_bar + 16;
    a.flags = (int *)d_bar + 32;
    a.lstate = (int *)d_lst;
    const char *stall = getenv("WD_BATCH_STALL_TEST");
    a.stall_test = stall && std::strcmp(stall, "1") == 0;
    // about one second at GB300 clocks; a tenth of that for the stalled-wait test
    a.spin_limit = a.stall_test ? 200000000ll : 2000000000ll;

    const int r64 = link_recon(c0, F64), rin = link_recon(c0, sp);
    if (rin != r64 && r64 != 18)
        return fail(c0, WD_ERR_ARG, "wd_cg_solve_batched: with compressed FP64 links the inner precision needs the "
                                    "same compression");
    char key[160];
    snprintf(key, sizeof key, "batch|%d|%d,%d|%d|%d|%d|%d|%p|%p", (int)sp, r64, rin, n, ntiles, prm->max_iter,
             a.stall_test, d_part, d_lat);
    cudaGraphExec_t exec = (cudaGraphExec_t)graph_get(c0, key);
    if (!exec) {
        const cudaError_t e = with_recon_pair(r64, rin, [&](auto ra, auto rb) {
            constexpr int R = decltype(ra)::value, RI = decltype(rb)::value;
            return sp == F32 ? build_batched<F32, R, RI>(a, &exec) : build_batched<F16, R, RI>(a, &exec);
        });
        if (e != cudaSuccess) return cuda_fail(c0, e, "building the batched persistent CG graph");
        graph_put(c0, key, exec, {});
    }
    EventPair ev;
    WD_CUDA(c0, ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    WD_CUDA(c0, cudaEventRecord(e0, st));
    WD_CUDA(c0, cudaGraphLaunch(exec, st));
    WD_CUDA(c0, cudaEventRecord(e1, st));
    for (int i = 0; i < n; ++i)
        WD_CUDA(c0, cudaMemcpyAsync(x[i], lat[i].x, spinor_bytes(F64, lat[i].g.Vs), cudaMemcpyDeviceToDevice, st));
    int flags[4];
    WD_CUDA(c0, cudaMemcpyAsync(h.data(), d_sc, sizeof(Scalars) * n, cudaMemcpyDeviceToHost, st));
    WD_CUDA(c0, cudaMemcpyAsync(flags, (int *)d_bar + 32, sizeof flags, cudaMemcpyDeviceToHost, st));
    WD_CUDA(c0, cudaStreamSynchronize(st));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    c0->launches = 1;
    wd_status worst = WD_OK;
    for (int i = 0; i < n; ++i) {
        res[i].iters = h[i].iter;
        res[i].reliable_updates = h[i].reliable;
        res[i].inner_corrections = 0;
        res[i].true_rel_resid = h[i].rhs2 > 0 ? std::sqrt(h[i].true_n2 / h[i].rhs2) : std::sqrt(h[i].true_n2);
        res[i].true_rel_resid_b = h[i].b2 > 0 ? std::sqrt(h[i].true_b2 / h[i].b2) : std::sqrt(h[i].true_b2);
        res[i].seconds = ms * 1e-3;
        res[i].status = flags[0] ? WD_ERR_TIMEOUT : h[i].status;
        if (res[i].status != WD_OK && worst == WD_OK) worst = (wd_status)res[i].status;
    }
    if (worst != WD_OK) c0->last_error = std::string("wd_cg_solve_batched: ") + wd_status_string(worst);
    return worst;
}
