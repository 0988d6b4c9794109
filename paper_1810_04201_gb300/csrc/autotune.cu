// Autotuner for the Dslash launch shape (the paper's compile-time knobs of §7.1 --
// partition and unroll factors, number of kernel instances -- become a timed
// sweep over the thread-block shape at run time).
//
// Candidates: site_tile in {16, 32, 64, 128, 256} threads along the sites and
// rhs_tile in {1, 2, 3, 4, 6, 8, 12, 16} right-hand sides per block, with
// site_tile * rhs_tile <= 256, a multiple of 32, and rhs_tile <= nrhs (FP64 and
// DF32, two lanes per site: site_tile >= 32, i.e. site_tile / 2 sites per block); for
// FP32 also 2, 3 or 4 right-hand sides per thread (K dividing rhs_tile; not on a split
// sub-lattice, whose interior hops need the split_t form of the kernel).  Each candidate
// runs the plain D kernel twice untimed and five times timed, each timed launch with L2
// flushed before it (CUDA events on the context stream), on a non-zero input; the fastest
// is kept for (precision, nrhs) and used by every later operator call, and by the solvers
// unless wd_autotune_cg tuned their fused kernels.
#include <vector>
#include "blas.cuh"
#include "dslash.cuh"
#include "wd_host.h"

using namespace wd;

extern "C" {

wd_status wd_set_tiles(wd_ctx *c, wd_prec prec, int nrhs, int site_tile, int rhs_tile) {
    if (!c) return WD_ERR_ARG;
    if ((int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS || rhs_tile < 1 || rhs_tile > nrhs ||
        (site_tile != 16 && site_tile != 32 && site_tile != 64 && site_tile != 128 && site_tile != 256) ||
        site_tile * rhs_tile > 256 || (site_tile * rhs_tile) % 32 != 0)
        return fail(c, WD_ERR_ARG, "wd_set_tiles: unsupported tile shape");
    if (threads_per_site((Prec)prec) > 1 && site_tile % 32 != 0)
        return fail(c, WD_ERR_ARG, "wd_set_tiles: FP64 and DF32 run two lanes per site and need site_tile >= 32");
    DslashTiles t;
    t.site_tile = site_tile;
    t.rhs_tile = rhs_tile;
    c->tiles[(int)prec * 64 + nrhs] = t;
    return WD_OK;
}

wd_status wd_autotune(wd_ctx *c, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile) {
    wd::NvtxRange nvtx_("wd_autotune");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if ((int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, "wd_autotune: bad argument");
    const void *gauge;
    wd_status s = gauge_get(c, (Prec)prec, &gauge);
    if (s != WD_OK) return s;
    const size_t fb = spinor_bytes((Prec)prec, c->g.Vs);
    const size_t canon_bytes = (size_t)nrhs * c->g.V * 12 * 16;
    const size_t flush_bytes = (size_t)256 << 20;  // twice the L2 of a GB300
    void *in, *out, *canon, *flush;
    if ((s = ws_get(c, "tune_in", fb * nrhs, &in)) != WD_OK) return s;
    if ((s = ws_get(c, "tune_out", fb * nrhs, &out)) != WD_OK) return s;
    if ((s = ws_get(c, "tune_canon", canon_bytes, &canon)) != WD_OK) return s;
    if ((s = ws_get(c, "tune_flush", flush_bytes, &flush)) != WD_OK) return s;
    // a non-zero input in the field's own layout
    k_fill_hash<double><<<1024, 256, 0, c->stream>>>(static_cast<double *>(canon), canon_bytes / sizeof(double));
    WD_CUDA(c, cudaGetLastError());
    if ((s = wd_pack(c, static_cast<const double *>(canon), 1, in, prec, nrhs)) != WD_OK) return s;
    ws_release(c, "tune_canon");

    DslashArgs a{};
    a.g = c->g;
    a.in = in;
    a.out = out;
    a.in_stride = a.out_stride = fb;
    a.gauge = gauge;
    a.gauge_dir = gauge_dir_bytes(c, (Prec)prec);
    a.kappa = 0.1;
    a.nrhs = nrhs;

    const int sts[] = {16, 32, 64, 128, 256};
    const int rts[] = {1, 2, 3, 4, 6, 8, 12, 16};
    const int kts[] = {1, 2, 3, 4};
    EventPair ev;
    WD_CUDA(c, ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    float best = 1e30f;
    DslashTiles bt = tiles_for(c, (Prec)prec, nrhs);
    long long launches = 2;
    for (int st : sts)
        for (int rt : rts)
            for (int kt : kts) {
                if (rt > nrhs || st * rt > 256 || (st * rt) % 32 != 0) continue;
                if (threads_per_site((Prec)prec) > 1 && st % 32 != 0) continue;
                if (kt > 1 && (prec != WD_F32 || rt % kt != 0 || (st * rt / kt) % 32 != 0 || c->g.split_t)) continue;
                DslashTiles t;
                t.site_tile = st;
                t.rhs_tile = rt;
                t.rhs_per_thread = kt;
                for (int k = 0; k < 2; ++k)
                    WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), false, t, c->stream));
                // each timed launch starts with L2 flushed, as the bench times the operator
                float ms = 0.f;
                for (int k = 0; k < 5; ++k) {
                    WD_CUDA(c, cudaMemsetAsync(flush, k, flush_bytes, c->stream));
                    WD_CUDA(c, cudaEventRecord(e0, c->stream));
                    WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), false, t, c->stream));
                    WD_CUDA(c, cudaEventRecord(e1, c->stream));
                    WD_CUDA(c, cudaEventSynchronize(e1));
                    float m = 0.f;
                    WD_CUDA(c, cudaEventElapsedTime(&m, e0, e1));
                    ms += m;
                }
                launches += 7;
                if (ms < best) {
                    best = ms;
                    bt = t;
                }
            }
    ws_release(c, "tune_flush");
    c->tiles[(int)prec * 64 + nrhs] = bt;
    c->launches = launches;
    if (site_tile) *site_tile = bt.site_tile;
    if (rhs_tile) *rhs_tile = bt.rhs_tile;
    return WD_OK;
}

wd_status wd_get_tiles(wd_ctx *c, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile, int *rhs_per_thread) {
    if (!c || (int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS) return WD_ERR_ARG;
    const DslashTiles t = tiles_for(c, (Prec)prec, nrhs);
    if (site_tile) *site_tile = t.site_tile;
    if (rhs_tile) *rhs_tile = t.rhs_tile;
    if (rhs_per_thread) *rhs_per_thread = t.rhs_per_thread;
    return WD_OK;
}

wd_status wd_set_rhs_per_thread(wd_ctx *c, wd_prec prec, int nrhs, int k) {
    if (!c) return WD_ERR_ARG;
    if ((int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS || k < 1 || k > 4)
        return fail(c, WD_ERR_ARG, "wd_set_rhs_per_thread: bad argument");
    DslashTiles t = tiles_for(c, (Prec)prec, nrhs);
    if (k > 1 && (prec != WD_F32 || t.rhs_tile % k != 0 || (t.site_tile * t.rhs_tile / k) % 32 != 0))
        return fail(c, WD_ERR_ARG, "wd_set_rhs_per_thread: FP32 only, k dividing rhs_tile, a multiple of 32 threads");
    if (k > 1 && c->split)
        return fail(c, WD_ERR_STATE, "wd_set_rhs_per_thread: a split sub-lattice runs one right-hand side per thread");
    t.rhs_per_thread = k;
    c->tiles[(int)prec * 64 + nrhs] = t;
    return WD_OK;
}

}  // extern "C"
