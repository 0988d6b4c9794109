// Autotuner for the Dslash launch shape (the paper's compile-time knobs of §7.1 --
// partition and unroll factors, number of kernel instances -- become a timed
// sweep over the thread-block shape at run time).
//
// Candidates: site_tile in {16, 32, 64, 128, 256} threads along the sites and
// rhs_tile in {1, 2, 3, 4, 6, 8, 12, 16} right-hand sides per block, with
// site_tile * rhs_tile <= 256, a multiple of 32, and rhs_tile <= nrhs (FP64 and
// DF32, two lanes per site: site_tile >= 32, i.e. site_tile / 2 sites per block).  Each
// candidate runs the plain D kernel 2 + 5 times on context scratch fields; the
// fastest mean of the last 5 (CUDA events on the context stream) is kept for
// (precision, nrhs) and used by every later operator and solver call.
#include <vector>
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
    void *in, *out;
    if ((s = ws_get(c, "tune_in", fb * nrhs, &in)) != WD_OK) return s;
    if ((s = ws_get(c, "tune_out", fb * nrhs, &out)) != WD_OK) return s;
    WD_CUDA(c, cudaMemsetAsync(in, 0, fb * nrhs, c->stream));

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
    EventPair ev;
    WD_CUDA(c, ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    float best = 1e30f;
    DslashTiles bt = tiles_for(c, (Prec)prec, nrhs);
    for (int st : sts)
        for (int rt : rts) {
            if (rt > nrhs || st * rt > 256 || (st * rt) % 32 != 0) continue;
            if (threads_per_site((Prec)prec) > 1 && st % 32 != 0) continue;
            DslashTiles t;
            t.site_tile = st;
            t.rhs_tile = rt;
            for (int k = 0; k < 2; ++k) WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), false, t, c->stream));
            WD_CUDA(c, cudaEventRecord(e0, c->stream));
            for (int k = 0; k < 5; ++k) WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), false, t, c->stream));
            WD_CUDA(c, cudaEventRecord(e1, c->stream));
            WD_CUDA(c, cudaEventSynchronize(e1));
            float ms = 0.f;
            WD_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
            c->launches += 7;
            if (ms < best) {
                best = ms;
                bt = t;
            }
        }
    c->tiles[(int)prec * 64 + nrhs] = bt;
    if (site_tile) *site_tile = bt.site_tile;
    if (rhs_tile) *rhs_tile = bt.rhs_tile;
    return WD_OK;
}

}  // extern "C"
