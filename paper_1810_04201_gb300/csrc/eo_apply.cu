// The even-odd Schur operator as a standalone call (FP64), for users and tests.
//
// D = 1 - kappa H couples only sites of opposite parity (section 2.1, Eq. (1):
// nearest neighbours), so in even/odd blocks D = [[1, -kappa H_eo], [-kappa H_oe, 1]]
// and its Schur complement on the even sites is 1 - kappa^2 H_eo H_oe.
#include "dslash.cuh"
#include "blas.cuh"
#include "wd_host.h"

using namespace wd;

template <int RECON, bool DAG>
static cudaError_t schur(const DslashArgs &hop, const DslashArgs &back, DslashTiles t, cudaStream_t st) {
    dim3 block(t.site_tile, 1);
    dim3 grid(site_blocks<F64>(hop.g.V, t.site_tile), 1);
    dslash_kernel<F64, RECON, DAG, EpHop, true><<<grid, block, 0, st>>>(hop);
    dslash_kernel<F64, RECON, DAG, EpXpay, true><<<grid, block, 0, st>>>(back);
    return cudaGetLastError();
}

extern "C" wd_status wd_apply_schur(wd_ctx *c, double kappa, const void *in, void *out, int dagger) {
    wd::NvtxRange nvtx_("wd_apply_schur");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if (!in || !out || in == out) return fail(c, WD_ERR_ARG, "wd_apply_schur: bad field pointers");
    if (c->split) return fail(c, WD_ERR_STATE, "wd_apply_schur: not on a split sub-lattice");
    for (int mu = 0; mu < 4; ++mu)
        if (c->g.L[mu] % 2) return fail(c, WD_ERR_ARG, "wd_apply_schur: needs even extents");
    const void *gauge;
    size_t gdir;
    wd_status s = gauge_get_eo(c, F64, &gauge, &gdir);
    if (s != WD_OK) return s;
    const Geom ge = eo_geom(c, 0), go = eo_geom(c, 1);
    const size_t sh = spinor_bytes(F64, ge.Vs), sf = spinor_bytes(F64, c->g.Vs);
    void *ie, *io, *tmp, *oe;
    if ((s = ws_get(c, "schur_ie", sh, &ie)) != WD_OK) return s;
    if ((s = ws_get(c, "schur_io", sh, &io)) != WD_OK) return s;
    if ((s = ws_get(c, "schur_tmp", sh, &tmp)) != WD_OK) return s;
    if ((s = ws_get(c, "schur_oe", sh, &oe)) != WD_OK) return s;
    EoVecArgs e{};
    e.v.V = c->g.V;
    e.v.Vs = c->g.Vs;
    e.v.nrhs = 1;
    e.v.a = in; e.v.a_stride = sf; e.v.b = ie; e.v.c = io; e.v.b_stride = sh;
    e.Vhs = ge.Vs;
    e.g = c->g;
    const dim3 vgrid((c->g.V + 127) / 128, 1);
    k_split_eo<0><<<vgrid, 128, 0, c->stream>>>(e);
    DslashArgs h{};
    h.g = go;
    h.gauge = gauge;
    h.gauge_dir = gdir;
    h.nrhs = 1;
    h.in = ie; h.in_stride = sh;
    h.out = tmp; h.out_stride = sh;
    h.kappa = -1.0;
    DslashArgs b = h;
    b.g = ge;
    b.in = tmp;
    b.xsrc = ie; b.xsrc_stride = sh;
    b.out = oe;
    b.kappa = kappa * kappa;
    const DslashTiles t = tiles_for(c, F64, 1);
    const cudaError_t err = with_recon(link_recon(c, F64), [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        return dagger ? schur<R, true>(h, b, t, c->stream) : schur<R, false>(h, b, t, c->stream);
    });
    WD_CUDA(c, err);
    WD_CUDA(c, cudaMemsetAsync(io, 0, sh, c->stream));
    e.v.a = oe; e.v.a_stride = sh; e.v.c = io; e.v.b = out; e.v.b_stride = sf;
    k_join_eo<0><<<vgrid, 128, 0, c->stream>>>(e);
    WD_CUDA(c, cudaGetLastError());
    c->launches = 4;
    return WD_OK;
}
