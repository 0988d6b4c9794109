// Entry points whose implementation is not in this build yet: they fail cleanly.
#include "wd_host.h"

using namespace wd;

namespace wd {
wd_status block_cg_solve(wd_ctx *c, double, const void *, void *, const wd_cg_params *, wd_cg_result *) {
    return fail(c, WD_ERR_ARG, "block CG is not available in this build");
}
}  // namespace wd

extern "C" {
wd_status wd_cg_solve_batched(wd_ctx *const *ctxs, const double *, const void *const *, void *const *, int,
                              const wd_cg_params *, wd_cg_result *) {
    return fail(ctxs ? ctxs[0] : nullptr, WD_ERR_ARG, "batched solver is not available in this build");
}
wd_status wd_autotune(wd_ctx *c, wd_prec, int, int *, int *) {
    return fail(c, WD_ERR_ARG, "autotuner is not available in this build");
}
wd_status wd_set_tiles(wd_ctx *c, wd_prec prec, int nrhs, int site_tile, int rhs_tile) {
    if (!c) return WD_ERR_ARG;
    if ((int)prec < 0 || (int)prec > 2 || nrhs < 1 || nrhs > WD_MAX_RHS || rhs_tile < 1 || rhs_tile > nrhs ||
        (site_tile != 16 && site_tile != 32 && site_tile != 64 && site_tile != 128 && site_tile != 256) ||
        site_tile * rhs_tile > 256 || (site_tile * rhs_tile) % 32 != 0)
        return fail(c, WD_ERR_ARG, "wd_set_tiles: unsupported tile shape");
    DslashTiles t;
    t.site_tile = site_tile;
    t.rhs_tile = rhs_tile;
    c->tiles[(int)prec * 64 + nrhs] = t;
    return WD_OK;
}
}
