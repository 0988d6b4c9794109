// Entry points whose implementation is not in this build yet: they fail cleanly.
#include "wd_host.h"

using namespace wd;

extern "C" {
wd_status wd_cg_solve_batched(wd_ctx *const *ctxs, const double *, const void *const *, void *const *, int,
                              const wd_cg_params *, wd_cg_result *) {
    return fail(ctxs ? ctxs[0] : nullptr, WD_ERR_ARG, "batched solver is not available in this build");
}
}
