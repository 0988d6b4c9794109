// wd_normal_apply_noalloc: the normal operator D^dag D with no device allocation.
//
// wd_normal_apply keeps its intermediate field D*in in context workspace that
// it allocates with cudaMalloc on first use.  This variant keeps that
// intermediate field in one file-scope device array instead, so the call never
// allocates or frees device memory.
//
// Scratch: g_noalloc_scratch, WD_NOALLOC_SCRATCH_BYTES (16 MiB) with 256-byte
// alignment.  Every GPU that loads the library holds this array until the
// process exits.  All calls on a device share it and it keeps the contents of
// the last call; the first pass overwrites every byte the second pass reads, so
// nothing needs clearing.  Calls whose kernels overlap on the GPU (two streams,
// or two host threads) race on the array.
#include <cmath>
#include "dslash.cuh"
#include "wd_host.h"

using namespace wd;

#define WD_NOALLOC_SCRATCH_BYTES (16u << 20)

static __device__ __align__(256) unsigned char g_noalloc_scratch[WD_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch for this context.  In host code the symbol
// names a host-side stand-in, so the address is looked up with the context's device
// current, on the first call of each context, and kept in the context beside its
// other device resources: it is valid in the CUDA context that was current then (the
// one the wd_ctx's own buffers belong to), and a wd_ctx never outlives that.
static wd_status scratch_address(wd_ctx *c, void **out) {
    if (!c->noalloc_scratch) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        c->noalloc_scratch = p;
    }
    *out = c->noalloc_scratch;
    return WD_OK;
}

extern "C" wd_status wd_normal_apply_noalloc(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec,
                                             int nrhs) {
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if (!in || !out || (int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, "wd_normal_apply_noalloc: bad argument");
    if (in == out) return fail(c, WD_ERR_ARG, "wd_normal_apply_noalloc: in and out must be distinct");
    if (!std::isfinite(kappa)) return fail(c, WD_ERR_ARG, "wd_normal_apply_noalloc: kappa not finite");
    if (c->split) return fail(c, WD_ERR_STATE, "wd_normal_apply_noalloc: not on a split sub-lattice");
    const size_t need = spinor_bytes((Prec)prec, c->g.Vs) * (size_t)nrhs;
    if (need > WD_NOALLOC_SCRATCH_BYTES) {
        char msg[200];
        snprintf(msg, sizeof msg,
                 "wd_normal_apply_noalloc: needs %zu bytes of scratch for this lattice, precision and nrhs; "
                 "the fixed scratch holds %u bytes",
                 need, (unsigned)WD_NOALLOC_SCRATCH_BYTES);
        return fail(c, WD_ERR_ARG, msg);
    }
    if (!c->has_gauge) return fail(c, WD_ERR_STATE, "wd_normal_apply_noalloc: no gauge field set");
    if (!c->gauge[prec])
        return fail(c, WD_ERR_STATE,
                    "wd_normal_apply_noalloc: the gauge copy in this precision does not exist (yet, or any more "
                    "after wd_set_link_compression); one wd_apply in this precision creates it (and allocates)");
    int dev = -1;
    WD_CUDA(c, cudaGetDevice(&dev));
    if (dev != c->device)
        return fail(c, WD_ERR_ARG, "wd_normal_apply_noalloc: the context's device must be the current device");
    void *tmp = nullptr;
    wd_status s = scratch_address(c, &tmp);
    if (s != WD_OK) return s;

    DslashArgs a{};
    a.g = c->g;
    a.in_stride = a.out_stride = spinor_bytes((Prec)prec, c->g.Vs);
    a.gauge = c->gauge[prec];
    a.gauge_dir = gauge_dir_bytes(c, (Prec)prec);
    a.kappa = kappa;
    a.nrhs = nrhs;
    const DslashTiles t = tiles_for(c, (Prec)prec, nrhs);
    a.in = in;
    a.out = tmp;
    WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), false, t, c->stream));
    a.in = tmp;
    a.out = out;
    WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), true, t, c->stream));
    c->launches = 2;
    return WD_OK;
}
