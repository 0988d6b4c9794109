// Host-side internal interface shared by the translation units of libwd.
#pragma once
#include <cstdio>
#include <string>
#include <type_traits>
#include <nvtx3/nvToolsExt.h>
#include "wd_internal.cuh"
#include "wd_ctx.h"

namespace wd {

struct DslashArgs;
struct VecArgs;

// Default reliable-update threshold per inner precision: an FP64 update runs when
// the iterated residual has dropped by this factor since the last one.  Low
// precisions need frequent updates; FP64 updates are expensive on a part with a
// thin FP64 pipe, so the threshold is as small as each precision allows.  The
// partial solution of a segment is summed in FP32 for every inner precision, which
// bounds DF32 too (1e-9 no longer converges).  FP32: 3e-6 takes a 1e-10 solve in
// two updates (1e-4 took three) at the same iteration count on the 32^3 x 64 and
// 24^3 x 48 workloads.  FP16: 3e-3 saves two of six updates on the better
// conditioned even-odd system, but costs 10 % more iterations on the full one.
// FP32 corrections of an FP16 inner iteration run when its residual has dropped by
// this factor since the last correction or reliable update (FP16 storage resolves about
// three decimal digits; the FP64 updates then follow the FP32 threshold).
constexpr double kCorrectDelta = 1e-2;

inline double default_delta(Prec p, bool eo) {
    switch (p) {
    case F16: return eo ? 3e-3 : 1e-2;
    case F32: return 3e-6;
    case DF32: return 1e-6;
    default: return 0.1;
    }
}

// status helpers
wd_status fail(wd_ctx *c, wd_status s, const std::string &msg);
wd_status cuda_fail(wd_ctx *c, cudaError_t e, const char *where);
#define WD_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return ::wd::cuda_fail(ctx, e_, #call); \
    } while (0)

// An NVTX range over one library call (seen by profilers that record NVTX, e.g.
// ncu --nvtx --nvtx-include "wd_cg_solve/"); free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// A pair of CUDA events released on every return path.
struct EventPair {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t create() {
        cudaError_t e = cudaEventCreate(&e0);
        return e == cudaSuccess ? cudaEventCreate(&e1) : e;
    }
    float ms() const {
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        return t;
    }
    ~EventPair() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    }
};

// Calls f(std::integral_constant<int, R>{}) for the link compression R in {18, 12, 8}.
template <class F> decltype(auto) with_recon(int recon, F &&f) {
    if (recon == 12) return f(std::integral_constant<int, 12>{});
    if (recon == 8) return f(std::integral_constant<int, 8>{});
    return f(std::integral_constant<int, 18>{});
}

// WD_ERR_ARG unless every link suits the 8-real parametrisation (see wd_set_gauge)
wd_status check_recon8(wd_ctx *c, const char *who);

// Calls f(integral_constant<R64>, integral_constant<RIN>) for the pairs of link
// compressions (FP64, inner precision) the solvers are built for: equal ones, and
// whole FP64 links beside recon-12 or recon-8 inner links.
template <class F> decltype(auto) with_recon_pair(int r64, int rin, F &&f) {
    using std::integral_constant;
    if (r64 == 18 && rin == 12) return f(integral_constant<int, 18>{}, integral_constant<int, 12>{});
    if (r64 == 18 && rin == 8) return f(integral_constant<int, 18>{}, integral_constant<int, 8>{});
    return with_recon(r64, [&](auto rc) { return f(rc, rc); });
}

// workspace: named device buffer of at least `bytes` (kept across calls)
wd_status ws_get(wd_ctx *c, const std::string &name, size_t bytes, void **out);
// device gauge field of precision p at the context's recon (created on first use)
wd_status gauge_get(wd_ctx *c, Prec p, const void **out);
size_t gauge_dir_bytes(const wd_ctx *c, Prec p);
// checkerboard gauge copy (parity-major, see dslash.cuh) of precision p, and its
// direction stride in bytes
wd_status gauge_get_eo(wd_ctx *c, Prec p, const void **out, size_t *dir_bytes);
// geometry of one parity of the lattice (all extents even)
Geom eo_geom(const wd_ctx *c, int parity);

DslashTiles tiles_for(wd_ctx *c, Prec p, int nrhs);
// launch shape of the solvers' fused Dslash kernels, for plain or even-odd solves:
// wd_autotune_cg's choice, else tiles_for
constexpr int kEoTileKey = 1024;
DslashTiles cg_tiles_for(wd_ctx *c, Prec p, int nrhs, bool eo);
// frees a workspace buffer (no-op when absent)
void ws_release(wd_ctx *c, const std::string &name);

// The context's cache of executable CUDA graphs (solver plans keyed by their signature:
// precision, tiles, kappa, ...).  It holds at most kMaxGraphs; graph_put evicts the least
// recently used one (a graph still executing is freed by CUDA when it completes), so a
// caller that scans kappa or many masses does not grow it without bound.
constexpr size_t kMaxGraphs = 16;
void *graph_get(wd_ctx *c, const std::string &key);  // nullptr when absent; marks it used
void graph_put(wd_ctx *c, const std::string &key, void *exec, const std::vector<long long> &info);
void graph_clear(wd_ctx *c);

// Launchers of the plain operators (xpay epilogue): out = in - kappa * hop
// (dagger = 0: D, dagger = 1: D^dag).  Used by wd_apply and the autotuner.
cudaError_t launch_apply(const DslashArgs &a, Prec p, int recon, bool dagger, DslashTiles t, cudaStream_t st);
// The same operator with the neighbour spinors staged through shared memory (FP32, FP16;
// tiles of `rows` x-rows, `stages` tiles in flight per block); err: set to 1 when a wait runs out.
cudaError_t launch_apply_staged(const DslashArgs &a, Prec p, int recon, bool dagger, int rows, int stages,
                                unsigned *err, cudaStream_t st);
bool staged_ok(Prec p, const Geom &g, int rows, int stages);
// allocates (and zeroes) the staged kernel's error word of the context on first use
wd_status staged_error_word(wd_ctx *c);
// The plain FP32 operator with each thread prefetching its next hops' neighbour spinors into
// shared memory by cp.async (tiles as for launch_apply, one right-hand side per thread).
cudaError_t launch_apply_prefetch(const DslashArgs &a, int recon, bool dagger, DslashTiles t, cudaStream_t st);

// Kernel-node description for graph building and direct launches.
struct KernelCall {
    const void *func;
    dim3 grid, block;
    size_t smem;
    void *args[1];  // every kernel of the library takes one struct argument
};

}  // namespace wd
