// The library context (opaque in the C ABI): host-side state of one lattice -- its
// geometry, stream, gauge copies, workspace, cached solver graphs and launch shapes.
// Kept apart from the device code of wd_internal.cuh.
#pragma once
#include <map>
#include <string>
#include <vector>
#include "wd_internal.cuh"

// The context (opaque in the C ABI).
struct wd_ctx {
    wd::Geom g;
    cudaStream_t stream = nullptr;
    int device = 0;
    int recon = 18;                                    // link compression set by wd_set_gauge
    int recon_p[wd::kNumPrec] = {};                    // per-precision overrides (0: recon)
    bool has_gauge = false;
    void *gauge[wd::kNumPrec] = {};                    // per precision (at this->recon)
    void *gauge_eo[wd::kNumPrec] = {};                 // checkerboard copies, per precision
    double *gauge_canon = nullptr;                     // FP64 canonical copy on device
    std::string last_error;
    long long launches = 0;
    // workspace
    std::map<std::string, void *> ws;                  // named device buffers
    std::map<std::string, size_t> ws_size;
    std::map<std::string, void *> graphs;              // cached cudaGraphExec_t per solver signature
    std::map<std::string, std::vector<long long>> graph_info;
    std::map<std::string, unsigned long long> graph_used;  // last use of each graph (graph_get / graph_put)
    unsigned long long graph_tick = 0;
    std::map<int, wd::DslashTiles> tiles;              // key: prec*64 + nrhs
    std::map<int, wd::DslashTiles> cg_tiles;           // the solvers' fused kernels (wd_autotune_cg); same key
    int staged_rows[wd::kNumPrec] = {};                // plain operators through the staged kernel (0: off)
    bool prefetch[wd::kNumPrec] = {};                  // plain FP32 operator through the cp.async-prefetch kernel
    unsigned *staged_err = nullptr;                    // the staged kernel's error word (zeroed when allocated)
    int staged_stages[wd::kNumPrec] = {};
    void *noalloc_scratch = nullptr;                   // device address of the allocation-free scratch array
    // one sub-lattice of a lattice split along t (wd_create_split): ranks own consecutive
    // blocks of global t-slices; g.split_t is set and g.antiperiodic is 0 (the global
    // boundary sign is applied to the faces received across it)
    bool split = false;
    int split_rank = 0, split_nranks = 1, split_antiperiodic = 0, split_t0 = 0;
    ~wd_ctx();
};

namespace wd {
// link compression of the copy of precision p
inline int link_recon(const wd_ctx *c, Prec p) { return c->recon_p[p] ? c->recon_p[p] : c->recon; }
}  // namespace wd

