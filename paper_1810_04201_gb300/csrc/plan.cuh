// Solver plans: kernel calls recorded once, then built into a CUDA graph with
// device-side conditional nodes or launched one by one from a host loop.
#pragma once
#include <cstring>
#include <vector>
#include "dslash.cuh"
#include "blas.cuh"

namespace wd {

// A solver is recorded once as lists of kernel calls (setup, loop body before the
// reliable-update branch, the branch, loop body after it, final check); the plan
// is then either turned into one CUDA graph with device-side conditionals, or
// launched from a host loop (WD_CG_LOOP=host: the same kernels, launched one by
// one, so that profilers that cannot see conditional graph nodes see them).
struct KCall {
    const void *func;
    dim3 grid, block;
    std::vector<unsigned char> arg;  // the kernel's single struct argument
};

struct Plan {
    std::vector<KCall> setup, pre, ifb, post, fin;
    bool has_if = false;
};

struct GraphBuilder {
    std::vector<KCall> *cur;
    explicit GraphBuilder(std::vector<KCall> *list) : cur(list) {}
    template <class Arg>
    void kernel(void (*f)(Arg), dim3 grid, dim3 block, const Arg &arg) {
        KCall k;
        k.func = (const void *)f;
        k.grid = grid;
        k.block = block;
        k.arg.resize(sizeof(Arg));
        std::memcpy(k.arg.data(), &arg, sizeof(Arg));
        cur->push_back(std::move(k));
    }
};

static inline cudaError_t add_chain(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, const std::vector<KCall> &calls) {
    for (const KCall &k : calls) {
        void *params[1] = {const_cast<unsigned char *>(k.arg.data())};
        cudaKernelNodeParams p{};
        p.func = const_cast<void *>(k.func);
        p.gridDim = k.grid;
        p.blockDim = k.block;
        p.sharedMemBytes = 0;
        p.kernelParams = params;
        cudaGraphNode_t n;
        cudaError_t e = cudaGraphAddKernelNode(&n, g, deps.data(), deps.size(), &p);
        if (e != cudaSuccess) return e;
        deps.assign(1, n);
    }
    return cudaSuccess;
}

static inline cudaError_t add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
                                   cudaGraphConditionalNodeType type, cudaGraph_t *body) {
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t n;
    cudaError_t e = cudaGraphAddNode(&n, g, deps.data(), nullptr, deps.size(), &np);
    if (e != cudaSuccess) return e;
    deps.assign(1, n);
    *body = np.conditional.phGraph_out[0];
    return cudaSuccess;
}

static inline cudaError_t launch_chain(const std::vector<KCall> &calls, cudaStream_t st) {
    for (const KCall &k : calls) {
        void *params[1] = {const_cast<unsigned char *>(k.arg.data())};
        cudaError_t e = cudaLaunchKernel(k.func, k.grid, k.block, params, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static inline int num_sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

// Grid for a reducing Dslash (one partial per block and row; the partial buffers hold
// kMaxPartialBlocks per row).  Up to that many site tiles get one block each and the
// hardware scheduler balances them across the SMs to the end of the launch; larger
// lattices get the blocks that are resident at once, each walking many tiles.
constexpr int kMaxPartialBlocks = 8192;
template <int P, class K>
static dim3 reduce_grid(K kernel, const Geom &g, DslashTiles t, int nrhs) {
    const dim3 rows(1, (nrhs + t.rhs_tile - 1) / t.rhs_tile);
    const int need = site_blocks<P>(g.V, t.site_tile);
    if (need <= kMaxPartialBlocks) return dim3(need, rows.y);
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, t.site_tile * t.rhs_tile, 0);
    if (per_sm < 1) per_sm = 1;
    const int cap = per_sm * num_sms();
    return dim3(cap < kMaxPartialBlocks ? cap : kMaxPartialBlocks, rows.y);
}

// Even-odd preconditioning: the solver works on the even half of the lattice
// with the Schur operator 1 - kappa^2 H_eo H_oe; these are its extra operands.
struct EoInfo {
    Geom ge, go;                          // checkerboard geometry, output parity 0 / 1
    const void *gauge[kNumPrec];          // checkerboard gauge per precision
    size_t gdir[kNumPrec];
    void *tmp64, *tmps;                   // odd-parity temporaries (FP64, inner precision)
    void *tmp32;                          // and FP32, for the corrections of an FP16 iteration
    void *bfull, *xfull, *tfull, *dbfull; // full-lattice fields for the split, join and final check
    void *be, *bo, *xo;                   // even / odd halves
};

struct Fields {
    void *b, *x, *db, *r, *p, *t;      // FP64
    void *rs, *ps, *ts, *xs;            // inner precision (xs FP32)
    void *t32;                          // FP16 iteration: FP32 field of the corrections (null: none)
    const void *g32;                    // and the FP32 links they use,
    int c32_inner;                      // compressed as the inner links (1) or the FP64 ones (0)
    Scalars *sc;
    double *partial;
    unsigned *counter;
    int *state;
    EoInfo eo;
};

template <int P, int RECON, bool DAG, class Ep, bool EO = false>
static void add_dslash(GraphBuilder &gb, const DslashArgs &a, DslashTiles t, bool reduce) {
    auto k = dslash_kernel<P, RECON, DAG, Ep, EO>;
    dim3 block(t.site_tile, t.rhs_tile);
    dim3 grid = reduce ? reduce_grid<P>(k, a.g, t, a.nrhs)
                       : dim3(site_blocks<P>(a.g.V, t.site_tile), (a.nrhs + t.rhs_tile - 1) / t.rhs_tile);
    gb.kernel(k, grid, block, a);
}

template <class K>
static void add_vec(GraphBuilder &gb, K k, const VecArgs &v) {
    gb.kernel(k, dim3((v.V + 127) / 128, v.nrhs), dim3(128), v);
}

struct SolverPlan {
    int recon;      // link compression of the FP64 copy
    int recon_in;   // and of the inner precision's copy
    double kappa;
    int nrhs;
    Prec inner;
    DslashTiles t64, tin;
    int ne;  // 0: CGNR on D^dag D x = D^dag b; 1: CGNE on D D^dag y = b, x = D^dag y
    int eo;  // 1: even-odd preconditioned (Schur complement on the even sites)
};

// One application of the solver's operator: D (or D^dag) on the full lattice, or,
// with even-odd preconditioning, the Schur operator 1 - kappa^2 H_eo H_oe (or its
// adjoint) as two checkerboard kernels: a bare hop into an odd temporary, then
// the hop back with the epilogue, which adds the even input.
template <int P, int RECON, bool DAG, class Ep, bool EO>
static void add_op(GraphBuilder &gb, const DslashArgs &a, DslashTiles t, bool reduce, const Fields &f) {
    if constexpr (!EO) {
        add_dslash<P, RECON, DAG, Ep>(gb, a, t, reduce);
    } else {
        const size_t sp = spinor_bytes((Prec)P, f.eo.ge.Vs);
        void *tmp = P == F64 ? f.eo.tmp64 : (P == F32 && f.eo.tmp32) ? f.eo.tmp32 : f.eo.tmps;
        DslashArgs h = a;
        h.g = f.eo.go;
        h.gauge = f.eo.gauge[P];
        h.gauge_dir = f.eo.gdir[P];
        h.out = tmp;
        h.out_stride = sp;
        h.kappa = -1.0;
        h.xsrc = nullptr;
        // a zero input (in_nonzero flag 0) needs no bare hop: the epilogue kernel skips it too
        if (a.in_nonzero) h.run_flag = a.in_nonzero, h.in_nonzero = nullptr;
        add_dslash<P, RECON, DAG, EpHop, true>(gb, h, t, false);
        DslashArgs e = a;
        e.g = f.eo.ge;
        e.gauge = f.eo.gauge[P];
        e.gauge_dir = f.eo.gdir[P];
        e.xsrc = a.in;
        e.xsrc_stride = a.in_stride;
        e.in = tmp;
        e.in_stride = sp;
        e.kappa = a.kappa * a.kappa;
        add_dslash<P, RECON, DAG, Ep, true>(gb, e, t, reduce);
    }
}

}  // namespace wd
