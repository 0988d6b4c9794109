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

static cudaError_t add_chain(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, const std::vector<KCall> &calls) {
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

static cudaError_t add_conditional(cudaGraph_t g, std::vector<cudaGraphNode_t> &deps, cudaGraphConditionalHandle h,
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

static cudaError_t launch_chain(const std::vector<KCall> &calls, cudaStream_t st) {
    for (const KCall &k : calls) {
        void *params[1] = {const_cast<unsigned char *>(k.arg.data())};
        cudaError_t e = cudaLaunchKernel(k.func, k.grid, k.block, params, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

static int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

// Grid for a reducing Dslash: at most the blocks that fit on the machine at once.
template <class K>
static dim3 reduce_grid(K kernel, const Geom &g, DslashTiles t, int nrhs) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, t.site_tile * t.rhs_tile, 0);
    if (per_sm < 1) per_sm = 1;
    const int need = (g.V + t.site_tile - 1) / t.site_tile;
    int cap = per_sm * num_sms();
    return dim3(need < cap ? need : cap, (nrhs + t.rhs_tile - 1) / t.rhs_tile);
}

struct Fields {
    void *b, *x, *db, *r, *p, *t;      // FP64
    void *rs, *ps, *ts, *xs;            // inner precision (xs FP32)
    Scalars *sc;
    double *partial;
    unsigned *counter;
    int *state;
};

template <int P, int RECON, bool DAG, class Ep>
static void add_dslash(GraphBuilder &gb, const DslashArgs &a, DslashTiles t, bool reduce) {
    auto k = dslash_kernel<P, RECON, DAG, Ep>;
    dim3 block(t.site_tile, t.rhs_tile);
    dim3 grid = reduce ? reduce_grid(k, a.g, t, a.nrhs)
                       : dim3((a.g.V + t.site_tile - 1) / t.site_tile, (a.nrhs + t.rhs_tile - 1) / t.rhs_tile);
    gb.kernel(k, grid, block, a);
}

template <class K>
static void add_vec(GraphBuilder &gb, K k, const VecArgs &v) {
    gb.kernel(k, dim3((v.V + 127) / 128, v.nrhs), dim3(128), v);
}

struct SolverPlan {
    int recon;
    double kappa;
    int nrhs;
    Prec inner;
    DslashTiles t64, tin;
    int ne;  // 0: CGNR on D^dag D x = D^dag b; 1: CGNE on D D^dag y = b, x = D^dag y
};

}  // namespace wd
