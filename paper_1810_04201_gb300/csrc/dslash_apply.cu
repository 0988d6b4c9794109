// Plain Dslash launches: out = D in or out = D^dag in, every precision and link
// compression (18, 12 or 8 reals) (section 2.1, Eq. (1); section 2.2, gamma5-hermiticity).
#include "dslash.cuh"
#include "wd_host.h"

namespace wd {

template <int P, int RECON, bool DAG>
static cudaError_t go(const DslashArgs &a, DslashTiles t, cudaStream_t st) {
    if constexpr (P == F32) {
        const int k = t.rhs_per_thread;
        // the K-per-thread kernel has no sub-lattice (split_t) form
        if (k > 1 && t.rhs_tile % k == 0 && !a.g.split_t) {
            dim3 block(t.site_tile, t.rhs_tile / k);
            dim3 grid(site_blocks<P>(a.g.V, t.site_tile), (a.nrhs + t.rhs_tile - 1) / t.rhs_tile);
            if (k == 2) dslash_multi_kernel<RECON, DAG, 2><<<grid, block, 0, st>>>(a);
            else if (k == 3) dslash_multi_kernel<RECON, DAG, 3><<<grid, block, 0, st>>>(a);
            else dslash_multi_kernel<RECON, DAG, 4><<<grid, block, 0, st>>>(a);
            return cudaGetLastError();
        }
    }
    dim3 block(t.site_tile, t.rhs_tile);
    dim3 grid(site_blocks<P>(a.g.V, t.site_tile), (a.nrhs + t.rhs_tile - 1) / t.rhs_tile);
    dslash_kernel<P, RECON, DAG, EpXpay><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

template <int P>
static cudaError_t go_p(const DslashArgs &a, int recon, bool dagger, DslashTiles t, cudaStream_t st) {
    return with_recon(recon, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        return dagger ? go<P, R, true>(a, t, st) : go<P, R, false>(a, t, st);
    });
}

cudaError_t launch_apply(const DslashArgs &a, Prec p, int recon, bool dagger, DslashTiles t, cudaStream_t st) {
    switch (p) {
    case F64: return go_p<F64>(a, recon, dagger, t, st);
    case F32: return go_p<F32>(a, recon, dagger, t, st);
    case DF32: return go_p<DF32>(a, recon, dagger, t, st);
    default: return go_p<F16>(a, recon, dagger, t, st);
    }
}

}  // namespace wd
