// Device-resident CG solver plans for recon-8 links (see cg_impl.cuh).
#include "cg_impl.cuh"

namespace wd {
template cudaError_t build_for<8, 8>(wd_ctx *, const SolverPlan &, const Fields &, const void *, const void *,
                                         cudaGraphExec_t *, std::vector<long long> &);
template void record_for<8, 8>(wd_ctx *, const SolverPlan &, const Fields &, const void *, const void *, Plan &);
}  // namespace wd
