// Device-resident CG on the normal equations (section 2.2), FP64 and mixed
// precision with FP64 reliable updates, for one or many right-hand sides.
//
// The whole solve is one CUDA graph: setup kernels, a conditional WHILE node
// whose body is one CG step (three kernels; the mixed-precision body adds a
// conditional IF node holding the reliable update), and the final FP64
// true-residual check.  The loop condition is set on the device, so the host
// waits only once, for the result.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "plan.cuh"
#include "wd_host.h"

using namespace wd;

namespace wd {

// Solver plans per pair of link compressions (FP64, inner precision), instantiated in
// cg_recon18.cu, cg_recon12.cu, cg_recon8.cu, cg_recon18_12.cu and cg_recon18_8.cu.
template <int RECON, int RIN>
cudaError_t build_for(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                      cudaGraphExec_t *exec, std::vector<long long> &counts);
template <int RECON, int RIN>
void record_for(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin, Plan &plan);


// The same plan launched kernel by kernel from the host; the active flags are read
// back every `chunk` iterations.  Loop kernels of converged rows return at once,
// so iterations launched after convergence change nothing.
static cudaError_t run_host_loop(wd_ctx *c, const Plan &plan, const Fields &f, int nrhs, int max_iter,
                                 long long *launched) {
    const int chunk = 4;
    std::vector<Scalars> h(nrhs);
    cudaError_t e = launch_chain(plan.setup, c->stream);
    long long n = (long long)plan.setup.size();
    int it = 0;
    while (e == cudaSuccess && it <= max_iter + 1) {
        for (int k = 0; k < chunk && e == cudaSuccess; ++k, ++it) {
            e = launch_chain(plan.pre, c->stream);
            if (e == cudaSuccess) e = launch_chain(plan.ifb, c->stream);
            if (e == cudaSuccess) e = launch_chain(plan.post, c->stream);
            n += (long long)(plan.pre.size() + plan.ifb.size() + plan.post.size());
        }
        if (e != cudaSuccess) break;
        e = cudaMemcpyAsync(h.data(), f.sc, sizeof(Scalars) * nrhs, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        bool any = false;
        for (int r = 0; r < nrhs; ++r) any |= h[r].active != 0;
        if (!any) break;
    }
    if (e == cudaSuccess) e = launch_chain(plan.fin, c->stream);
    *launched = n + (long long)plan.fin.size();
    return e;
}

wd_status block_cg_solve(wd_ctx *c, double kappa, const void *b, void *x, const wd_cg_params *prm,
                         wd_cg_result *res);

}  // namespace wd

extern "C" {

wd_status wd_cg_solve(wd_ctx *c, double kappa, const void *b, void *x, const wd_cg_params *prm, wd_cg_result *res) {
    wd::NvtxRange nvtx_("wd_cg_solve");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if (!b || !x || !prm || !res) return fail(c, WD_ERR_ARG, "wd_cg_solve: null argument");
    if (c->split) return fail(c, WD_ERR_STATE, "wd_cg_solve: a split sub-lattice (use wd_cg_solve_split)");
    const int nrhs = prm->nrhs < 1 ? 1 : prm->nrhs;
    if (nrhs > WD_MAX_RHS) return fail(c, WD_ERR_ARG, "wd_cg_solve: nrhs above WD_MAX_RHS");
    if (prm->inner_prec < 0 || prm->inner_prec >= kNumPrec) return fail(c, WD_ERR_ARG, "wd_cg_solve: bad inner_prec");
    if (!(prm->tol > 0) || !std::isfinite(kappa)) return fail(c, WD_ERR_ARG, "wd_cg_solve: bad tol or kappa");
    if (b == x) return fail(c, WD_ERR_ARG, "wd_cg_solve: b and x must be distinct");
    if (prm->normal_eq != 0 && prm->normal_eq != 1) return fail(c, WD_ERR_ARG, "wd_cg_solve: normal_eq must be 0 or 1");
    if (prm->precondition != WD_PRECOND_NONE && prm->precondition != WD_PRECOND_EO)
        return fail(c, WD_ERR_ARG, "wd_cg_solve: unknown preconditioner");
    if (prm->stop_rule != WD_STOP_NORMAL && prm->stop_rule != WD_STOP_SYSTEM)
        return fail(c, WD_ERR_ARG, "wd_cg_solve: unknown stop_rule");
    const bool eo = prm->precondition == WD_PRECOND_EO;
    // CGNE iterates b - D x itself; CGNR resumes until the recomputed |b - D x| meets tol
    const bool stop_sys = prm->stop_rule == WD_STOP_SYSTEM && !prm->normal_eq;
    if (eo) {
        if (prm->block || prm->normal_eq)
            return fail(c, WD_ERR_ARG, "wd_cg_solve: even-odd preconditioning is built for plain CGNR");
        for (int mu = 0; mu < 4; ++mu)
            if (c->g.L[mu] % 2) return fail(c, WD_ERR_ARG, "wd_cg_solve: even-odd preconditioning needs even extents");
    }
    if (prm->block) {
        if (prm->inner_prec != WD_F64) return fail(c, WD_ERR_ARG, "wd_cg_solve: block CG runs in FP64 only");
        if (prm->normal_eq) return fail(c, WD_ERR_ARG, "wd_cg_solve: block CG solves D^dag D only");
        if (prm->stop_rule != WD_STOP_NORMAL)
            return fail(c, WD_ERR_ARG, "wd_cg_solve: block CG stops on the normal residual only");
        return block_cg_solve(c, kappa, b, x, prm, res);
    }
    const Prec inner = (Prec)prm->inner_prec;
    const void *g64, *gin;
    wd_status s = gauge_get(c, F64, &g64);
    if (s != WD_OK) return s;
    s = gauge_get(c, inner, &gin);
    if (s != WD_OK) return s;

    // iterated fields live on the full lattice, or on the even half with even-odd
    const Geom gw = eo ? eo_geom(c, 0) : c->g;
    const std::string pre = eo ? "eo_" : "cg_";
    const size_t sfull = spinor_bytes(F64, c->g.Vs) * nrhs;
    const size_t s64 = spinor_bytes(F64, gw.Vs) * nrhs;
    Fields f{};
    const char *n64[6] = {"b", "x", "db", "r", "p", "t"};
    void **p64[6] = {&f.b, &f.x, &f.db, &f.r, &f.p, &f.t};
    for (int i = 0; i < 6; ++i)
        if ((s = ws_get(c, pre + n64[i], s64, p64[i])) != WD_OK) return s;
    if (inner != F64) {
        const size_t sin = spinor_bytes(inner, gw.Vs) * nrhs;
        std::string sfx = inner == F32 ? "32" : inner == F16 ? "16" : "d32";
        if ((s = ws_get(c, pre + "rs" + sfx, sin, &f.rs)) != WD_OK) return s;
        if ((s = ws_get(c, pre + "ps" + sfx, sin, &f.ps)) != WD_OK) return s;
        if ((s = ws_get(c, pre + "ts" + sfx, sin, &f.ts)) != WD_OK) return s;
        if ((s = ws_get(c, pre + "xs", spinor_bytes(F32, gw.Vs) * nrhs, &f.xs)) != WD_OK) return s;
    }
    // An FP16 iteration is corrected in FP32 between its FP64 reliable updates, with the
    // FP32 copy of the links, compressed as the FP64 copy or as the FP16 one (with a third
    // compression on the FP32 copy, no corrections: the FP64 updates alone, at the FP16
    // threshold)
    const int rc32 = link_recon(c, F32);
    const bool corr = inner == F16 && (rc32 == link_recon(c, F64) || rc32 == link_recon(c, F16));
    f.c32_inner = corr && rc32 != link_recon(c, F64);
    if (corr) {
        if ((s = gauge_get(c, F32, &f.g32)) != WD_OK) return s;
        if ((s = ws_get(c, pre + "t32c", spinor_bytes(F32, gw.Vs) * nrhs, &f.t32)) != WD_OK) return s;
    }
    if (eo) {
        f.eo.ge = eo_geom(c, 0);
        f.eo.go = eo_geom(c, 1);
        if ((s = gauge_get_eo(c, F64, &f.eo.gauge[F64], &f.eo.gdir[F64])) != WD_OK) return s;
        if ((s = gauge_get_eo(c, inner, &f.eo.gauge[inner], &f.eo.gdir[inner])) != WD_OK) return s;
        if ((s = ws_get(c, "eo_tmp64", s64, &f.eo.tmp64)) != WD_OK) return s;
        if (inner != F64 &&
            (s = ws_get(c, std::string("eo_tmps") + std::to_string((int)inner), spinor_bytes(inner, gw.Vs) * nrhs,
                        &f.eo.tmps)) != WD_OK)
            return s;
        if (corr) {
            if ((s = gauge_get_eo(c, F32, &f.eo.gauge[F32], &f.eo.gdir[F32])) != WD_OK) return s;
            if ((s = ws_get(c, std::string("eo_tmps") + std::to_string((int)F32), spinor_bytes(F32, gw.Vs) * nrhs,
                            &f.eo.tmp32)) != WD_OK)
                return s;
        }
        const char *nh[3] = {"eo_be", "eo_bo", "eo_xo"};
        void **ph[3] = {&f.eo.be, &f.eo.bo, &f.eo.xo};
        for (int i = 0; i < 3; ++i)
            if ((s = ws_get(c, nh[i], s64, ph[i])) != WD_OK) return s;
        const char *nf[4] = {"eo_bfull", "eo_xfull", "eo_tfull", "eo_dbfull"};
        void **pf[4] = {&f.eo.bfull, &f.eo.xfull, &f.eo.tfull, &f.eo.dbfull};
        for (int i = 0; i < 4; ++i)
            if ((s = ws_get(c, nf[i], sfull, pf[i])) != WD_OK) return s;
    }
    void *tmp;
    if ((s = ws_get(c, "cg_scalars", sizeof(Scalars) * WD_MAX_RHS, &tmp)) != WD_OK) return s;
    f.sc = (Scalars *)tmp;
    const size_t npart = (size_t)WD_MAX_RHS * 3 * kMaxPartialBlocks;
    if ((s = ws_get(c, "partial", npart * sizeof(double), &tmp)) != WD_OK) return s;
    f.partial = (double *)tmp;
    if ((s = ws_get(c, "counter", 256, &tmp)) != WD_OK) return s;
    f.counter = (unsigned *)tmp;
    f.state = (int *)((char *)tmp + 64);

    const int r64 = link_recon(c, F64), rin = inner == F64 ? r64 : link_recon(c, inner);
    if (rin != r64 && r64 != 18)
        return fail(c, WD_ERR_ARG, "wd_cg_solve: with compressed FP64 links the inner precision needs the same "
                                   "compression (see wd_set_link_compression)");
    SolverPlan pl{r64, rin, kappa, nrhs, inner, cg_tiles_for(c, F64, nrhs, eo), cg_tiles_for(c, inner, nrhs, eo),
                  prm->normal_eq ? 1 : 0, eo ? 1 : 0};
    if (prm->rhs_tile > 0) {
        // a fixed right-hand-side tile for the fused kernels, with the tuned site tile
        // shrunk where site_tile x rhs_tile would pass 256 threads
        const int rt = prm->rhs_tile < nrhs ? prm->rhs_tile : nrhs;
        for (DslashTiles *t : {&pl.t64, &pl.tin}) {
            t->rhs_tile = rt;
            t->rhs_per_thread = 1;
            while (t->site_tile > 32 && t->site_tile * rt > 256) t->site_tile /= 2;
            if (t->site_tile * rt > 256 || (t->site_tile * rt) % 32 != 0)
                return fail(c, WD_ERR_ARG, "wd_cg_solve: rhs_tile gives no launch shape of at most 256 threads, a "
                                           "multiple of 32");
        }
    }
    char key[256];
    snprintf(key, sizeof key, "cg|%d|%d|%d,%d|%a|%d,%d|%d,%d|%d|%d|%d", (int)inner, nrhs, r64, rin, kappa,
             pl.t64.site_tile, pl.t64.rhs_tile, pl.tin.site_tile, pl.tin.rhs_tile, pl.ne, pl.eo,
             corr ? 1 + f.c32_inner : 0);
    const char *loop_env = getenv("WD_CG_LOOP");
    const bool host_loop = loop_env && std::strcmp(loop_env, "host") == 0;
    cudaGraphExec_t exec = nullptr;
    Plan hplan;
    if (host_loop) {
        with_recon_pair(r64, rin, [&](auto ra, auto rb) {
            record_for<decltype(ra)::value, decltype(rb)::value>(c, pl, f, g64, gin, hplan);
        });
        WD_CUDA(c, cudaMemsetAsync(f.counter, 0, 64, c->stream));
    } else {
        exec = (cudaGraphExec_t)graph_get(c, key);
        if (!exec) {
            std::vector<long long> counts;
            cudaError_t e = with_recon_pair(r64, rin, [&](auto ra, auto rb) {
                return build_for<decltype(ra)::value, decltype(rb)::value>(c, pl, f, g64, gin, &exec, counts);
            });
            if (e != cudaSuccess) return cuda_fail(c, e, "building the CG graph");
            graph_put(c, key, exec, counts);
            WD_CUDA(c, cudaMemsetAsync(f.counter, 0, 256, c->stream));
        }
    }

    // per-RHS state.  With even-odd preconditioning tol applies to the reduced system,
    // so the solve runs with half of it and is resumed from its own solution, with a
    // tighter reduced tolerance, until the recomputed full-lattice residual meets tol.
    // With the system-residual rule the same resumption runs until |b - D x| meets tol.
    std::vector<Scalars> h(nrhs);
    const double delta = prm->delta > 0 ? prm->delta : corr ? default_delta(F32, eo) : default_delta(inner, eo);
    void *bin = eo ? f.eo.bfull : f.b, *xin = eo ? f.eo.xfull : f.x;
    WD_CUDA(c, cudaMemcpyAsync(bin, b, sfull, cudaMemcpyDeviceToDevice, c->stream));
    if (pl.ne) WD_CUDA(c, cudaMemsetAsync(xin, 0, sfull, c->stream));  // CGNE starts from y = 0
    else WD_CUDA(c, cudaMemcpyAsync(xin, x, sfull, cudaMemcpyDeviceToDevice, c->stream));
    double tol_run = eo ? 0.5 * prm->tol : prm->tol;
    std::vector<int> iters(nrhs, 0), reliable(nrhs, 0), corrections(nrhs, 0);
    float ms_total = 0.f;
    long long launches = 0;
    const int attempts = (eo || stop_sys) ? 4 : 1;
    for (int attempt = 0; attempt < attempts; ++attempt) {
        for (int r = 0; r < nrhs; ++r) {
            std::memset(&h[r], 0, sizeof(Scalars));
            h[r].tol2 = tol_run * tol_run;
            h[r].max_iter = prm->max_iter - iters[r] > 0 ? prm->max_iter - iters[r] : 0;
            h[r].delta2 = delta * delta;
            h[r].delta2_lo = corr ? kCorrectDelta * kCorrectDelta : 0.0;
            h[r].active = 1;
            h[r].status = WD_ERR_NOT_CONVERGED;
        }
        WD_CUDA(c, cudaMemcpyAsync(f.sc, h.data(), sizeof(Scalars) * nrhs, cudaMemcpyHostToDevice, c->stream));
        // state: [0] loop bodies, [1] reliable updates run, [2] nonzero x0, [3] rows stopped
        // at a reliable update, [4] final check needed (bytes 0x01: nonzero)
        WD_CUDA(c, cudaMemsetAsync(f.state, 0, 4 * sizeof(int), c->stream));
        WD_CUDA(c, cudaMemsetAsync(f.state + 4, 1, sizeof(int), c->stream));
        EventPair ev;
        WD_CUDA(c, ev.create());
        cudaEvent_t e0 = ev.e0, e1 = ev.e1;
        WD_CUDA(c, cudaEventRecord(e0, c->stream));
        long long host_launched = 0;
        if (host_loop) WD_CUDA(c, run_host_loop(c, hplan, f, nrhs, h[0].max_iter, &host_launched));
        else WD_CUDA(c, cudaGraphLaunch(exec, c->stream));
        WD_CUDA(c, cudaEventRecord(e1, c->stream));
        WD_CUDA(c, cudaMemcpyAsync(h.data(), f.sc, sizeof(Scalars) * nrhs, cudaMemcpyDeviceToHost, c->stream));
        int st[2];
        WD_CUDA(c, cudaMemcpyAsync(st, f.state, sizeof st, cudaMemcpyDeviceToHost, c->stream));
        WD_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms_total += ms;
        if (host_loop) {
            launches += host_launched;
        } else {
            const std::vector<long long> &cnt = c->graph_info[key];
            launches += cnt[0] + (long long)st[0] * cnt[1] + (long long)st[1] * cnt[2] + cnt[3];
        }
        double worst_resid = 0.0;
        bool all_ok = true;
        for (int r = 0; r < nrhs; ++r) {
            iters[r] += h[r].iter;
            reliable[r] += h[r].reliable;
            corrections[r] += h[r].corrections;
            all_ok &= h[r].status == WD_OK;
            const double tr = stop_sys ? (h[r].b2 > 0 ? std::sqrt(h[r].true_b2 / h[r].b2) : std::sqrt(h[r].true_b2))
                                       : (h[r].rhs2 > 0 ? std::sqrt(h[r].true_n2 / h[r].rhs2) : std::sqrt(h[r].true_n2));
            worst_resid = tr > worst_resid ? tr : worst_resid;
        }
        if (attempts == 1 || !all_ok || worst_resid <= prm->tol || !(worst_resid > 0)) break;
        tol_run *= (eo ? 0.5 : 0.7) * prm->tol / worst_resid;
        if (attempt == attempts - 1)
            for (int r = 0; r < nrhs; ++r) h[r].status = WD_ERR_NOT_CONVERGED;
    }
    WD_CUDA(c, cudaMemcpyAsync(x, xin, sfull, cudaMemcpyDeviceToDevice, c->stream));
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->launches = launches;

    wd_status worst = WD_OK;
    for (int r = 0; r < nrhs; ++r) {
        res[r].iters = iters[r];
        res[r].reliable_updates = reliable[r];
        res[r].inner_corrections = corrections[r];
        res[r].true_rel_resid = h[r].rhs2 > 0 ? std::sqrt(h[r].true_n2 / h[r].rhs2) : std::sqrt(h[r].true_n2);
        res[r].true_rel_resid_b = h[r].b2 > 0 ? std::sqrt(h[r].true_b2 / h[r].b2) : std::sqrt(h[r].true_b2);
        res[r].seconds = ms_total * 1e-3;
        res[r].status = h[r].status;
        if (h[r].status != WD_OK && worst == WD_OK) worst = (wd_status)h[r].status;
    }
    if (worst != WD_OK) c->last_error = std::string("wd_cg_solve: ") + wd_status_string(worst);
    return worst;
}

wd_status wd_cg_solve_canonical(wd_ctx *c, double kappa, const double *b_canon, double *x_canon, int on_device,
                                const wd_cg_params *prm, wd_cg_result *res) {
    wd::NvtxRange nvtx_("wd_cg_solve_canonical");
    if (!c) return WD_ERR_ARG;
    if (!b_canon || !x_canon || !prm || !res) return fail(c, WD_ERR_ARG, "wd_cg_solve_canonical: null argument");
    const int nrhs = prm->nrhs < 1 ? 1 : prm->nrhs;
    if (nrhs > WD_MAX_RHS) return fail(c, WD_ERR_ARG, "wd_cg_solve_canonical: nrhs above WD_MAX_RHS");
    const size_t fb = spinor_bytes(F64, c->g.Vs) * nrhs;
    void *bf, *xf;
    wd_status s;
    if ((s = ws_get(c, "canon_b", fb, &bf)) != WD_OK) return s;
    if ((s = ws_get(c, "canon_x", fb, &xf)) != WD_OK) return s;
    if ((s = wd_pack(c, b_canon, on_device, bf, WD_F64, nrhs)) != WD_OK) return s;
    if ((s = wd_pack(c, x_canon, on_device, xf, WD_F64, nrhs)) != WD_OK) return s;
    wd_status sol = wd_cg_solve(c, kappa, bf, xf, prm, res);
    const long long l = c->launches;
    if (sol != WD_OK && sol != WD_ERR_NOT_CONVERGED && sol != WD_ERR_BREAKDOWN && sol != WD_ERR_NONFINITE) return sol;
    if ((s = wd_unpack(c, xf, WD_F64, nrhs, x_canon, on_device)) != WD_OK) return s;
    c->launches = l + 4;
    return sol;
}

// Solver autotuner: the launch shape of the fused CG kernels is timed as the solver runs
// them, a fixed number of iterations of the device-resident loop on a non-zero right-hand
// side, with L2 flushed before each timed solve (the candidates as in wd_autotune).
wd_status wd_autotune_cg(wd_ctx *c, wd_prec prec, int nrhs, int *site_tile, int *rhs_tile) {
    wd::NvtxRange nvtx_("wd_autotune_cg");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if ((int)prec < 0 || (int)prec >= kNumPrec || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, "wd_autotune_cg: bad argument");
    if (c->split) return fail(c, WD_ERR_STATE, "wd_autotune_cg: not on a split sub-lattice");
    if (!c->has_gauge) return fail(c, WD_ERR_STATE, "wd_autotune_cg: no gauge field set");
    const size_t fb = spinor_bytes(F64, c->g.Vs) * (size_t)nrhs;
    const size_t flush_bytes = (size_t)256 << 20;  // twice the L2 of a GB300
    void *b, *x, *flush;
    wd_status s;
    if ((s = ws_get(c, "tunecg_b", fb, &b)) != WD_OK) return s;
    if ((s = ws_get(c, "tunecg_x", fb, &x)) != WD_OK) return s;
    if ((s = ws_get(c, "tunecg_flush", flush_bytes, &flush)) != WD_OK) return s;
    k_fill_hash<double><<<1024, 256, 0, c->stream>>>(static_cast<double *>(b), fb / sizeof(double));
    WD_CUDA(c, cudaGetLastError());
    wd_cg_params prm{};
    prm.tol = 1e-20;  // never met: every candidate runs max_iter iterations
    prm.max_iter = 10;
    prm.inner_prec = prec;
    prm.nrhs = nrhs;
    std::vector<wd_cg_result> res(nrhs);
    const int sts[] = {16, 32, 64, 128, 256};
    const int rts[] = {1, 2, 3, 4, 6, 8, 12, 16};
    bool even = true;
    for (int mu = 0; mu < 4; ++mu) even &= c->g.L[mu] % 2 == 0;
    long long launches = 1;
    DslashTiles chosen{};
    // plain solves, then (all extents even) even-odd solves, whose checkerboard kernels
    // may prefer another shape
    for (int pc = 0; pc < (even ? 2 : 1); ++pc) {
        prm.precondition = pc;
        const int key = (int)prec * 64 + nrhs + (pc ? kEoTileKey : 0);
        double best = 1e30;
        DslashTiles bt = cg_tiles_for(c, (Prec)prec, nrhs, pc != 0);
        for (int st : sts)
            for (int rt : rts) {
                if (rt > nrhs || st * rt > 256 || (st * rt) % 32 != 0) continue;
                if (threads_per_site((Prec)prec) > 1 && st % 32 != 0) continue;
                DslashTiles t;
                t.site_tile = st;
                t.rhs_tile = rt;
                c->cg_tiles[key] = t;
                double secs = 0.0;
                for (int rep = 0; rep < 2; ++rep) {  // the first run builds and uploads the graph
                    WD_CUDA(c, cudaMemsetAsync(x, 0, fb, c->stream));
                    WD_CUDA(c, cudaMemsetAsync(flush, rep, flush_bytes, c->stream));
                    s = wd_cg_solve(c, 0.12, b, x, &prm, res.data());
                    if (s != WD_OK && s != WD_ERR_NOT_CONVERGED) {
                        c->cg_tiles[key] = bt;
                        return s;
                    }
                    launches += c->launches;
                    secs = res[0].seconds;
                }
                if (secs < best) {
                    best = secs;
                    bt = t;
                }
            }
        c->cg_tiles[key] = bt;
        if (pc == 0) chosen = bt;
    }
    const DslashTiles bt = chosen;
    ws_release(c, "tunecg_flush");
    ws_release(c, "tunecg_b");
    ws_release(c, "tunecg_x");
    c->launches = launches;
    if (site_tile) *site_tile = bt.site_tile;
    if (rhs_tile) *rhs_tile = bt.rhs_tile;
    return WD_OK;
}

}  // extern "C"
