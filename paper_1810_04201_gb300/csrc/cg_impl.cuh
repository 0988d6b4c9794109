// Solver plans of the device-resident CG (section 2.2): the recording of every
// kernel of one solve for a given link compression, inner precision, normal form
// and preconditioning, and its assembly into a CUDA graph with device-side loop.
// Each pair of link compressions (FP64, inner precision) is instantiated in its own
// translation unit (cg_recon18.cu, cg_recon12.cu, cg_recon8.cu, cg_recon18_12.cu,
// cg_recon18_8.cu), which keeps the build parallel.
#pragma once
#include <vector>
#include "cg_kernels.cuh"
#include "plan.cuh"
#include "wd_host.h"

namespace wd {

// Record the FP64 (inner == F64) or mixed-precision solver.  hwhile / hif are the
// conditional handles the loop kernels set (0 for the host-driven loop).
// NE = false: CGNR, A = D^dag D, rhs D^dag b.  NE = true: CGNE, the paper's form
// (section 2.2): A = D D^dag, rhs b, iterate y (kept in the x field), x = D^dag y.
// The two share every kernel; only which of D and D^dag comes first changes.
// EO = true: even-odd preconditioning; the iteration runs on the even half with
// the Schur operator, the odd half is rebuilt at the end (CGNR only).
template <int RECON, int RIN, int SP, bool NE, bool EO>
static void record_plan(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                        cudaGraphConditionalHandle hwhile, cudaGraphConditionalHandle hif, Plan &plan) {
    static_assert(!(NE && EO), "even-odd preconditioning is built for CGNR");
    GraphBuilder gb(&plan.setup);
    const Geom gw = EO ? f.eo.ge : c->g;  // geometry of the iterated fields
    const size_t s64 = spinor_bytes(F64, gw.Vs), sin = spinor_bytes((Prec)SP, gw.Vs), s32 = spinor_bytes(F32, gw.Vs);
    const bool mixed = SP != F64;

    DslashArgs base{};
    base.g = gw;
    base.gauge = g64;
    base.gauge_dir = gauge_dir_bytes(c, F64);
    base.kappa = pl.kappa;
    base.nrhs = pl.nrhs;
    base.sc = f.sc;
    base.partial = f.partial;
    base.counter = f.counter;
    base.state = f.state;
    base.in_stride = base.out_stride = base.a0_stride = base.a1_stride = base.a2_stride = base.a3_stride = s64;

    VecArgs vb{};
    vb.V = gw.V;
    vb.Vs = gw.Vs;
    vb.nrhs = pl.nrhs;
    vb.sc = f.sc;
    vb.state = f.state;

    // first (OP1) and second (OP2) operator of A: CGNR D then D^dag, CGNE D^dag then D
    constexpr bool OP1 = NE, OP2 = !NE;
    const size_t sfull = spinor_bytes(F64, c->g.Vs);
    if constexpr (EO) {
        // split b and x0 into halves; the Schur right-hand side b^ = b_e + kappa H_eo b_o
        VecArgs v = vb;
        v.V = c->g.V;
        v.Vs = c->g.Vs;
        v.mask = 0;
        v.a = f.eo.bfull; v.a_stride = sfull; v.b = f.eo.be; v.c = f.eo.bo; v.b_stride = s64;
        gb.kernel(k_split_eo<0>, dim3((v.V + 127) / 128, v.nrhs), dim3(128), EoVecArgs{v, gw.Vs, c->g});
        v.a = f.eo.xfull; v.b = f.x; v.c = f.eo.xo;
        gb.kernel(k_split_eo<0>, dim3((v.V + 127) / 128, v.nrhs), dim3(128), EoVecArgs{v, gw.Vs, c->g});
        DslashArgs a = base;
        a.mask = 0;
        a.g = f.eo.ge;
        a.gauge = f.eo.gauge[F64];
        a.gauge_dir = f.eo.gdir[F64];
        a.in = f.eo.bo; a.xsrc = f.eo.be; a.xsrc_stride = s64; a.out = f.b;
        a.kappa = -pl.kappa;
        add_dslash<F64, RECON, false, EpXpay, true>(gb, a, pl.t64, false);
    }
    // ---- setup (FP64): db = rhs; t = OP1 x0; r = db - OP2 t; p = r
    {
        DslashArgs a = base;
        a.mask = 0;
        a.in = f.b; a.out = f.db;
        if (NE) a.kappa = 0.0;  // D with kappa = 0 is the identity: db = b, |b|^2
        add_op<F64, RECON, true, EpSetupDb, EO>(gb, a, pl.t64, true, f);
        // a zero start vector (the usual case) makes t = OP1 x0 and OP2 t vanish:
        // state[2] marks a nonzero x0, and without one those kernels do no work
        VecArgs v = vb;
        v.mask = 0;
        v.a = f.x; v.a_stride = s64;
        gb.kernel(k_any_nonzero<0>, dim3((v.V + 127) / 128, v.nrhs), dim3(128), v);
        a.kappa = pl.kappa;
        a.in = f.x; a.out = f.t;
        a.run_flag = f.state + 2;
        add_op<F64, RECON, OP1, EpXpay, EO>(gb, a, pl.t64, false, f);
        a.run_flag = nullptr;
        a.in = f.t; a.a0 = f.db; a.a1 = f.r; a.a2 = f.p;
        a.in_nonzero = f.state + 2;
        add_op<F64, RECON, OP2, EpSetupR, EO>(gb, a, pl.t64, true, f);
        a.in_nonzero = nullptr;
    }
    if (mixed) {
        VecArgs v = vb;
        v.mask = 0;
        v.a = f.r; v.a_stride = s64; v.b = f.rs; v.b_stride = sin;
        add_vec(gb, k_convert<F64, SP>, v);
        v.b = f.ps;
        add_vec(gb, k_convert<F64, SP>, v);
        v.b = f.xs; v.b_stride = s32;
        add_vec(gb, k_zero<F32>, v);
    }

    // ---- loop
    {
        GraphBuilder bb(&plan.pre);
        if (!mixed) {
            DslashArgs a = base;
            a.mask = 1;
            a.in = f.p; a.out = f.t;
            add_op<F64, RECON, OP1, EpCG1, EO>(bb, a, pl.t64, true, f);
            a.in = f.t; a.a0 = f.p; a.a1 = f.r; a.a2 = f.x;
            add_op<F64, RECON, OP2, EpCG2, EO>(bb, a, pl.t64, true, f);
            VecArgs v = vb;
            v.mask = 1;
            v.a = f.r; v.a_stride = s64; v.b = f.p; v.b_stride = s64; v.cond = hwhile;
            add_vec(bb, k_xpby<F64>, v);
        } else {
            DslashArgs a = base;
            a.mask = 1;
            a.gauge = gin;
            a.gauge_dir = gauge_dir_bytes(c, (Prec)SP);
            a.in_stride = a.out_stride = a.a0_stride = a.a1_stride = sin;
            a.a2_stride = s32;
            a.in = f.ps; a.out = f.ts;
            add_op<SP, RIN, OP1, EpCG1, EO>(bb, a, pl.tin, true, f);
            a.in = f.ts; a.a0 = f.ps; a.a1 = f.rs; a.a2 = f.xs; a.cond = hif;
            add_op<SP, RIN, OP2, EpCG2Mixed, EO>(bb, a, pl.tin, true, f);
            plan.has_if = true;
            {
                GraphBuilder ib(&plan.ifb);
                VecArgs v = vb;
                v.mask = 2;
                v.a = f.xs; v.a_stride = s32; v.b = f.x; v.b_stride = s64;
                add_vec(ib, k_reliable_x<0>, v);
                DslashArgs r = base;
                r.mask = 2;
                r.in = f.x; r.out = f.t;
                if constexpr (!EO && !NE) {
                    // t = D x with |b - t|^2: an update that stops a row is its final check
                    r.a0 = f.b;
                    add_op<F64, RECON, OP1, EpTrue1, EO>(ib, r, pl.t64, true, f);
                    r.a0 = nullptr;
                } else {
                    add_op<F64, RECON, OP1, EpXpay, EO>(ib, r, pl.t64, false, f);
                }
                r.in = f.t; r.a0 = f.db; r.a1 = f.r;
                add_op<F64, RECON, OP2, EpReliable, EO>(ib, r, pl.t64, true, f);
                v.a = f.r; v.a_stride = s64; v.b = f.rs; v.b_stride = sin;
                add_vec(ib, k_convert<F64, SP>, v);
                if constexpr (SP == F16) {
                    if (f.t32) {
                        // FP32 correction (rows with do_correct): t32 = A1 xs; rs = r64 - A2 t32,
                        // on the FP32 links (compressed as the FP64 copy, or as the inner one)
                        DslashArgs q = base;
                        q.mask = 3;
                        q.gauge = f.g32;
                        q.gauge_dir = gauge_dir_bytes(c, F32);
                        q.in_stride = q.out_stride = s32;
                        q.in = f.xs; q.out = f.t32;
                        DslashArgs q2 = q;
                        q2.in = f.t32; q2.a0 = f.r; q2.a0_stride = s64; q2.a1 = f.rs; q2.a1_stride = sin;
                        if (f.c32_inner) {
                            add_op<F32, RIN, OP1, EpXpay, EO>(ib, q, pl.tin, false, f);
                            add_op<F32, RIN, OP2, EpCorrect<SP>, EO>(ib, q2, pl.tin, true, f);
                        } else {
                            add_op<F32, RECON, OP1, EpXpay, EO>(ib, q, pl.tin, false, f);
                            add_op<F32, RECON, OP2, EpCorrect<SP>, EO>(ib, q2, pl.tin, true, f);
                        }
                    }
                }
            }
            bb.cur = &plan.post;
            VecArgs v = vb;
            v.mask = 1;
            v.a = f.rs; v.a_stride = sin; v.b = f.ps; v.b_stride = sin; v.cond = hwhile;
            add_vec(bb, k_xpby<SP>, v);
        }
    }

    // ---- final FP64 check: t = D x, |b - t|^2; |D^dag b - D^dag t|^2 (full lattice)
    gb.cur = &plan.fin;
    DslashArgs a = base;
    a.mask = 0;
    void *xf = f.x, *bf = f.b, *tf = f.t, *dbt = f.db;
    if constexpr (EO) {
        // x_o = b_o + kappa H_oe x_e, join the halves, then check on the full lattice
        DslashArgs o = base;
        o.mask = 0;
        o.g = f.eo.go;
        o.gauge = f.eo.gauge[F64];
        o.gauge_dir = f.eo.gdir[F64];
        o.in = f.x; o.xsrc = f.eo.bo; o.xsrc_stride = s64; o.out = f.eo.xo;
        o.kappa = -pl.kappa;
        add_dslash<F64, RECON, false, EpXpay, true>(gb, o, pl.t64, false);
        VecArgs v = vb;
        v.V = c->g.V;
        v.Vs = c->g.Vs;
        v.mask = 0;
        v.a = f.x; v.c = f.eo.xo; v.a_stride = s64; v.b = f.eo.xfull; v.b_stride = sfull;
        gb.kernel(k_join_eo<0>, dim3((v.V + 127) / 128, v.nrhs), dim3(128), EoVecArgs{v, gw.Vs, c->g});
        a.g = c->g;
        a.gauge = g64;
        a.gauge_dir = gauge_dir_bytes(c, F64);
        a.in_stride = a.out_stride = a.a0_stride = sfull;
        xf = f.eo.xfull; bf = f.eo.bfull; tf = f.eo.tfull; dbt = f.eo.dbfull;
        a.in = bf; a.out = dbt;
        add_dslash<F64, RECON, true, EpSetupDb>(gb, a, pl.t64, true);
    }
    if (NE) {
        // x = D^dag y ; D^dag b (into p) and its norm for the normal-equation residual
        a.in = f.x; a.out = f.t;
        add_dslash<F64, RECON, true, EpXpay>(gb, a, pl.t64, false);
        VecArgs v = vb;
        v.mask = 0;
        v.a = f.t; v.a_stride = s64; v.b = f.x; v.b_stride = s64;
        add_vec(gb, k_convert<F64, F64>, v);
        a.in = f.b; a.out = f.p;
        add_dslash<F64, RECON, true, EpSetupDb>(gb, a, pl.t64, true);
        dbt = f.p;
    }
    a.in = xf; a.out = tf; a.a0 = bf;
    // mixed precision on the full lattice: skipped when every row stopped at a reliable
    // update, which computed these norms for the x it returns (state[4] = 0)
    if (mixed && !EO && !NE) a.run_flag = f.state + 4;
    add_dslash<F64, RECON, false, EpTrue1>(gb, a, pl.t64, true);
    a.in = tf; a.a0 = dbt;
    add_dslash<F64, RECON, true, EpTrue2>(gb, a, pl.t64, true);
}

// One CUDA graph: setup -> WHILE { pre -> IF { ifb } -> post } -> final.
template <int RECON, int RIN, int SP, bool NE, bool EO>
static cudaError_t build_graph(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                               cudaGraphExec_t *exec, std::vector<long long> &counts) {
    cudaGraph_t graph;
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e != cudaSuccess) return e;
    cudaGraphConditionalHandle hwhile = 0, hif = 0;
    e = cudaGraphConditionalHandleCreate(&hwhile, graph, 1, cudaGraphCondAssignDefault);
    if (e == cudaSuccess && SP != F64) e = cudaGraphConditionalHandleCreate(&hif, graph, 0, cudaGraphCondAssignDefault);
    Plan plan;
    if (e == cudaSuccess) record_plan<RECON, RIN, SP, NE, EO>(c, pl, f, g64, gin, hwhile, hif, plan);
    std::vector<cudaGraphNode_t> deps;
    if (e == cudaSuccess) e = add_chain(graph, deps, plan.setup);
    cudaGraph_t body = nullptr;
    if (e == cudaSuccess) e = add_conditional(graph, deps, hwhile, cudaGraphCondTypeWhile, &body);
    if (e == cudaSuccess) {
        std::vector<cudaGraphNode_t> bd;
        e = add_chain(body, bd, plan.pre);
        if (e == cudaSuccess && plan.has_if) {
            cudaGraph_t ifg = nullptr;
            e = add_conditional(body, bd, hif, cudaGraphCondTypeIf, &ifg);
            std::vector<cudaGraphNode_t> id;
            if (e == cudaSuccess) e = add_chain(ifg, id, plan.ifb);
        }
        if (e == cudaSuccess) e = add_chain(body, bd, plan.post);
    }
    if (e == cudaSuccess) e = add_chain(graph, deps, plan.fin);
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    counts = {(long long)plan.setup.size(), (long long)(plan.pre.size() + plan.post.size()),
              (long long)plan.ifb.size(), (long long)plan.fin.size()};
    return e;
}

// RIN: link compression of the inner precision; a plain FP64 solve has none of its own
// (RIN == RECON), a mixed one may keep whole FP64 links (RECON == 18) beside any RIN.
template <int RECON, int RIN, bool NE, bool EO>
static cudaError_t build_for_ne(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                                cudaGraphExec_t *exec, std::vector<long long> &counts) {
    switch (pl.inner) {
    case F64:
        if constexpr (RIN == RECON) return build_graph<RECON, RIN, F64, NE, EO>(c, pl, f, g64, gin, exec, counts);
        else return cudaErrorInvalidValue;
    case F32: return build_graph<RECON, RIN, F32, NE, EO>(c, pl, f, g64, gin, exec, counts);
    case DF32: return build_graph<RECON, RIN, DF32, NE, EO>(c, pl, f, g64, gin, exec, counts);
    default: return build_graph<RECON, RIN, F16, NE, EO>(c, pl, f, g64, gin, exec, counts);
    }
}

template <int RECON, int RIN>
cudaError_t build_for(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                             cudaGraphExec_t *exec, std::vector<long long> &counts) {
    if (pl.eo) return build_for_ne<RECON, RIN, false, true>(c, pl, f, g64, gin, exec, counts);
    return pl.ne ? build_for_ne<RECON, RIN, true, false>(c, pl, f, g64, gin, exec, counts)
                 : build_for_ne<RECON, RIN, false, false>(c, pl, f, g64, gin, exec, counts);
}

template <int RECON, int RIN, bool NE, bool EO>
static void record_for_ne(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin,
                          Plan &plan) {
    switch (pl.inner) {
    case F64:
        if constexpr (RIN == RECON) record_plan<RECON, RIN, F64, NE, EO>(c, pl, f, g64, gin, 0, 0, plan);
        break;
    case F32: record_plan<RECON, RIN, F32, NE, EO>(c, pl, f, g64, gin, 0, 0, plan); break;
    case DF32: record_plan<RECON, RIN, DF32, NE, EO>(c, pl, f, g64, gin, 0, 0, plan); break;
    default: record_plan<RECON, RIN, F16, NE, EO>(c, pl, f, g64, gin, 0, 0, plan); break;
    }
}

template <int RECON, int RIN>
void record_for(wd_ctx *c, const SolverPlan &pl, const Fields &f, const void *g64, const void *gin, Plan &plan) {
    if (pl.eo) record_for_ne<RECON, RIN, false, true>(c, pl, f, g64, gin, plan);
    else if (pl.ne) record_for_ne<RECON, RIN, true, false>(c, pl, f, g64, gin, plan);
    else record_for_ne<RECON, RIN, false, false>(c, pl, f, g64, gin, plan);
}

}  // namespace wd
