// Block CG over k right-hand sides (k <= WD_MAX_RHS), FP64, on A = D^dag D.
//
// One Krylov space for all columns (O'Leary's block conjugate gradient):
//   R = D^dag B - A X, P = R, G = R^dag R
//   loop:  W = D P;  Pi = W^dag W (= P^dag A P);  alpha = Pi^-1 G
//          Q = D^dag W;  X += P alpha;  R -= Q alpha
//          G' = R^dag R;  beta = G^-1 G';  G = G'
//          P <- R + P beta
//   stop when every column has |R_j|^2 <= tol^2 |D^dag b_j|^2
// The k x k Hermitian systems are solved by Cholesky in the last block of the
// Gram-matrix kernel; a non-positive pivot is a breakdown (rank-deficient block).
// P and W swap roles every iteration (the update of P reads every old column),
// so the graph body holds two iterations.  Applied to D x = b through the normal
// equations of section 2.2, with the 12 spin-colour point sources of section 2.3.
#include <cmath>
#include <cstdlib>
#include "cg_kernels.cuh"
#include "plan.cuh"
#include "wd_host.h"

using namespace wd;

namespace wd {

struct BlockState {
    double2 gam[WD_MAX_RHS * WD_MAX_RHS];    // R^dag R
    double2 alpha[WD_MAX_RHS * WD_MAX_RHS];
    double2 beta[WD_MAX_RHS * WD_MAX_RHS];
    int k, iter, max_iter, status, active, pad[3];
};

struct GramArgs {
    int V, Vs, k;
    const void *A, *B;
    size_t stride;
    Scalars *sc;
    BlockState *bs;
    double *partial;
    unsigned *counter;
};

struct MixArgs {
    int V, Vs, k;
    void *X, *R;              // X += P alpha ; R -= Q alpha      (mode 0)
    const void *P, *Q;        // W = R + P beta                    (mode 1: X = W)
    size_t stride;
    BlockState *bs;
    unsigned long long cond;  // set the loop condition (mode 2)
};

__device__ __forceinline__ double2 cm(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 cmc(double2 a, double2 b) { return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }

// Cholesky M = L L^dag in place (lower triangle), k x k row-major; false on a
// non-positive or non-finite pivot.
__device__ bool cholesky(double2 *M, int k) {
    for (int j = 0; j < k; ++j) {
        double d = M[j * k + j].x;
        for (int p = 0; p < j; ++p) d -= M[j * k + p].x * M[j * k + p].x + M[j * k + p].y * M[j * k + p].y;
        if (!(d > 0.0) || !isfinite(d)) return false;
        const double l = sqrt(d);
        M[j * k + j] = make_double2(l, 0.0);
        for (int i = j + 1; i < k; ++i) {
            double2 s = M[i * k + j];
            for (int p = 0; p < j; ++p) {
                const double2 t = cmc(M[j * k + p], M[i * k + p]);  // conj(L_jp) L_ip
                s.x -= t.x;
                s.y -= t.y;
            }
            M[i * k + j] = make_double2(s.x / l, s.y / l);
        }
    }
    return true;
}

// Solve L L^dag Y = Rhs (k x k, column by column) in place in Rhs.
__device__ void chol_solve(const double2 *L, double2 *Y, int k) {
    for (int c = 0; c < k; ++c) {
        for (int i = 0; i < k; ++i) {  // L z = y
            double2 s = Y[i * k + c];
            for (int p = 0; p < i; ++p) {
                const double2 t = cm(L[i * k + p], Y[p * k + c]);
                s.x -= t.x;
                s.y -= t.y;
            }
            Y[i * k + c] = make_double2(s.x / L[i * k + i].x, s.y / L[i * k + i].x);
        }
        for (int i = k - 1; i >= 0; --i) {  // L^dag y = z
            double2 s = Y[i * k + c];
            for (int p = i + 1; p < k; ++p) {
                const double2 t = cmc(L[p * k + i], Y[p * k + c]);
                s.x -= t.x;
                s.y -= t.y;
            }
            Y[i * k + c] = make_double2(s.x / L[i * k + i].x, s.y / L[i * k + i].x);
        }
    }
}

constexpr int kGramNV = 2 * WD_MAX_RHS;

// G = A^dag B (k x k) over all sites; thread (x, i) accumulates row i.  MODE 0:
// G -> gam (initial residual Gram matrix, convergence check); MODE 1: alpha =
// G^-1 gam; MODE 2: beta = gam^-1 G, gam = G, iteration count and stopping test.
template <int MODE>
__global__ void __launch_bounds__(512) k_gram(GramArgs g) {
    if (MODE != 0 && g.bs->active == 0) return;
    const int i = threadIdx.y, k = g.k;
    double v[kGramNV];
#pragma unroll
    for (int q = 0; q < kGramNV; ++q) v[q] = 0.0;
    for (int s0 = blockIdx.x * blockDim.x; s0 < g.V; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        if (s < g.V && i < k) {
            C<double> a[12];
            SpinorIO<F64>::load(reinterpret_cast<const char *>(g.A) + g.stride * i, g.Vs, s, a);
#pragma unroll
            for (int j = 0; j < WD_MAX_RHS; ++j) {
                if (j < k) {
                    C<double> b[12];
                    SpinorIO<F64>::load(reinterpret_cast<const char *>(g.B) + g.stride * j, g.Vs, s, b);
                    double re = 0.0, im = 0.0;
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        re += a[c].re * b[c].re + a[c].im * b[c].im;
                        im += a[c].re * b[c].im - a[c].im * b[c].re;
                    }
                    v[2 * j] += re;
                    v[2 * j + 1] += im;
                }
            }
        }
    }
    __shared__ double smem[WD_MAX_RHS * kGramNV];
    __shared__ double tot[WD_MAX_RHS * kGramNV];
    block_reduce_rows<kGramNV, 1>(v, smem);  // site tiles of at most 32 threads
    if (threadIdx.x == 0 && i < k)
#pragma unroll
        for (int q = 0; q < kGramNV; ++q) g.partial[((size_t)i * kGramNV + q) * gridDim.x + blockIdx.x] = v[q];
    if (!last_block(g.counter)) return;
    sum_partials<kGramNV>(g.partial, gridDim.x, k, tot);
    __shared__ double2 G[WD_MAX_RHS * WD_MAX_RHS], L[WD_MAX_RHS * WD_MAX_RHS];
    if (threadIdx.x != 0 || threadIdx.y != 0) return;
    *g.counter = 0;
    BlockState &bs = *g.bs;
    bool finite = true;
    for (int r = 0; r < k; ++r)
        for (int c = 0; c < k; ++c) {
            G[r * k + c] = make_double2(tot[r * kGramNV + 2 * c], tot[r * kGramNV + 2 * c + 1]);
            finite &= isfinite(G[r * k + c].x) && isfinite(G[r * k + c].y);
        }
    auto stop_all = [&](int st) {
        bs.active = 0;
        bs.status = st;
        for (int r = 0; r < k; ++r) g.sc[r].status = st;
    };
    if (!finite) { stop_all(WD_ERR_NONFINITE); return; }
    if (MODE == 0 || MODE == 2) {
        if (MODE == 2) {
            for (int q = 0; q < k * k; ++q) { L[q] = bs.gam[q]; bs.beta[q] = G[q]; }
            bs.iter += 1;
            for (int r = 0; r < k; ++r) g.sc[r].iter = bs.iter;
            if (!cholesky(L, k)) { stop_all(WD_ERR_BREAKDOWN); return; }
            chol_solve(L, bs.beta, k);
        }
        bool conv = true;
        for (int q = 0; q < k * k; ++q) bs.gam[q] = G[q];
        for (int r = 0; r < k; ++r) {
            g.sc[r].rho = G[r * k + r].x;
            conv &= G[r * k + r].x <= g.sc[r].tol2;
        }
        if (conv) stop_all(WD_OK);
        else if (bs.iter >= bs.max_iter) stop_all(WD_ERR_NOT_CONVERGED);
    } else {
        for (int q = 0; q < k * k; ++q) bs.alpha[q] = bs.gam[q];
        if (!cholesky(G, k)) { stop_all(WD_ERR_BREAKDOWN); return; }
        chol_solve(G, bs.alpha, k);
    }
}

// MODE 0: X_j += sum_i P_i alpha_ij, R_j -= sum_i Q_i alpha_ij.
// MODE 1: X_j (= W_j) = R_j + sum_i P_i beta_ij.
template <int MODE>
__global__ void __launch_bounds__(512) k_block_mix(MixArgs m) {
    if (m.bs->active == 0) return;
    __shared__ double2 coef[WD_MAX_RHS * WD_MAX_RHS];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x, k = m.k;
    for (int q = tid; q < k * k; q += blockDim.x * blockDim.y) coef[q] = MODE == 0 ? m.bs->alpha[q] : m.bs->beta[q];
    __syncthreads();
    const int j = threadIdx.y;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= m.V || j >= k) return;
    C<double> sp[12], sq[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) sp[c] = sq[c] = C<double>{0.0, 0.0};
    for (int i = 0; i < k; ++i) {
        const double2 w = coef[i * k + j];
        C<double> p[12];
        SpinorIO<F64>::load(reinterpret_cast<const char *>(m.P) + m.stride * i, m.Vs, s, p);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            sp[c].re += p[c].re * w.x - p[c].im * w.y;
            sp[c].im += p[c].re * w.y + p[c].im * w.x;
        }
        if (MODE == 0) {
            SpinorIO<F64>::load(reinterpret_cast<const char *>(m.Q) + m.stride * i, m.Vs, s, p);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                sq[c].re += p[c].re * w.x - p[c].im * w.y;
                sq[c].im += p[c].re * w.y + p[c].im * w.x;
            }
        }
    }
    C<double> x[12], r[12];
    char *xb = reinterpret_cast<char *>(m.X) + m.stride * j;
    char *rb = reinterpret_cast<char *>(m.R) + m.stride * j;
    SpinorIO<F64>::load(rb, m.Vs, s, r);
    if (MODE == 0) {
        SpinorIO<F64>::load(xb, m.Vs, s, x);
#pragma unroll
        for (int c = 0; c < 12; ++c) {
            x[c] = cadd(x[c], sp[c]);
            r[c] = csub(r[c], sq[c]);
        }
        SpinorIO<F64>::store(xb, m.Vs, s, x);
        SpinorIO<F64>::store(rb, m.Vs, s, r);
    } else {
#pragma unroll
        for (int c = 0; c < 12; ++c) x[c] = cadd(r[c], sp[c]);
        SpinorIO<F64>::store(xb, m.Vs, s, x);
    }
}

__global__ void k_block_cond(MixArgs m) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int cap = m.bs->max_iter + 4;
        cudaGraphSetConditional((cudaGraphConditionalHandle)m.cond,
                                (m.bs->active && m.bs->iter < cap) ? 1u : 0u);
    }
}

struct BlockBufs {
    void *B, *X, *DB, *R, *P, *W, *Q, *T;
    Scalars *sc;
    BlockState *bs;
    double *partial;
    unsigned *counter;
    int *state;
};

template <int RECON>
static void record_block(wd_ctx *c, double kappa, int k, const void *g64, const BlockBufs &f,
                         cudaGraphConditionalHandle hw, Plan &plan) {
    const size_t fs = spinor_bytes(F64, c->g.Vs);
    const DslashTiles t64 = tiles_for(c, F64, k);
    DslashArgs base{};
    base.g = c->g;
    base.gauge = g64;
    base.gauge_dir = gauge_dir_bytes(c, F64);
    base.kappa = kappa;
    base.nrhs = k;
    base.sc = f.sc;
    base.mask = 0;
    base.partial = f.partial;
    base.counter = f.counter;
    base.state = f.state;
    base.in_stride = base.out_stride = base.a0_stride = base.a1_stride = base.a2_stride = base.a3_stride = fs;
    GramArgs ga{};
    ga.V = c->g.V; ga.Vs = c->g.Vs; ga.k = k; ga.stride = fs; ga.sc = f.sc; ga.bs = f.bs;
    ga.partial = f.partial; ga.counter = f.counter;
    MixArgs ma{};
    ma.V = c->g.V; ma.Vs = c->g.Vs; ma.k = k; ma.stride = fs; ma.bs = f.bs;
    // (site tile x k) blocks: 16 sites when 16k is a multiple of 32, else 32 (<= 512 threads)
    const int st = (16 * k) % 32 == 0 ? 16 : 32;
    const int tiles = (c->g.V + st - 1) / st;
    const int gcap = 2 * num_sms();  // Gram kernels: at most two blocks per SM, one partial each
    const dim3 blk(st, k), ggrid(tiles < gcap ? tiles : gcap), mgrid(tiles);
    {
        GraphBuilder gb(&plan.setup);
        DslashArgs a = base;
        a.in = f.B; a.out = f.DB;
        add_dslash<F64, RECON, true, EpSetupDb>(gb, a, t64, true);
        a.in = f.X; a.out = f.T;
        add_dslash<F64, RECON, false, EpXpay>(gb, a, t64, false);
        a.in = f.T; a.a0 = f.DB; a.a1 = f.R; a.a2 = f.P;
        add_dslash<F64, RECON, true, EpSetupR>(gb, a, t64, true);
        GramArgs g0 = ga;
        g0.A = f.R; g0.B = f.R;
        gb.kernel(k_gram<0>, ggrid, blk, g0);
    }
    {
        GraphBuilder bb(&plan.pre);
        void *PP[2] = {f.P, f.W};
        for (int h = 0; h < 2; ++h) {
            void *Pc = PP[h], *Wc = PP[1 - h];
            DslashArgs a = base;
            a.run_flag = &f.bs->active;
            a.in = Pc; a.out = Wc;
            add_dslash<F64, RECON, false, EpXpay>(bb, a, t64, false);
            GramArgs g1 = ga;
            g1.A = Wc; g1.B = Wc;
            bb.kernel(k_gram<1>, ggrid, blk, g1);
            a.in = Wc; a.out = f.Q;
            add_dslash<F64, RECON, true, EpXpay>(bb, a, t64, false);
            MixArgs m0 = ma;
            m0.X = f.X; m0.R = f.R; m0.P = Pc; m0.Q = f.Q;
            bb.kernel(k_block_mix<0>, mgrid, blk, m0);
            GramArgs g2 = ga;
            g2.A = f.R; g2.B = f.R;
            bb.kernel(k_gram<2>, ggrid, blk, g2);
            MixArgs m1 = ma;
            m1.X = Wc; m1.R = f.R; m1.P = Pc;
            bb.kernel(k_block_mix<1>, mgrid, blk, m1);
        }
        MixArgs mc = ma;
        mc.cond = hw;
        bb.kernel(k_block_cond, dim3(1), dim3(32), mc);
    }
    {
        GraphBuilder gb(&plan.fin);
        DslashArgs a = base;
        a.in = f.X; a.out = f.T; a.a0 = f.B;
        add_dslash<F64, RECON, false, EpTrue1>(gb, a, t64, true);
        a.in = f.T; a.a0 = f.DB;
        add_dslash<F64, RECON, true, EpTrue2>(gb, a, t64, true);
    }
}

wd_status block_cg_solve(wd_ctx *c, double kappa, const void *b, void *x, const wd_cg_params *prm,
                         wd_cg_result *res) {
    const int k = prm->nrhs < 1 ? 1 : prm->nrhs;
    const void *g64;
    wd_status s = gauge_get(c, F64, &g64);
    if (s != WD_OK) return s;
    const size_t fk = spinor_bytes(F64, c->g.Vs) * k;
    BlockBufs f{};
    void *tmp;
    const char *names[8] = {"bk_b", "bk_x", "bk_db", "bk_r", "bk_p", "bk_w", "bk_q", "bk_t"};
    void **ptrs[8] = {&f.B, &f.X, &f.DB, &f.R, &f.P, &f.W, &f.Q, &f.T};
    for (int i = 0; i < 8; ++i)
        if ((s = ws_get(c, names[i], fk, ptrs[i])) != WD_OK) return s;
    if ((s = ws_get(c, "cg_scalars", sizeof(Scalars) * WD_MAX_RHS, &tmp)) != WD_OK) return s;
    f.sc = (Scalars *)tmp;
    if ((s = ws_get(c, "bk_state", sizeof(BlockState), &tmp)) != WD_OK) return s;
    f.bs = (BlockState *)tmp;
    const size_t npart = (size_t)WD_MAX_RHS * 3 * kMaxPartialBlocks;
    if ((s = ws_get(c, "partial", npart * sizeof(double), &tmp)) != WD_OK) return s;
    f.partial = (double *)tmp;
    if ((s = ws_get(c, "counter", 256, &tmp)) != WD_OK) return s;
    f.counter = (unsigned *)tmp;
    f.state = (int *)((char *)tmp + 64);
    Scalars *sc = f.sc;
    BlockState *bs = f.bs;
    void *B = f.B, *X = f.X;

    const DslashTiles t64 = tiles_for(c, F64, k);
    char key[200];
    snprintf(key, sizeof key, "bcg|%d|%d|%a|%d,%d", k, link_recon(c, F64), kappa, t64.site_tile, t64.rhs_tile);
    cudaGraphExec_t exec = (cudaGraphExec_t)graph_get(c, key);
    if (!exec) {
        cudaGraph_t graph;
        WD_CUDA(c, cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle hw = 0;
        cudaError_t e = cudaGraphConditionalHandleCreate(&hw, graph, 1, cudaGraphCondAssignDefault);
        Plan plan;
        with_recon(link_recon(c, F64), [&](auto rc) { record_block<decltype(rc)::value>(c, kappa, k, g64, f, hw, plan); });
        std::vector<cudaGraphNode_t> deps;
        if (e == cudaSuccess) e = add_chain(graph, deps, plan.setup);
        cudaGraph_t body = nullptr;
        if (e == cudaSuccess) e = add_conditional(graph, deps, hw, cudaGraphCondTypeWhile, &body);
        if (e == cudaSuccess) {
            std::vector<cudaGraphNode_t> bd;
            e = add_chain(body, bd, plan.pre);
        }
        if (e == cudaSuccess) e = add_chain(graph, deps, plan.fin);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(c, e, "building the block-CG graph");
        graph_put(c, key, exec, {(long long)plan.setup.size(), (long long)plan.pre.size(), 0,
                                 (long long)plan.fin.size()});
        WD_CUDA(c, cudaMemsetAsync(f.counter, 0, 256, c->stream));
    }

    std::vector<Scalars> h(k);
    for (int r = 0; r < k; ++r) {
        std::memset(&h[r], 0, sizeof(Scalars));
        h[r].tol2 = prm->tol * prm->tol;
        h[r].max_iter = prm->max_iter;
        h[r].active = 1;
        h[r].status = WD_ERR_NOT_CONVERGED;
    }
    BlockState hb;
    std::memset(&hb, 0, sizeof hb);
    hb.k = k;
    hb.max_iter = prm->max_iter;
    hb.active = 1;
    hb.status = WD_ERR_NOT_CONVERGED;
    WD_CUDA(c, cudaMemcpyAsync(sc, h.data(), sizeof(Scalars) * k, cudaMemcpyHostToDevice, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(bs, &hb, sizeof hb, cudaMemcpyHostToDevice, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(B, b, fk, cudaMemcpyDeviceToDevice, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(X, x, fk, cudaMemcpyDeviceToDevice, c->stream));
    EventPair ev;
    WD_CUDA(c, ev.create());
    cudaEvent_t e0 = ev.e0, e1 = ev.e1;
    WD_CUDA(c, cudaEventRecord(e0, c->stream));
    WD_CUDA(c, cudaGraphLaunch(exec, c->stream));
    WD_CUDA(c, cudaEventRecord(e1, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(x, X, fk, cudaMemcpyDeviceToDevice, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(h.data(), sc, sizeof(Scalars) * k, cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(c, cudaMemcpyAsync(&hb, bs, sizeof hb, cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    const std::vector<long long> &cnt = c->graph_info[key];
    c->launches = cnt[0] + (long long)((hb.iter + 1) / 2 + 1) * cnt[1] + cnt[3];
    wd_status worst = WD_OK;
    for (int r = 0; r < k; ++r) {
        res[r].iters = hb.iter;
        res[r].reliable_updates = 0;
        res[r].inner_corrections = 0;
        res[r].true_rel_resid = h[r].rhs2 > 0 ? std::sqrt(h[r].true_n2 / h[r].rhs2) : std::sqrt(h[r].true_n2);
        res[r].true_rel_resid_b = h[r].b2 > 0 ? std::sqrt(h[r].true_b2 / h[r].b2) : std::sqrt(h[r].true_b2);
        res[r].seconds = ms * 1e-3;
        res[r].status = hb.status;
        if (hb.status != WD_OK && worst == WD_OK) worst = (wd_status)hb.status;
    }
    if (worst != WD_OK) c->last_error = std::string("block CG: ") + wd_status_string(worst);
    return worst;
}

}  // namespace wd
