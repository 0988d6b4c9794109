// C ABI of libwd: contexts, gauge upload, pack/unpack and the plain operators.
#include <algorithm>
#include <cstring>
#include <cmath>
#include "dslash.cuh"
#include "blas.cuh"
#include "wd_host.h"

using namespace wd;

namespace wd {

wd_status fail(wd_ctx *c, wd_status s, const std::string &msg) {
    if (c) c->last_error = msg;
    return s;
}

wd_status cuda_fail(wd_ctx *c, cudaError_t e, const char *where) {
    std::string m = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(c, e == cudaErrorMemoryAllocation ? WD_ERR_OOM : WD_ERR_CUDA, m);
}

wd_status ws_get(wd_ctx *c, const std::string &name, size_t bytes, void **out) {
    auto it = c->ws.find(name);
    if (it != c->ws.end() && c->ws_size[name] >= bytes) {
        *out = it->second;
        return WD_OK;
    }
    if (it != c->ws.end()) {
        cudaStreamSynchronize(c->stream);
        cudaFree(it->second);
        c->ws.erase(it);
        // graphs may hold the old pointer
        graph_clear(c);
    }
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, ("cudaMalloc(" + name + ")").c_str());
    c->ws[name] = p;
    c->ws_size[name] = bytes;
    *out = p;
    return WD_OK;
}

size_t gauge_dir_bytes(const wd_ctx *c, Prec p) { return round_up(link_dir_bytes(p, link_recon(c, p), c->g.Vs), 256); }

template <int P, int RECON>
static void gauge_pack(const double *canon, void *dst, const Geom &g, size_t dir, cudaStream_t st) {
    dim3 grid((g.V + 127) / 128, 4);
    k_gauge_pack<P, RECON><<<grid, 128, 0, st>>>(reinterpret_cast<const double2 *>(canon), dst, g.V, g.Vs, dir);
}

wd_status gauge_get(wd_ctx *c, Prec p, const void **out) {
    if (!c->has_gauge) return fail(c, WD_ERR_STATE, "no gauge field set (call wd_set_gauge first)");
    if (!c->gauge[p]) {
        void *d = nullptr;
        WD_CUDA(c, cudaMalloc(&d, gauge_bytes(p, link_recon(c, p), c->g.Vs)));
        const size_t dir = gauge_dir_bytes(c, p);
        with_recon(link_recon(c, p), [&](auto rc) {
            constexpr int R = decltype(rc)::value;
            if (p == F64) gauge_pack<F64, R>(c->gauge_canon, d, c->g, dir, c->stream);
            else if (p == F32) gauge_pack<F32, R>(c->gauge_canon, d, c->g, dir, c->stream);
            else if (p == DF32) gauge_pack<DF32, R>(c->gauge_canon, d, c->g, dir, c->stream);
            else gauge_pack<F16, R>(c->gauge_canon, d, c->g, dir, c->stream);
        });
        WD_CUDA(c, cudaGetLastError());
        c->launches += 1;
        c->gauge[p] = d;
    }
    *out = c->gauge[p];
    return WD_OK;
}

// The 8-real parametrisation divides by |u01|^2 + |u02|^2 (zero for the unit link):
// WD_ERR_ARG unless it is at least 1e-6 on every link of the canonical copy.
wd_status check_recon8(wd_ctx *c, const char *who) {
    void *w;
    wd_status s = ws_get(c, "gauge_check", sizeof(unsigned), &w);
    if (s != WD_OK) return s;
    WD_CUDA(c, cudaMemsetAsync(w, 0x7f, sizeof(unsigned), c->stream));
    const size_t nl = (size_t)4 * c->g.V;
    k_gauge_min_offdiag<<<(int)std::min<size_t>((nl + 255) / 256, 4096), 256, 0, c->stream>>>(
        reinterpret_cast<const double2 *>(c->gauge_canon), nl, static_cast<unsigned *>(w));
    WD_CUDA(c, cudaGetLastError());
    c->launches += 1;
    unsigned bits = 0;
    WD_CUDA(c, cudaMemcpyAsync(&bits, w, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    float nmin;
    std::memcpy(&nmin, &bits, sizeof nmin);
    if (!(nmin >= 1e-6f))
        return fail(c, WD_ERR_ARG, std::string(who) + ": recon 8 needs |U01|^2 + |U02|^2 >= 1e-6 on every link "
                                   "(smallest: " + std::to_string(nmin) + "); use recon 12 or 18");
    return WD_OK;
}

Geom eo_geom(const wd_ctx *c, int parity) {
    Geom g = c->g;
    g.V = c->g.V / 2;
    g.Vs = (int)round_up((size_t)g.V, kSiteAlign);
    g.eo_parity = parity;
    return g;
}

template <int P, int RECON>
static void gauge_pack_eo(const double *canon, void *dst, const Geom &g, int Vhs, size_t dir, cudaStream_t st) {
    dim3 grid((g.V + 127) / 128, 4);
    k_gauge_pack_eo<P, RECON><<<grid, 128, 0, st>>>(reinterpret_cast<const double2 *>(canon), dst, g, Vhs, dir);
}

wd_status gauge_get_eo(wd_ctx *c, Prec p, const void **out, size_t *dir_bytes) {
    if (!c->has_gauge) return fail(c, WD_ERR_STATE, "no gauge field set (call wd_set_gauge first)");
    const int Vhs = eo_geom(c, 0).Vs;
    const size_t dir = round_up(link_dir_bytes(p, link_recon(c, p), Vhs), 256);
    if (!c->gauge_eo[p]) {
        void *d = nullptr;
        WD_CUDA(c, cudaMalloc(&d, 8 * dir));
        with_recon(link_recon(c, p), [&](auto rc) {
            constexpr int R = decltype(rc)::value;
            if (p == F64) gauge_pack_eo<F64, R>(c->gauge_canon, d, c->g, Vhs, dir, c->stream);
            else if (p == F32) gauge_pack_eo<F32, R>(c->gauge_canon, d, c->g, Vhs, dir, c->stream);
            else if (p == DF32) gauge_pack_eo<DF32, R>(c->gauge_canon, d, c->g, Vhs, dir, c->stream);
            else gauge_pack_eo<F16, R>(c->gauge_canon, d, c->g, Vhs, dir, c->stream);
        });
        WD_CUDA(c, cudaGetLastError());
        c->launches += 1;
        c->gauge_eo[p] = d;
    }
    *out = c->gauge_eo[p];
    *dir_bytes = dir;
    return WD_OK;
}

void *graph_get(wd_ctx *c, const std::string &key) {
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) return nullptr;
    c->graph_used[key] = ++c->graph_tick;
    return it->second;
}

void graph_put(wd_ctx *c, const std::string &key, void *exec, const std::vector<long long> &info) {
    while (c->graphs.size() >= kMaxGraphs) {
        auto lru = c->graph_used.begin();
        for (auto it = c->graph_used.begin(); it != c->graph_used.end(); ++it)
            if (it->second < lru->second) lru = it;
        cudaGraphExecDestroy((cudaGraphExec_t)c->graphs[lru->first]);
        c->graphs.erase(lru->first);
        c->graph_info.erase(lru->first);
        c->graph_used.erase(lru);
    }
    c->graphs[key] = exec;
    c->graph_info[key] = info;
    c->graph_used[key] = ++c->graph_tick;
}

void graph_clear(wd_ctx *c) {
    for (auto &g : c->graphs) cudaGraphExecDestroy((cudaGraphExec_t)g.second);
    c->graphs.clear();
    c->graph_info.clear();
    c->graph_used.clear();
}

DslashTiles cg_tiles_for(wd_ctx *c, Prec p, int nrhs, bool eo) {
    auto it = c->cg_tiles.find(p * 64 + nrhs + (eo ? kEoTileKey : 0));
    return it != c->cg_tiles.end() ? it->second : tiles_for(c, p, nrhs);
}

void ws_release(wd_ctx *c, const std::string &name) {
    auto it = c->ws.find(name);
    if (it == c->ws.end()) return;
    cudaStreamSynchronize(c->stream);
    cudaFree(it->second);
    c->ws.erase(it);
    c->ws_size.erase(name);
}

DslashTiles tiles_for(wd_ctx *c, Prec p, int nrhs) {
    auto it = c->tiles.find(p * 64 + nrhs);
    if (it != c->tiles.end()) return it->second;
    DslashTiles t;
    t.site_tile = 64;
    t.rhs_tile = nrhs < 4 ? nrhs : 4;
    return t;
}

}  // namespace wd

wd_ctx::~wd_ctx() {
    for (auto &g : graphs) cudaGraphExecDestroy((cudaGraphExec_t)g.second);
    for (auto &w : ws) cudaFree(w.second);
    for (int p = 0; p < kNumPrec; ++p) {
        if (gauge[p]) cudaFree(gauge[p]);
        if (gauge_eo[p]) cudaFree(gauge_eo[p]);
    }
    if (gauge_canon) cudaFree(gauge_canon);
    if (g.dbg) cudaFree(g.dbg);
    if (staged_err) cudaFree(staged_err);
}

static bool bad_prec(int p) { return p < 0 || p >= kNumPrec; }

extern "C" {

const char *wd_status_string(wd_status s) {
    switch (s) {
    case WD_OK: return "ok";
    case WD_ERR_ARG: return "invalid argument";
    case WD_ERR_CUDA: return "CUDA error";
    case WD_ERR_OOM: return "out of device memory";
    case WD_ERR_NOT_CONVERGED: return "not converged";
    case WD_ERR_BREAKDOWN: return "CG breakdown";
    case WD_ERR_NONFINITE: return "non-finite value";
    case WD_ERR_TIMEOUT: return "device-side wait timed out";
    case WD_ERR_STATE: return "call out of order";
    }
    return "unknown status";
}

const char *wd_last_error(const wd_ctx *c) { return c ? c->last_error.c_str() : "null context"; }

long long wd_kernel_launches(const wd_ctx *c) { return c ? c->launches : 0; }

wd_status wd_create(wd_ctx **out, const int dims[4], int antiperiodic_t, void *stream) {
    if (!out || !dims) return WD_ERR_ARG;
    *out = nullptr;
    long long V = 1;
    for (int mu = 0; mu < 4; ++mu) {
        if (dims[mu] < 2) return WD_ERR_ARG;
        V *= dims[mu];
    }
    if (V > (1ll << 30)) return WD_ERR_ARG;
    wd_ctx *c = new wd_ctx();
    for (int mu = 0; mu < 4; ++mu) c->g.L[mu] = dims[mu];
    c->g.V = (int)V;
    c->g.Vs = (int)round_up((size_t)V, kSiteAlign);
    c->g.stride[0] = 1;
    c->g.stride[1] = dims[0];
    c->g.stride[2] = dims[0] * dims[1];
    c->g.stride[3] = dims[0] * dims[1] * dims[2];
    c->g.antiperiodic = antiperiodic_t ? 1 : 0;
    c->g.eo_parity = -1;
    c->g.dbg = nullptr;
    c->g.split_t = 0;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess) {
        delete c;
        return WD_ERR_CUDA;
    }
#ifdef WD_DEBUG
    if (cudaMalloc(&c->g.dbg, sizeof(unsigned)) != cudaSuccess || cudaMemset(c->g.dbg, 0, sizeof(unsigned)) != cudaSuccess) {
        delete c;
        return WD_ERR_CUDA;
    }
#endif
    *out = c;
    return WD_OK;
}

wd_status wd_destroy(wd_ctx *c) {
    if (!c) return WD_ERR_ARG;
    cudaStreamSynchronize(c->stream);
    delete c;
    return WD_OK;
}

wd_status wd_set_stream(wd_ctx *c, void *stream) {
    if (!c) return WD_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return WD_OK;
}

wd_status wd_set_gauge(wd_ctx *c, const double *U, int on_device, int recon) {
    wd::NvtxRange nvtx_("wd_set_gauge");
    if (!c) return WD_ERR_ARG;
    if (!U) return fail(c, WD_ERR_ARG, "wd_set_gauge: null gauge pointer");
    if (recon != 18 && recon != 12 && recon != 8) return fail(c, WD_ERR_ARG, "wd_set_gauge: recon must be 18, 12 or 8");
    const size_t bytes = (size_t)4 * c->g.V * 9 * 16;
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int p = 0; p < kNumPrec; ++p) {
        if (c->gauge[p]) {
            cudaFree(c->gauge[p]);
            c->gauge[p] = nullptr;
        }
        if (c->gauge_eo[p]) {
            cudaFree(c->gauge_eo[p]);
            c->gauge_eo[p] = nullptr;
        }
    }
    if (!c->gauge_canon) WD_CUDA(c, cudaMalloc(&c->gauge_canon, bytes));
    WD_CUDA(c, cudaMemcpyAsync(c->gauge_canon, U, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                               c->stream));
    c->recon = recon;
    for (int p = 0; p < kNumPrec; ++p) c->recon_p[p] = 0;
    c->has_gauge = false;
    // graphs bake gauge pointers in
    graph_clear(c);
    if (recon == 8) {
        wd_status s = check_recon8(c, "wd_set_gauge");
        if (s != WD_OK) return s;
    }
    c->has_gauge = true;
    const void *d;
    wd_status s = gauge_get(c, F64, &d);
    if (s != WD_OK) return s;
    if (!on_device) WD_CUDA(c, cudaStreamSynchronize(c->stream));
    return WD_OK;
}

wd_status wd_debug_word(wd_ctx *c, unsigned *word, int *is_debug) {
    if (!c || !word) return WD_ERR_ARG;
    *word = 0;
#ifdef WD_DEBUG
    if (is_debug) *is_debug = 1;
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    WD_CUDA(c, cudaMemcpy(word, c->g.dbg, sizeof(unsigned), cudaMemcpyDeviceToHost));
    WD_CUDA(c, cudaMemset(c->g.dbg, 0, sizeof(unsigned)));
#else
    if (is_debug) *is_debug = 0;
#endif
    return WD_OK;
}

wd_status wd_set_link_compression(wd_ctx *c, wd_prec prec, int recon) {
    if (!c) return WD_ERR_ARG;
    if (bad_prec(prec)) return fail(c, WD_ERR_ARG, "wd_set_link_compression: bad precision");
    if (recon != 18 && recon != 12 && recon != 8)
        return fail(c, WD_ERR_ARG, "wd_set_link_compression: recon must be 18, 12 or 8");
    if (!c->has_gauge) return fail(c, WD_ERR_STATE, "no gauge field set (call wd_set_gauge first)");
    if (recon == link_recon(c, (Prec)prec)) return WD_OK;
    if (recon == 8) {
        wd_status s = check_recon8(c, "wd_set_link_compression");
        if (s != WD_OK) return s;
    }
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->gauge[prec]) cudaFree(c->gauge[prec]);
    if (c->gauge_eo[prec]) cudaFree(c->gauge_eo[prec]);
    c->gauge[prec] = c->gauge_eo[prec] = nullptr;
    c->recon_p[prec] = recon;
    graph_clear(c);
    return WD_OK;
}

size_t wd_field_bytes(const wd_ctx *c, wd_prec prec, int nrhs) {
    if (!c || bad_prec(prec) || nrhs < 1) return 0;
    return spinor_bytes((Prec)prec, c->g.Vs) * (size_t)nrhs;
}

static wd_status canon_stage(wd_ctx *c, const double *canon, int nrhs, int on_device, const double **dev) {
    if (on_device) {
        *dev = canon;
        return WD_OK;
    }
    void *buf;
    const size_t bytes = (size_t)nrhs * c->g.V * 12 * 16;
    wd_status s = ws_get(c, "canon_stage", bytes, &buf);
    if (s != WD_OK) return s;
    WD_CUDA(c, cudaMemcpyAsync(buf, canon, bytes, cudaMemcpyHostToDevice, c->stream));
    *dev = (const double *)buf;
    return WD_OK;
}

wd_status wd_pack(wd_ctx *c, const double *canon, int on_device, void *field, wd_prec prec, int nrhs) {
    wd::NvtxRange nvtx_("wd_pack");
    if (!c) return WD_ERR_ARG;
    if (!canon || !field || bad_prec(prec) || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, "wd_pack: bad argument");
    const double *src = nullptr;
    wd_status s = canon_stage(c, canon, nrhs, on_device, &src);
    if (s != WD_OK) return s;
    VecArgs v{};
    v.V = c->g.V; v.Vs = c->g.Vs; v.nrhs = nrhs;
    v.a = src;
    v.b = field; v.b_stride = spinor_bytes((Prec)prec, c->g.Vs);
    dim3 grid((c->g.V + 127) / 128, nrhs);
    if (prec == WD_F64) k_pack<F64><<<grid, 128, 0, c->stream>>>(v);
    else if (prec == WD_F32) k_pack<F32><<<grid, 128, 0, c->stream>>>(v);
    else if (prec == WD_DF32) k_pack<DF32><<<grid, 128, 0, c->stream>>>(v);
    else k_pack<F16><<<grid, 128, 0, c->stream>>>(v);
    WD_CUDA(c, cudaGetLastError());
    c->launches += 1;
    if (!on_device) WD_CUDA(c, cudaStreamSynchronize(c->stream));
    return WD_OK;
}

wd_status wd_unpack(wd_ctx *c, const void *field, wd_prec prec, int nrhs, double *canon, int on_device) {
    wd::NvtxRange nvtx_("wd_unpack");
    if (!c) return WD_ERR_ARG;
    if (!canon || !field || bad_prec(prec) || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, "wd_unpack: bad argument");
    const size_t bytes = (size_t)nrhs * c->g.V * 12 * 16;
    void *dst = canon;
    if (!on_device) {
        wd_status s = ws_get(c, "canon_stage", bytes, &dst);
        if (s != WD_OK) return s;
    }
    VecArgs v{};
    v.V = c->g.V; v.Vs = c->g.Vs; v.nrhs = nrhs;
    v.a = field; v.a_stride = spinor_bytes((Prec)prec, c->g.Vs);
    v.b = dst;
    dim3 grid((c->g.V + 127) / 128, nrhs);
    if (prec == WD_F64) k_unpack<F64><<<grid, 128, 0, c->stream>>>(v);
    else if (prec == WD_F32) k_unpack<F32><<<grid, 128, 0, c->stream>>>(v);
    else if (prec == WD_DF32) k_unpack<DF32><<<grid, 128, 0, c->stream>>>(v);
    else k_unpack<F16><<<grid, 128, 0, c->stream>>>(v);
    WD_CUDA(c, cudaGetLastError());
    c->launches += 1;
    if (!on_device) {
        WD_CUDA(c, cudaMemcpyAsync(canon, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
        WD_CUDA(c, cudaStreamSynchronize(c->stream));
    }
    return WD_OK;
}

static wd_status apply_common(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec, int nrhs,
                              bool dagger, const char *who) {
    if (!c) return WD_ERR_ARG;
    if (!in || !out || bad_prec(prec) || nrhs < 1 || nrhs > WD_MAX_RHS)
        return fail(c, WD_ERR_ARG, std::string(who) + ": bad argument");
    if (in == out) return fail(c, WD_ERR_ARG, std::string(who) + ": in and out must be distinct");
    if (!std::isfinite(kappa)) return fail(c, WD_ERR_ARG, std::string(who) + ": kappa not finite");
    if (c->split)
        return fail(c, WD_ERR_STATE, std::string(who) + ": a split sub-lattice needs its faces "
                                                      "(wd_apply_interior and wd_apply_faces)");
    const void *gauge;
    wd_status s = gauge_get(c, (Prec)prec, &gauge);
    if (s != WD_OK) return s;
    DslashArgs a{};
    a.g = c->g;
    a.in = in;
    a.in_stride = a.out_stride = spinor_bytes((Prec)prec, c->g.Vs);
    a.out = out;
    a.gauge = gauge;
    a.gauge_dir = gauge_dir_bytes(c, (Prec)prec);
    a.kappa = kappa;
    a.nrhs = nrhs;
    if (c->prefetch[prec] && prec == WD_F32) {
        DslashTiles t = tiles_for(c, F32, nrhs);
        t.rhs_per_thread = 1;
        WD_CUDA(c, launch_apply_prefetch(a, link_recon(c, F32), dagger, t, c->stream));
    } else if (c->staged_rows[prec]) {
        if ((s = staged_error_word(c)) != WD_OK) return s;
        WD_CUDA(c, launch_apply_staged(a, (Prec)prec, link_recon(c, (Prec)prec), dagger, c->staged_rows[prec],
                                       c->staged_stages[prec], c->staged_err, c->stream));
    } else {
        WD_CUDA(c, launch_apply(a, (Prec)prec, link_recon(c, (Prec)prec), dagger, tiles_for(c, (Prec)prec, nrhs),
                                c->stream));
    }
    c->launches += 1;
    return WD_OK;
}

wd_status wd_apply(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec, int nrhs) {
    wd::NvtxRange nvtx_("wd_apply");
    if (c) c->launches = 0;
    return apply_common(c, kappa, in, out, prec, nrhs, false, "wd_apply");
}

wd_status wd_apply_dagger(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec, int nrhs) {
    wd::NvtxRange nvtx_("wd_apply_dagger");
    if (c) c->launches = 0;
    return apply_common(c, kappa, in, out, prec, nrhs, true, "wd_apply_dagger");
}

wd_status wd_normal_apply(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec, int nrhs) {
    wd::NvtxRange nvtx_("wd_normal_apply");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    if (bad_prec(prec) || nrhs < 1 || nrhs > WD_MAX_RHS) return fail(c, WD_ERR_ARG, "wd_normal_apply: bad argument");
    if (c->split) return fail(c, WD_ERR_STATE, "wd_normal_apply: not on a split sub-lattice");
    void *tmp;
    wd_status s = ws_get(c, "normal_tmp", spinor_bytes((Prec)prec, c->g.Vs) * nrhs, &tmp);
    if (s != WD_OK) return s;
    s = apply_common(c, kappa, in, tmp, prec, nrhs, false, "wd_normal_apply");
    if (s != WD_OK) return s;
    return apply_common(c, kappa, tmp, out, prec, nrhs, true, "wd_normal_apply");
}

}  // extern "C"
