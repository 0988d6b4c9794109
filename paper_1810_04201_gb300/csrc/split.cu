// Domain decomposition along t (section 2.3: the lattice is divided into sub-lattices,
// one per process, which hold copies of their neighbours' boundary sites, and the global
// scalar products of CG are gathered from all of them; section 8: multi-node systems).
//
// Rank k of P owns the global t-slices [k Lt / P, (k + 1) Lt / P).  The Dslash of a
// sub-lattice is split in two launches:
//   interior  every hop whose neighbour is local (the dslash kernel with Geom::split_t:
//             the t hops that leave the sub-lattice are omitted), with the xpay epilogue;
//   faces     the two t hops that cross to the neighbouring sub-lattices, added to the
//             output at the first and the last local slice.
// What crosses is a projected half spinor (6 complex numbers per face site, 96 bytes in
// FP64, 48 in FP32), packed by the sender:
//   to_prev  (first slice)  h = psi_up + s psi_dn, with s the sign of the forward
//            projector 1 + s gamma_t (A_t = 1 in the gamma basis of Appendix A), for the
//            previous sub-lattice's forward hop, which multiplies it by its own U_t;
//   to_next  (last slice)   U_t(n)^dag (psi_up - s psi_dn), the whole backward hop but
//            the reconstruction, for the next sub-lattice: links never cross.
// The antiperiodic sign of the global boundary is applied by the receiver: by rank P - 1
// to what it receives from rank 0, and by rank 0 to what it receives from rank P - 1.
//
// wd_cg_solve_split runs CGNR over the sub-lattices one process holds (consecutive ranks
// on one device), exchanging faces between them by device copies and with the other
// processes through caller-supplied callbacks, and summing every scalar product over all
// sub-lattices before the host computes alpha, beta and the stopping test.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>
#include "dslash.cuh"
#include "wd_host.h"

using namespace wd;

namespace wd {

struct FaceArgs {
    Geom g;                        // the local sub-lattice
    int Vf, Vfs;                   // face sites (Lx Ly Lz) and the stride of a face array
    const void *in; size_t in_stride;
    void *out; size_t out_stride;
    const void *gauge; size_t gauge_dir;
    void *to_prev, *to_next;
    const void *from_prev, *from_next;
    size_t face_stride;            // bytes between right-hand sides of a face buffer
    double kappa;
    int nrhs;
    int flip_prev, flip_next;      // global boundary sign on what came from prev / next
};

inline int face_stride_sites(int Vf) { return (int)round_up((size_t)Vf, kSiteAlign); }
inline size_t face_buffer_bytes(Prec p, int Vf) { return (size_t)6 * face_stride_sites(Vf) * (p == F64 ? 16 : 8); }

// a half spinor of a face site: 6 arrays (spin 0, 1 x colour) of Vfs complex numbers
template <int P> struct FaceIO;
template <> struct FaceIO<F64> {
    static __device__ __forceinline__ void load(const void *b, int Vfs, int f, C<double> (&h)[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 t = __ldg(reinterpret_cast<const double2 *>(b) + (size_t)k * Vfs + f);
            h[k] = C<double>{t.x, t.y};
        }
    }
    static __device__ __forceinline__ void store(void *b, int Vfs, int f, const C<double> (&h)[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) reinterpret_cast<double2 *>(b)[(size_t)k * Vfs + f] = make_double2(h[k].re, h[k].im);
    }
};
template <> struct FaceIO<F32> {
    static __device__ __forceinline__ void load(const void *b, int Vfs, int f, C<float> (&h)[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float2 t = __ldg(reinterpret_cast<const float2 *>(b) + (size_t)k * Vfs + f);
            h[k] = C<float>{t.x, t.y};
        }
    }
    static __device__ __forceinline__ void store(void *b, int Vfs, int f, const C<float> (&h)[6]) {
#pragma unroll
        for (int k = 0; k < 6; ++k) reinterpret_cast<float2 *>(b)[(size_t)k * Vfs + f] = make_float2(h[k].re, h[k].im);
    }
};

template <class T> __device__ __forceinline__ T *at_rhs(T *p, size_t stride, int r) {
    return reinterpret_cast<T *>(reinterpret_cast<char *>(p) + stride * (size_t)r);
}
template <class T> __device__ __forceinline__ const T *at_rhs(const T *p, size_t stride, int r) {
    return reinterpret_cast<const T *>(reinterpret_cast<const char *>(p) + stride * (size_t)r);
}

// One thread per face site and right-hand side: both send faces.
template <int P, int RECON, bool DAG>
__global__ void k_face_pack(FaceArgs a) {
    using R = typename Real<P>::T;
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_t
    const int f = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (f >= a.Vf || r >= a.nrhs) return;
    const void *in = at_rhs(a.in, a.in_stride, r);
    C<R> p[12], h[6];
    SpinorIO<P>::load(in, a.g.Vs, f, p);
    project<3, SF>(p, h);
    FaceIO<P>::store(at_rhs(a.to_prev, a.face_stride, r), a.Vfs, f, h);
    const int n1 = f + (a.g.L[3] - 1) * a.Vf;
    SpinorIO<P>::load(in, a.g.Vs, n1, p);
    project<3, -SF>(p, h);
    C<R> u[9], w[6];
    LinkIO<P, RECON>::load(reinterpret_cast<const char *>(a.gauge) + 3 * a.gauge_dir, a.g.Vs, n1, u);
    su3_mult<true>(u, h, w, false);
    FaceIO<P>::store(at_rhs(a.to_next, a.face_stride, r), a.Vfs, f, w);
}

template <int P>
__device__ __forceinline__ void sub_kappa(void *out, int Vs, int n, double kappa, const C<typename Real<P>::T> (&acc)[12]) {
    using R = typename Real<P>::T;
    C<R> o[12];
    SpinorIO<P>::template load<false>(out, Vs, n, o);
    const R k = R(kappa);
#pragma unroll
    for (int c = 0; c < 12; ++c) o[c] = C<R>{o[c].re - k * acc[c].re, o[c].im - k * acc[c].im};
    SpinorIO<P>::store(out, Vs, n, o);
}

// One thread per face site and right-hand side: out -= kappa * (the hops across the faces).
template <int P, int RECON, bool DAG>
__global__ void k_face_apply(FaceArgs a) {
    using R = typename Real<P>::T;
    constexpr int SF = DAG ? +1 : -1;
    const int f = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
    if (f >= a.Vf || r >= a.nrhs) return;
    void *out = at_rhs(a.out, a.out_stride, r);
    const int Lt = a.g.L[3];
    const int n1 = f + (Lt - 1) * a.Vf;
    C<R> h[6], w[6], u[9], acc1[12], acc0[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) acc1[c] = acc0[c] = C<R>{R(0), R(0)};
    // last slice: forward hop onto the next sub-lattice's first slice
    FaceIO<P>::load(at_rhs(a.from_next, a.face_stride, r), a.Vfs, f, h);
    LinkIO<P, RECON>::load(reinterpret_cast<const char *>(a.gauge) + 3 * a.gauge_dir, a.g.Vs, n1, u);
    su3_mult<false>(u, h, w, a.flip_next != 0);
    accumulate<3, SF>(acc1, w);
    // first slice: backward hop from the previous sub-lattice's last slice (U^dag h came with it)
    FaceIO<P>::load(at_rhs(a.from_prev, a.face_stride, r), a.Vfs, f, w);
    if (a.flip_prev) {
#pragma unroll
        for (int k = 0; k < 6; ++k) w[k] = cneg(w[k]);
    }
    accumulate<3, -SF>(acc0, w);
    if (Lt == 1) {
#pragma unroll
        for (int c = 0; c < 12; ++c) acc0[c] = cadd(acc0[c], acc1[c]);
        sub_kappa<P>(out, a.g.Vs, f, a.kappa, acc0);
    } else {
        sub_kappa<P>(out, a.g.Vs, n1, a.kappa, acc1);
        sub_kappa<P>(out, a.g.Vs, f, a.kappa, acc0);
    }
}

// ---- FP64 vector kernels of the decomposed CG (sites < V of the 12 component arrays)
struct LinArgs {
    int V, Vs;
    double *out;
    const double *a, *b;
    double alpha, beta;
};
// out = alpha a + beta b
__global__ void k_lincomb(LinArgs l) {
    const long long n = 12ll * l.V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long comp = i / l.V, s = i - comp * l.V;
        const size_t k = 2 * ((size_t)comp * l.Vs + (size_t)s);
        const double2 x = *reinterpret_cast<const double2 *>(l.a + k);
        const double2 y = *reinterpret_cast<const double2 *>(l.b + k);
        *reinterpret_cast<double2 *>(l.out + k) = make_double2(fma(l.alpha, x.x, l.beta * y.x), fma(l.alpha, x.y, l.beta * y.y));
    }
}

constexpr int kDotBlocks = 256, kDotThreads = 256;
// partial[blockIdx.x] = sum over the block's sites of Re <a, b>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const double *a, const double *b, int V, int Vs, double *partial) {
    __shared__ double sm[kDotThreads];
    double acc = 0.0;
    const long long n = 12ll * V;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const long long comp = i / V, s = i - comp * V;
        const size_t k = 2 * ((size_t)comp * Vs + (size_t)s);
        acc = fma(a[k], b[k], fma(a[k + 1], b[k + 1], acc));
    }
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kDotThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sm[threadIdx.x] += sm[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sm[0];
}
// out[0] = the partials summed in block order (deterministic)
__global__ void k_sum_partials(const double *partial, int n, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += partial[i];
        out[0] = s;
    }
}

}  // namespace wd

namespace {

bool split_prec_ok(int p) { return p == WD_F64 || p == WD_F32; }

FaceArgs face_args(wd_ctx *c, Prec p, int nrhs) {
    FaceArgs a{};
    a.g = c->g;
    a.Vf = c->g.stride[3];
    a.Vfs = face_stride_sites(a.Vf);
    a.in_stride = a.out_stride = spinor_bytes(p, c->g.Vs);
    a.gauge_dir = gauge_dir_bytes(c, p);
    a.face_stride = face_buffer_bytes(p, a.Vf);
    a.nrhs = nrhs;
    a.flip_prev = c->split_antiperiodic && c->split_rank == 0;
    a.flip_next = c->split_antiperiodic && c->split_rank == c->split_nranks - 1;
    return a;
}

template <int P, int RECON>
cudaError_t launch_face(const FaceArgs &a, bool pack, bool dagger, cudaStream_t st) {
    const dim3 grid((a.Vf + 127) / 128, a.nrhs), block(128);
    if (pack) {
        if (dagger) k_face_pack<P, RECON, true><<<grid, block, 0, st>>>(a);
        else k_face_pack<P, RECON, false><<<grid, block, 0, st>>>(a);
    } else {
        if (dagger) k_face_apply<P, RECON, true><<<grid, block, 0, st>>>(a);
        else k_face_apply<P, RECON, false><<<grid, block, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_face_p(const FaceArgs &a, Prec p, int recon, bool pack, bool dagger, cudaStream_t st) {
    return with_recon(recon, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        return p == F64 ? launch_face<F64, R>(a, pack, dagger, st) : launch_face<F32, R>(a, pack, dagger, st);
    });
}

wd_status check_split(wd_ctx *c, int prec, int nrhs, const char *who) {
    if (!c->split) return fail(c, WD_ERR_STATE, std::string(who) + ": not a split sub-lattice (wd_create_split)");
    if (!split_prec_ok(prec)) return fail(c, WD_ERR_ARG, std::string(who) + ": split sub-lattices run in WD_F64 or WD_F32");
    if (nrhs < 1 || nrhs > WD_MAX_RHS) return fail(c, WD_ERR_ARG, std::string(who) + ": bad nrhs");
    return WD_OK;
}

// the three launches of one split Dslash on stream st (faces already exchanged when
// from_prev / from_next are read: the caller orders that)
wd_status interior(wd_ctx *c, double kappa, const void *in, void *out, Prec p, int nrhs, bool dagger, cudaStream_t st) {
    const void *gauge;
    wd_status s = gauge_get(c, p, &gauge);
    if (s != WD_OK) return s;
    DslashArgs a{};
    a.g = c->g;
    a.in = in;
    a.in_stride = a.out_stride = spinor_bytes(p, c->g.Vs);
    a.out = out;
    a.gauge = gauge;
    a.gauge_dir = gauge_dir_bytes(c, p);
    a.kappa = kappa;
    a.nrhs = nrhs;
    WD_CUDA(c, launch_apply(a, p, link_recon(c, p), dagger, tiles_for(c, p, nrhs), st));
    return WD_OK;
}

wd_status faces(wd_ctx *c, const void *in, void *to_prev, void *to_next, const void *from_prev, const void *from_next,
                void *out, double kappa, Prec p, int nrhs, bool pack, bool dagger, cudaStream_t st) {
    const void *gauge;
    wd_status s = gauge_get(c, p, &gauge);
    if (s != WD_OK) return s;
    FaceArgs a = face_args(c, p, nrhs);
    a.gauge = gauge;
    a.in = in;
    a.out = out;
    a.to_prev = to_prev;
    a.to_next = to_next;
    a.from_prev = from_prev;
    a.from_next = from_next;
    a.kappa = kappa;
    WD_CUDA(c, launch_face_p(a, p, link_recon(c, p), pack, dagger, st));
    return WD_OK;
}

}  // namespace

extern "C" {

wd_status wd_create_split(wd_ctx **out, const int global_dims[4], int nranks, int rank, int antiperiodic_t,
                          void *stream) {
    if (!out || !global_dims) return WD_ERR_ARG;
    *out = nullptr;
    if (nranks < 2 || rank < 0 || rank >= nranks) return WD_ERR_ARG;
    if (global_dims[3] < 2 || global_dims[3] % nranks != 0) return WD_ERR_ARG;
    const int lt = global_dims[3] / nranks;
    const int dims2[4] = {global_dims[0], global_dims[1], global_dims[2], 2};
    wd_ctx *c = nullptr;
    wd_status s = wd_create(&c, dims2, 0, stream);
    if (s != WD_OK) return s;
    const long long V = (long long)c->g.stride[3] * lt;
    if (V > (1ll << 30)) {
        wd_destroy(c);
        return WD_ERR_ARG;
    }
    c->g.L[3] = lt;
    c->g.V = (int)V;
    c->g.Vs = (int)round_up((size_t)V, kSiteAlign);
    c->g.antiperiodic = 0;
    c->g.split_t = 1;
    c->split = true;
    c->split_rank = rank;
    c->split_nranks = nranks;
    c->split_antiperiodic = antiperiodic_t ? 1 : 0;
    c->split_t0 = rank * lt;
    *out = c;
    return WD_OK;
}

size_t wd_face_bytes(const wd_ctx *c, wd_prec prec, int nrhs) {
    if (!c || !c->split || !split_prec_ok(prec) || nrhs < 1) return 0;
    return face_buffer_bytes((Prec)prec, c->g.stride[3]) * (size_t)nrhs;
}

wd_status wd_face_pack(wd_ctx *c, const void *in, void *to_prev, void *to_next, wd_prec prec, int nrhs, int dagger) {
    wd::NvtxRange nvtx_("wd_face_pack");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    wd_status s = check_split(c, prec, nrhs, "wd_face_pack");
    if (s != WD_OK) return s;
    if (!in || !to_prev || !to_next) return fail(c, WD_ERR_ARG, "wd_face_pack: null argument");
    s = faces(c, in, to_prev, to_next, nullptr, nullptr, nullptr, 0.0, (Prec)prec, nrhs, true, dagger != 0, c->stream);
    if (s == WD_OK) c->launches = 1;
    return s;
}

wd_status wd_apply_interior(wd_ctx *c, double kappa, const void *in, void *out, wd_prec prec, int nrhs, int dagger) {
    wd::NvtxRange nvtx_("wd_apply_interior");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    wd_status s = check_split(c, prec, nrhs, "wd_apply_interior");
    if (s != WD_OK) return s;
    if (!in || !out || in == out) return fail(c, WD_ERR_ARG, "wd_apply_interior: in and out must be distinct fields");
    if (!std::isfinite(kappa)) return fail(c, WD_ERR_ARG, "wd_apply_interior: kappa not finite");
    s = interior(c, kappa, in, out, (Prec)prec, nrhs, dagger != 0, c->stream);
    if (s == WD_OK) c->launches = 1;
    return s;
}

wd_status wd_apply_faces(wd_ctx *c, double kappa, const void *from_prev, const void *from_next, void *out, wd_prec prec,
                         int nrhs, int dagger) {
    wd::NvtxRange nvtx_("wd_apply_faces");
    if (!c) return WD_ERR_ARG;
    c->launches = 0;
    wd_status s = check_split(c, prec, nrhs, "wd_apply_faces");
    if (s != WD_OK) return s;
    if (!from_prev || !from_next || !out) return fail(c, WD_ERR_ARG, "wd_apply_faces: null argument");
    if (!std::isfinite(kappa)) return fail(c, WD_ERR_ARG, "wd_apply_faces: kappa not finite");
    s = faces(c, nullptr, nullptr, nullptr, from_prev, from_next, out, kappa, (Prec)prec, nrhs, false, dagger != 0,
              c->stream);
    if (s == WD_OK) c->launches = 1;
    return s;
}

}  // extern "C"

// ------------------------------------------------------------------ decomposed CG
namespace {

struct Sub {
    wd_ctx *c;
    void *b;  // only read
    void *x;
    void *db, *r, *p, *t, *q;
    void *to_prev, *to_next, *from_prev, *from_next;
    double *partial, *sum;
};

struct SplitCG {
    std::vector<Sub> s;
    cudaStream_t st = nullptr;   // the work stream (ctxs[0]'s)
    cudaStream_t xs = nullptr;   // the exchange stream (device copies beside the interior launch)
    cudaEvent_t packed = nullptr, exchanged = nullptr;
    const wd_comm *comm;
    bool all_local;
    size_t fbytes;
    int V, Vs;
    long long launches = 0;
    double *host = nullptr;  // pinned: one double per local sub-lattice
    wd_ctx *c0() const { return s[0].c; }
};

#define SPLIT_CUDA(call)                                                      \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return ::wd::cuda_fail(cg.c0(), e_, #call);    \
    } while (0)

// out_i = D in_i (or D^dag) on every local sub-lattice: faces packed, interior launched,
// faces exchanged (device copies on the exchange stream, the callback for other processes),
// then the face hops added.
wd_status split_apply(SplitCG &cg, void *Sub::*in, void *Sub::*out, double kappa, bool dagger) {
    const int n = (int)cg.s.size();
    wd_status st;
    for (Sub &u : cg.s)
        if ((st = faces(u.c, u.*in, u.to_prev, u.to_next, nullptr, nullptr, nullptr, 0.0, F64, 1, true, dagger, cg.st)) != WD_OK)
            return st;
    SPLIT_CUDA(cudaEventRecord(cg.packed, cg.st));
    SPLIT_CUDA(cudaStreamWaitEvent(cg.xs, cg.packed, 0));
    for (int i = 0; i + 1 < n; ++i) {
        SPLIT_CUDA(cudaMemcpyAsync(cg.s[i + 1].from_prev, cg.s[i].to_next, cg.fbytes, cudaMemcpyDeviceToDevice, cg.xs));
        SPLIT_CUDA(cudaMemcpyAsync(cg.s[i].from_next, cg.s[i + 1].to_prev, cg.fbytes, cudaMemcpyDeviceToDevice, cg.xs));
    }
    if (cg.all_local) {
        SPLIT_CUDA(cudaMemcpyAsync(cg.s[0].from_prev, cg.s[n - 1].to_next, cg.fbytes, cudaMemcpyDeviceToDevice, cg.xs));
        SPLIT_CUDA(cudaMemcpyAsync(cg.s[n - 1].from_next, cg.s[0].to_prev, cg.fbytes, cudaMemcpyDeviceToDevice, cg.xs));
    }
    SPLIT_CUDA(cudaEventRecord(cg.exchanged, cg.xs));
    for (Sub &u : cg.s)
        if ((st = interior(u.c, kappa, u.*in, u.*out, F64, 1, dagger, cg.st)) != WD_OK) return st;
    if (!cg.all_local) {
        if (cg.comm->exchange(cg.comm->user, cg.s[0].to_prev, cg.s[0].from_prev, cg.s[n - 1].to_next,
                              cg.s[n - 1].from_next, cg.fbytes, (void *)cg.st) != 0)
            return fail(cg.c0(), WD_ERR_CUDA, "wd_cg_solve_split: the exchange callback failed");
    }
    SPLIT_CUDA(cudaStreamWaitEvent(cg.st, cg.exchanged, 0));
    for (Sub &u : cg.s)
        if ((st = faces(u.c, nullptr, nullptr, nullptr, u.from_prev, u.from_next, u.*out, kappa, F64, 1, false, dagger,
                        cg.st)) != WD_OK)
            return st;
    cg.launches += 3ll * n;
    return WD_OK;
}

// Re <a, b> summed over every sub-lattice of the lattice
wd_status split_dot(SplitCG &cg, void *Sub::*a, void *Sub::*b, double *out) {
    const int n = (int)cg.s.size();
    for (Sub &u : cg.s) {
        k_dot_partial<<<kDotBlocks, kDotThreads, 0, cg.st>>>(static_cast<const double *>(u.*a),
                                                            static_cast<const double *>(u.*b), cg.V, cg.Vs, u.partial);
        k_sum_partials<<<1, 32, 0, cg.st>>>(u.partial, kDotBlocks, u.sum);
    }
    SPLIT_CUDA(cudaGetLastError());
    for (int i = 0; i < n; ++i) SPLIT_CUDA(cudaMemcpyAsync(cg.host + i, cg.s[i].sum, sizeof(double), cudaMemcpyDeviceToHost, cg.st));
    SPLIT_CUDA(cudaStreamSynchronize(cg.st));
    cg.launches += 2ll * n;
    double v = 0.0;
    for (int i = 0; i < n; ++i) v += cg.host[i];
    if (!cg.all_local && cg.comm->allreduce(cg.comm->user, &v, 1) != 0)
        return fail(cg.c0(), WD_ERR_CUDA, "wd_cg_solve_split: the allreduce callback failed");
    *out = v;
    return WD_OK;
}

// out_i = alpha a_i + beta b_i
wd_status split_lin(SplitCG &cg, void *Sub::*out, void *Sub::*a, void *Sub::*b, double alpha, double beta) {
    for (Sub &u : cg.s) {
        LinArgs l{cg.V, cg.Vs, static_cast<double *>(u.*out), static_cast<const double *>(u.*a),
                  static_cast<const double *>(u.*b), alpha, beta};
        k_lincomb<<<(int)std::min<long long>((12ll * cg.V + 255) / 256, 4096), 256, 0, cg.st>>>(l);
    }
    SPLIT_CUDA(cudaGetLastError());
    cg.launches += (long long)cg.s.size();
    return WD_OK;
}

}  // namespace

extern "C" wd_status wd_cg_solve_split(wd_ctx *const *ctxs, int n, double kappa, const void *const *b, void *const *x,
                                       const wd_cg_params *prm, wd_cg_result *res, const wd_comm *comm) {
    wd::NvtxRange nvtx_("wd_cg_solve_split");
    if (!ctxs || n < 1 || !ctxs[0]) return WD_ERR_ARG;
    wd_ctx *c0 = ctxs[0];
    c0->launches = 0;
    if (!b || !x || !prm || !res) return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: null argument");
    if (!(prm->tol > 0) || !std::isfinite(kappa)) return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: bad tol or kappa");
    if (prm->inner_prec != WD_F64 || prm->nrhs > 1 || prm->block || prm->normal_eq ||
        prm->precondition != WD_PRECOND_NONE || prm->stop_rule != WD_STOP_NORMAL)
        return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: plain FP64 CGNR with one right-hand side only");
    for (int i = 0; i < n; ++i) {
        wd_ctx *c = ctxs[i];
        if (!c || !c->split || !b[i] || !x[i] || b[i] == x[i])
            return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: every entry needs a split sub-lattice and distinct fields");
        if (c->split_nranks != c0->split_nranks || c->split_rank != c0->split_rank + i || c->device != c0->device ||
            c->split_antiperiodic != c0->split_antiperiodic || c->g.V != c0->g.V ||
            std::memcmp(c->g.L, c0->g.L, sizeof c->g.L) != 0)
            return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: the sub-lattices must be consecutive ranks of one lattice "
                                        "on one device");
        if (!c->has_gauge) return fail(c0, WD_ERR_STATE, "wd_cg_solve_split: no gauge field set");
    }
    const bool all_local = n == c0->split_nranks;
    if (!all_local && (!comm || !comm->exchange || !comm->allreduce))
        return fail(c0, WD_ERR_ARG, "wd_cg_solve_split: sub-lattices held by other processes need comm callbacks");

    SplitCG cg;
    cg.st = c0->stream;
    cg.comm = comm;
    cg.all_local = all_local;
    cg.fbytes = face_buffer_bytes(F64, c0->g.stride[3]);
    cg.V = c0->g.V;
    cg.Vs = c0->g.Vs;
    const size_t sbytes = spinor_bytes(F64, cg.Vs);
    wd_status s;
    for (int i = 0; i < n; ++i) {
        wd_ctx *c = ctxs[i];
        Sub u{};
        u.c = c;
        u.b = const_cast<void *>(b[i]);
        u.x = x[i];
        const char *names[5] = {"split_db", "split_r", "split_p", "split_t", "split_q"};
        void **ptrs[5] = {&u.db, &u.r, &u.p, &u.t, &u.q};
        for (int k = 0; k < 5; ++k)
            if ((s = ws_get(c, names[k], sbytes, ptrs[k])) != WD_OK) return s;
        const char *fn[4] = {"split_to_prev", "split_to_next", "split_from_prev", "split_from_next"};
        void **fp[4] = {&u.to_prev, &u.to_next, &u.from_prev, &u.from_next};
        for (int k = 0; k < 4; ++k)
            if ((s = ws_get(c, fn[k], cg.fbytes, fp[k])) != WD_OK) return s;
        void *tmp;
        if ((s = ws_get(c, "split_partial", (kDotBlocks + 8) * sizeof(double), &tmp)) != WD_OK) return s;
        u.partial = static_cast<double *>(tmp);
        u.sum = u.partial + kDotBlocks;
        const void *g;
        if ((s = gauge_get(c, F64, &g)) != WD_OK) return s;
        cg.s.push_back(u);
    }
    struct Guard {
        SplitCG &cg;
        ~Guard() {
            if (cg.xs) cudaStreamDestroy(cg.xs);
            if (cg.packed) cudaEventDestroy(cg.packed);
            if (cg.exchanged) cudaEventDestroy(cg.exchanged);
            if (cg.host) cudaFreeHost(cg.host);
        }
    } guard{cg};
    SPLIT_CUDA(cudaStreamCreateWithFlags(&cg.xs, cudaStreamNonBlocking));
    SPLIT_CUDA(cudaEventCreateWithFlags(&cg.packed, cudaEventDisableTiming));
    SPLIT_CUDA(cudaEventCreateWithFlags(&cg.exchanged, cudaEventDisableTiming));
    SPLIT_CUDA(cudaMallocHost(&cg.host, sizeof(double) * n));

    const auto t_start = std::chrono::steady_clock::now();
    // CGNR on D^dag D x = D^dag b (section 2.2), every scalar product summed over all sub-lattices
    double nb2, ndb2, nx2, rho, pAp, rho1;
    if ((s = split_dot(cg, &Sub::b, &Sub::b, &nb2)) != WD_OK) return s;
    if ((s = split_apply(cg, &Sub::b, &Sub::db, kappa, true)) != WD_OK) return s;
    if ((s = split_dot(cg, &Sub::db, &Sub::db, &ndb2)) != WD_OK) return s;
    if ((s = split_dot(cg, &Sub::x, &Sub::x, &nx2)) != WD_OK) return s;
    if (nx2 > 0 || !std::isfinite(nx2)) {
        // r = D^dag b - D^dag D x0
        if ((s = split_apply(cg, &Sub::x, &Sub::t, kappa, false)) != WD_OK) return s;
        if ((s = split_apply(cg, &Sub::t, &Sub::q, kappa, true)) != WD_OK) return s;
        if ((s = split_lin(cg, &Sub::r, &Sub::db, &Sub::q, 1.0, -1.0)) != WD_OK) return s;
    } else {
        if ((s = split_lin(cg, &Sub::r, &Sub::db, &Sub::db, 1.0, 0.0)) != WD_OK) return s;
    }
    if ((s = split_lin(cg, &Sub::p, &Sub::r, &Sub::r, 1.0, 0.0)) != WD_OK) return s;
    if ((s = split_dot(cg, &Sub::r, &Sub::r, &rho)) != WD_OK) return s;
    const double tol2 = prm->tol * prm->tol * ndb2;
    int status = WD_ERR_NOT_CONVERGED, k = 0;
    if (!std::isfinite(rho)) status = WD_ERR_NONFINITE;
    else if (rho <= tol2) status = WD_OK;
    while (status == WD_ERR_NOT_CONVERGED && k < prm->max_iter) {
        if ((s = split_apply(cg, &Sub::p, &Sub::t, kappa, false)) != WD_OK) return s;
        if ((s = split_dot(cg, &Sub::t, &Sub::t, &pAp)) != WD_OK) return s;
        if (!std::isfinite(pAp)) { status = WD_ERR_NONFINITE; break; }
        if (!(pAp > 0)) { status = WD_ERR_BREAKDOWN; break; }
        const double alpha = rho / pAp;
        if ((s = split_apply(cg, &Sub::t, &Sub::q, kappa, true)) != WD_OK) return s;
        if ((s = split_lin(cg, &Sub::x, &Sub::x, &Sub::p, 1.0, alpha)) != WD_OK) return s;
        if ((s = split_lin(cg, &Sub::r, &Sub::r, &Sub::q, 1.0, -alpha)) != WD_OK) return s;
        if ((s = split_dot(cg, &Sub::r, &Sub::r, &rho1)) != WD_OK) return s;
        ++k;
        if (!std::isfinite(rho1)) { status = WD_ERR_NONFINITE; break; }
        if (rho1 <= tol2) status = WD_OK;
        if ((s = split_lin(cg, &Sub::p, &Sub::r, &Sub::p, 1.0, rho1 / rho)) != WD_OK) return s;
        rho = rho1;
    }
    // the residuals of the returned x, recomputed in FP64: e = b - D x, D^dag e
    double ne2, nde2;
    if ((s = split_apply(cg, &Sub::x, &Sub::t, kappa, false)) != WD_OK) return s;
    if ((s = split_lin(cg, &Sub::t, &Sub::b, &Sub::t, 1.0, -1.0)) != WD_OK) return s;
    if ((s = split_dot(cg, &Sub::t, &Sub::t, &ne2)) != WD_OK) return s;
    if ((s = split_apply(cg, &Sub::t, &Sub::q, kappa, true)) != WD_OK) return s;
    if ((s = split_dot(cg, &Sub::q, &Sub::q, &nde2)) != WD_OK) return s;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
    res->iters = k;
    res->reliable_updates = 0;
    res->inner_corrections = 0;
    res->true_rel_resid = ndb2 > 0 ? std::sqrt(nde2 / ndb2) : std::sqrt(nde2);
    res->true_rel_resid_b = nb2 > 0 ? std::sqrt(ne2 / nb2) : std::sqrt(ne2);
    res->seconds = secs;
    res->status = status;
    c0->launches = cg.launches;
    if (status != WD_OK) c0->last_error = std::string("wd_cg_solve_split: ") + wd_status_string((wd_status)status);
    return (wd_status)status;
}
