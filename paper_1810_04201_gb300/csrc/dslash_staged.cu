// Dslash with the neighbour spinors staged through shared memory by the bulk-copy
// (TMA) unit: the GPU form of the paper's on-chip buffers that feed the first stage of
// the stencil pipeline (sections 6.3-6.4), for the memory-bound FP32 and FP16 operators.
//
// A tile is R whole x-rows of one (z, t) plane: T = R Lx consecutive sites.  All its
// neighbours lie in seven contiguous site ranges of every field array:
//   0 the tile itself (x neighbours, and y neighbours inside it)
//   1, 2 the rows y0 - 1 and y0 + R of the same plane (periodic in y)
//   3, 4 the same sites one plane back / ahead in z, 5, 6 one slice back / ahead in t
// so a tile's neighbour spinors arrive with 7 x (component arrays) 1-D bulk copies,
// cp.async.bulk global -> shared, completed on an mbarrier that counts the bytes.  The
// kernel is persistent: each block walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...,
// with `stages` tiles in flight: while it computes tile k from shared memory, the copies
// of tiles k+1 .. k+stages-1 are on their way, and no register holds a byte of them.
// Links are read directly (each is used by two sites of different tiles).
//
// Thread 0 issues the copies and waits on the mbarriers; a block-wide barrier then hands
// the stage to all threads and, after the tile, hands it back.  Every wait is bounded:
// when one runs out the kernel sets the context's error word, waits (bounded) for the
// copies it still has in flight, and returns.  With WD_STAGED_STALL_TEST=1 in the
// environment, block 0 first waits on an mbarrier that nothing completes: the test of
// that path, which faults nothing.
#include <cstdlib>
#include "dslash.cuh"
#include "wd_host.h"

namespace wd {

struct StagedArgs {
    Geom g;
    const void *in;
    void *out;
    size_t stride;         // bytes between right-hand sides
    const void *gauge;
    size_t gauge_dir;
    double kappa;
    int nrhs;
    int rows;              // R
    int tiles;             // tiles per right-hand side: V / (R Lx)
    int stages;
    unsigned stage_bytes;
    unsigned *err;         // 1 when a wait ran out
    long long spin_limit;  // SM clock cycles a wait may take before it gives up
    int stall_test;        // block 0 first waits on a barrier that nothing completes
};

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bytes (a multiple of 16) from global src to shared dst (both 16-byte aligned)
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, unsigned long long *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}
// wait for phase `parity` of bar, for at most limit SM clock cycles (try_wait may suspend
// the thread for a time of its own choosing, so the bound is on the clock, not on calls)
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// layout of one stage: per component array j (FP32: 6 float4, FP16: 3 uint4), the seven
// ranges back to back (S sites in all); FP16 then the S per-site scales
struct TileRanges {
    int start[7], len[7], off[7];  // global first site, sites, position in the stage's S
    int S;
};

__device__ __forceinline__ TileRanges tile_ranges(const Geom &g, int rows, int n0) {
    const int Lx = g.L[0], Ly = g.L[1], Lz = g.L[2], Lt = g.L[3];
    const int T = rows * Lx, plane = Lx * Ly, vol3 = plane * Lz;
    const int y0 = (n0 / Lx) % Ly, z = (n0 / plane) % Lz, t = n0 / vol3;
    const int base_row = n0 - y0 * Lx;  // first site of the (z, t) plane
    TileRanges r;
    r.start[0] = n0;
    r.start[1] = base_row + ((y0 + Ly - 1) % Ly) * Lx;
    r.start[2] = base_row + ((y0 + rows) % Ly) * Lx;
    r.start[3] = n0 + (((z + Lz - 1) % Lz) - z) * plane;
    r.start[4] = n0 + (((z + 1) % Lz) - z) * plane;
    r.start[5] = n0 + (((t + Lt - 1) % Lt) - t) * vol3;
    r.start[6] = n0 + (((t + 1) % Lt) - t) * vol3;
    r.len[0] = T;
    r.len[1] = r.len[2] = Lx;
    r.len[3] = r.len[4] = r.len[5] = r.len[6] = T;
    int o = 0;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        r.off[k] = o;
        o += r.len[k];
    }
    r.S = o;
    return r;
}

template <int P> struct StageLayout;
template <> struct StageLayout<F32> {
    static constexpr int comps = 6, comp_bytes = 16, norm = 0;
};
template <> struct StageLayout<F16> {
    static constexpr int comps = 3, comp_bytes = 16, norm = 1;
};

// thread 0: the copies of tile `id` (right-hand side id / tiles) into stage buffer buf
template <int P>
__device__ __forceinline__ void issue_tile(const StagedArgs &a, int id, unsigned char *buf, unsigned long long *bar) {
    using L = StageLayout<P>;
    const int r = id / a.tiles, tile = id - r * a.tiles;
    const int n0 = tile * a.rows * a.g.L[0];
    const TileRanges tr = tile_ranges(a.g, a.rows, n0);
    const char *in = reinterpret_cast<const char *>(a.in) + a.stride * (size_t)r;
    mbar_expect_tx(bar, a.stage_bytes);
#pragma unroll
    for (int j = 0; j < L::comps; ++j)
#pragma unroll
        for (int k = 0; k < 7; ++k)
            bulk_copy(buf + ((size_t)j * tr.S + tr.off[k]) * L::comp_bytes,
                      in + ((size_t)j * a.g.Vs + tr.start[k]) * L::comp_bytes, (unsigned)tr.len[k] * L::comp_bytes, bar);
    if (L::norm) {
        const char *nrm = in + (size_t)L::comps * a.g.Vs * 16;
        unsigned char *dn = buf + (size_t)L::comps * tr.S * 16;
#pragma unroll
        for (int k = 0; k < 7; ++k)
            bulk_copy(dn + (size_t)tr.off[k] * 4, nrm + (size_t)tr.start[k] * 4, (unsigned)tr.len[k] * 4, bar);
    }
}

// both hops of direction MU for local site i of the tile (global site s, coordinate c)
template <int P, int RECON, bool DAG, int MU>
__device__ __forceinline__ void staged_dir(const StagedArgs &a, const TileRanges &tr, const unsigned char *buf, int i,
                                           int s, int c, C<float> (&acc)[12]) {
    constexpr int SF = DAG ? +1 : -1;
    const Geom &g = a.g;
    const int Lx = g.L[0], L = g.L[MU], st = g.stride[MU];
    const int x = i % Lx, ry = i / Lx;
    int fi, bi;  // stage positions of the forward and backward neighbour
    if (MU == 0) {
        fi = i - x + (x + 1 == Lx ? 0 : x + 1);
        bi = i - x + (x == 0 ? Lx - 1 : x - 1);
    } else if (MU == 1) {
        fi = ry + 1 < a.rows ? i + Lx : tr.off[2] + x;
        bi = ry > 0 ? i - Lx : tr.off[1] + x;
    } else if (MU == 2) {
        fi = tr.off[4] + i;
        bi = tr.off[3] + i;
    } else {
        fi = tr.off[6] + i;
        bi = tr.off[5] + i;
    }
    const char *gdir = reinterpret_cast<const char *>(a.gauge) + (size_t)MU * a.gauge_dir;
    const int sb = (c == 0) ? s + (L - 1) * st : s - st;  // global backward neighbour (its link)
    const bool ff = MU == 3 && g.antiperiodic && c == L - 1, fb = MU == 3 && g.antiperiodic && c == 0;
    if constexpr (P == F16) {
        hop_f16<RECON, false, MU, SF, false>(buf, tr.S, fi, gdir, s, ff, acc, g.Vs);
        hop_f16<RECON, true, MU, -SF, false>(buf, tr.S, bi, gdir, sb, fb, acc, g.Vs);
    } else {
        {
            C<float> p[12], h[6], w[6], u[9];
            SpinorIO<F32>::template load<false>(buf, tr.S, fi, p);
            project<MU, SF>(p, h);
            LinkIO<F32, RECON>::load(gdir, g.Vs, s, u);
            su3_mult<false>(u, h, w, ff);
            accumulate<MU, SF>(acc, w);
        }
        {
            C<float> p[12], h[6], w[6], u[9];
            SpinorIO<F32>::template load<false>(buf, tr.S, bi, p);
            project<MU, -SF>(p, h);
            LinkIO<F32, RECON>::load(gdir, g.Vs, sb, u);
            su3_mult<true>(u, h, w, fb);
            accumulate<MU, -SF>(acc, w);
        }
    }
}

template <int P, int RECON, bool DAG>
__global__ void __launch_bounds__(256) dslash_staged_kernel(StagedArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ unsigned long long full[4], never;
    __shared__ int abort_flag;
    const int T = a.rows * a.g.L[0];
    const int total = a.tiles * a.nrhs;
    if (threadIdx.x == 0) {
        for (int k = 0; k < a.stages; ++k) mbar_init(&full[k], 1);
        mbar_init(&never, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
        for (int k = 0; k < a.stages; ++k) {
            const int id = blockIdx.x + k * gridDim.x;
            if (id < total) issue_tile<P>(a, id, smem + (size_t)k * a.stage_bytes, &full[k]);
        }
    }
    __syncthreads();
    int k = 0;
    for (int id = blockIdx.x; id < total; id += gridDim.x, ++k) {
        const int stage = k % a.stages;
        const unsigned parity = (unsigned)(k / a.stages) & 1u;
        unsigned char *buf = smem + (size_t)stage * a.stage_bytes;
        const bool stalled = a.stall_test && k == 0 && blockIdx.x == 0;
        if (threadIdx.x == 0 && ((stalled && !mbar_wait(&never, 0, a.spin_limit)) ||
                                 !mbar_wait(&full[stage], parity, a.spin_limit))) {
            atomicExch(a.err, 1u);
            abort_flag = 1;
            // the copies still in flight land in this block's shared memory: let them finish
            for (int j = 0; j < a.stages; ++j) {
                const int kk = k + j;
                if (blockIdx.x + kk * gridDim.x < total)
                    mbar_wait(&full[kk % a.stages], (unsigned)(kk / a.stages) & 1u, a.spin_limit);
            }
        }
        __syncthreads();
        if (abort_flag) return;
        const int r = id / a.tiles, tile = id - r * a.tiles;
        const int n0 = tile * T;
        const TileRanges tr = tile_ranges(a.g, a.rows, n0);
        for (int i = threadIdx.x; i < T; i += blockDim.x) {
            const int s = n0 + i;
            const int x = i % a.g.L[0];
            const int y = (s / a.g.L[0]) % a.g.L[1];
            const int z = (s / a.g.stride[2]) % a.g.L[2];
            const int t = s / a.g.stride[3];
            C<float> acc[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) acc[c] = C<float>{0.f, 0.f};
            staged_dir<P, RECON, DAG, 0>(a, tr, buf, i, s, x, acc);
            staged_dir<P, RECON, DAG, 1>(a, tr, buf, i, s, y, acc);
            staged_dir<P, RECON, DAG, 2>(a, tr, buf, i, s, z, acc);
            staged_dir<P, RECON, DAG, 3>(a, tr, buf, i, s, t, acc);
            C<float> p[12];
            SpinorIO<P>::template load<false>(buf, tr.S, i, p);
            const float kap = (float)a.kappa;
#pragma unroll
            for (int c = 0; c < 12; ++c) p[c] = C<float>{p[c].re - kap * acc[c].re, p[c].im - kap * acc[c].im};
            SpinorIO<P>::store(reinterpret_cast<char *>(a.out) + a.stride * (size_t)r, a.g.Vs, s, p);
        }
        __syncthreads();  // every thread is done with this stage
        if (threadIdx.x == 0) {
            const int nid = id + a.stages * gridDim.x;
            if (nid < total) issue_tile<P>(a, nid, buf, &full[stage]);
        }
    }
}

// ---------------------------------------------------------------- per-thread prefetch
// The FP32 operator with each thread (one site, one right-hand side) copying the neighbour
// spinors of its next hops into a private ring of shared-memory slots with cp.async (16-byte
// global -> shared copies that hold no register), `kRing` - 1 hops ahead of the one it
// computes; the links are read directly.  Occupancy stays that of the direct kernel (288
// bytes of shared memory per thread), while every thread keeps two more hops of spinor
// loads in flight.  Slots are [slot][component][thread]: a warp's copies and reads of one
// component are 512 contiguous bytes, free of bank conflicts.
constexpr int kRing = 3;

__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// global site of hop h (mu = h / 2, forward for even h) of site s with coordinates xc
__device__ __forceinline__ int hop_site(const Geom &g, int s, const int (&xc)[4], int h) {
    const int mu = h >> 1, L = g.L[mu], st = g.stride[mu], c = xc[mu];
    if ((h & 1) == 0) return c == L - 1 ? s - (L - 1) * st : s + st;
    return c == 0 ? s + (L - 1) * st : s - st;
}

__device__ __forceinline__ void prefetch_spinor(float4 *ring, int slot, int nthr, int tid, const void *in, int Vs,
                                                int site) {
    const float4 *src = reinterpret_cast<const float4 *>(in) + site;
#pragma unroll
    for (int j = 0; j < 6; ++j) cp_async16(ring + ((size_t)slot * 6 + j) * nthr + tid, src + (size_t)j * Vs);
}

template <int RECON, bool DAG, int H>
__device__ __forceinline__ void pipe_hop(const DslashArgs &a, const float4 *ring, int nthr, int tid, int s,
                                         const int (&xc)[4], int nb, C<float> (&acc)[12]) {
    constexpr int MU = H >> 1;
    constexpr bool FWD = (H & 1) == 0;
    constexpr int SF = DAG ? +1 : -1;
    constexpr int S = FWD ? SF : -SF;
    const Geom &g = a.g;
    C<float> p[12], h[6], w[6], u[9];
    const float4 *slot = ring + (size_t)(H % kRing) * 6 * nthr + tid;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const float4 t = slot[(size_t)j * nthr];
        p[2 * j] = C<float>{t.x, t.y};
        p[2 * j + 1] = C<float>{t.z, t.w};
    }
    project<MU, S>(p, h);
    const char *gdir = reinterpret_cast<const char *>(a.gauge) + (size_t)MU * a.gauge_dir;
    LinkIO<F32, RECON>::load(gdir, g.Vs, FWD ? s : nb, u);
    const int c = xc[MU];
    const bool flip = MU == 3 && g.antiperiodic && (FWD ? c == g.L[3] - 1 : c == 0);
    su3_mult<!FWD>(u, h, w, flip);
    accumulate<MU, S>(acc, w);
}

template <int RECON, bool DAG>
__global__ void __launch_bounds__(256, 3) dslash_pipe_kernel(DslashArgs a) {
    extern __shared__ __align__(16) float4 ring[];
    const int nthr = blockDim.x * blockDim.y;
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    const int r = tile_y() * blockDim.y + threadIdx.y;
    if (r >= a.nrhs) return;  // no block-wide step follows
    const void *in = rhs_ptr<float>(a.in, a.in_stride, r);
    for (int s0 = tile_x() * blockDim.x; s0 < a.g.V; s0 += gridDim.x * blockDim.x) {
        const int s = s0 + threadIdx.x;
        if (s >= a.g.V) continue;
        int xc[4], rem = s;
        xc[0] = rem % a.g.L[0]; rem /= a.g.L[0];
        xc[1] = rem % a.g.L[1]; rem /= a.g.L[1];
        xc[2] = rem % a.g.L[2];
        xc[3] = rem / a.g.L[2];
        // the first kRing - 1 hops in flight, then one more per hop computed
#pragma unroll
        for (int hh = 0; hh < kRing - 1; ++hh) {
            prefetch_spinor(ring, hh % kRing, nthr, tid, in, a.g.Vs, hop_site(a.g, s, xc, hh));
            cp_async_commit();
        }
        C<float> acc[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) acc[c] = C<float>{0.f, 0.f};
#define WD_PIPE_STEP(H)                                                                        \
        if (H + kRing - 1 < 8)                                                                 \
            prefetch_spinor(ring, (H + kRing - 1) % kRing, nthr, tid, in, a.g.Vs,              \
                            hop_site(a.g, s, xc, (H + kRing - 1) & 7));                        \
        cp_async_commit();                                                                     \
        cp_async_wait<kRing - 1>();                                                            \
        pipe_hop<RECON, DAG, H>(a, ring, nthr, tid, s, xc, hop_site(a.g, s, xc, H), acc);
        WD_PIPE_STEP(0) WD_PIPE_STEP(1) WD_PIPE_STEP(2) WD_PIPE_STEP(3)
        WD_PIPE_STEP(4) WD_PIPE_STEP(5) WD_PIPE_STEP(6) WD_PIPE_STEP(7)
#undef WD_PIPE_STEP
        C<float> p[12];
        SpinorIO<F32>::load(a.xsrc ? rhs_ptr<float>(a.xsrc, a.xsrc_stride, r) : in, a.g.Vs, s, p);
        const float kap = (float)a.kappa;
#pragma unroll
        for (int c = 0; c < 12; ++c) p[c] = C<float>{p[c].re - kap * acc[c].re, p[c].im - kap * acc[c].im};
        SpinorIO<F32>::store(rhs_ptr<float>(a.out, a.out_stride, r), a.g.Vs, s, p);
    }
}

cudaError_t launch_apply_prefetch(const DslashArgs &a, int recon, bool dagger, DslashTiles t, cudaStream_t st) {
    const dim3 block(t.site_tile, t.rhs_tile);
    const dim3 grid(site_blocks<F32>(a.g.V, t.site_tile), (a.nrhs + t.rhs_tile - 1) / t.rhs_tile);
    const size_t smem = (size_t)kRing * 6 * 16 * block.x * block.y;
    return with_recon(recon, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        auto k = dagger ? dslash_pipe_kernel<R, true> : dslash_pipe_kernel<R, false>;
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k<<<grid, block, smem, st>>>(a);
        return cudaGetLastError();
    });
}

// bytes of one stage: (5 T + 2 Lx) sites of every component array (and the FP16 scales)
inline unsigned staged_stage_bytes(Prec p, const Geom &g, int rows) {
    const size_t S = (size_t)5 * rows * g.L[0] + 2 * (size_t)g.L[0];
    return (unsigned)(p == F32 ? S * 96 : S * 52);
}

// Whether tiles of `rows` rows suit this lattice and precision: whole rows that divide
// the y extent, at most 256 sites, all copies 16-byte multiples (FP16 scales: Lx a
// multiple of 4), one stage within the shared memory of a block.
bool staged_ok(Prec p, const Geom &g, int rows, int stages) {
    if (p != F32 && p != F16) return false;
    if (rows < 1 || stages < 2 || stages > 4 || g.eo_parity >= 0 || g.split_t) return false;
    if (g.L[1] % rows != 0 || rows * g.L[0] > 256) return false;
    if (p == F16 && g.L[0] % 4 != 0) return false;
    return (size_t)staged_stage_bytes(p, g, rows) * stages <= (size_t)227 * 1024;
}

template <int P, int RECON, bool DAG>
static cudaError_t go_staged(StagedArgs a, cudaStream_t st) {
    auto k = dslash_staged_kernel<P, RECON, DAG>;
    const size_t smem = (size_t)a.stage_bytes * a.stages;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int threads = ((a.rows * a.g.L[0] + 31) / 32) * 32;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int total = a.tiles * a.nrhs;
    const int grid = per_sm * sms < total ? per_sm * sms : total;
    k<<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_apply_staged(const DslashArgs &d, Prec p, int recon, bool dagger, int rows, int stages,
                                unsigned *err, cudaStream_t st) {
    StagedArgs a{};
    a.g = d.g;
    a.in = d.in;
    a.out = d.out;
    a.stride = d.in_stride;
    a.gauge = d.gauge;
    a.gauge_dir = d.gauge_dir;
    a.kappa = d.kappa;
    a.nrhs = d.nrhs;
    a.rows = rows;
    a.tiles = d.g.V / (rows * d.g.L[0]);
    a.stages = stages;
    a.stage_bytes = staged_stage_bytes(p, d.g, rows);
    a.err = err;
    const char *stall = getenv("WD_STAGED_STALL_TEST");
    a.stall_test = stall && stall[0] == '1';
    a.spin_limit = a.stall_test ? 200000000ll : 2000000000ll;  // about 0.1 s / 1 s at GB300 clocks
    return with_recon(recon, [&](auto rc) {
        constexpr int R = decltype(rc)::value;
        if (p == F32) return dagger ? go_staged<F32, R, true>(a, st) : go_staged<F32, R, false>(a, st);
        return dagger ? go_staged<F16, R, true>(a, st) : go_staged<F16, R, false>(a, st);
    });
}

}  // namespace wd

using namespace wd;

namespace wd {
wd_status staged_error_word(wd_ctx *c) {
    if (c->staged_err) return WD_OK;
    void *p = nullptr;
    WD_CUDA(c, cudaMalloc(&p, sizeof(unsigned)));
    c->staged_err = static_cast<unsigned *>(p);
    WD_CUDA(c, cudaMemsetAsync(c->staged_err, 0, sizeof(unsigned), c->stream));
    return WD_OK;
}
}  // namespace wd

extern "C" {

wd_status wd_set_staging(wd_ctx *c, wd_prec prec, int rows, int stages) {
    if (!c) return WD_ERR_ARG;
    if ((int)prec < 0 || (int)prec >= kNumPrec) return fail(c, WD_ERR_ARG, "wd_set_staging: bad precision");
    if (rows == 0) {
        c->staged_rows[prec] = 0;
        return WD_OK;
    }
    if (!staged_ok((Prec)prec, c->g, rows, stages))
        return fail(c, WD_ERR_ARG, "wd_set_staging: FP32 or FP16 only, rows dividing Ly with rows * Lx <= 256 (FP16: Lx "
                                   "a multiple of 4), 2 to 4 stages within 227 KB of shared memory, a full lattice");
    c->staged_rows[prec] = rows;
    c->staged_stages[prec] = stages;
    return WD_OK;
}

wd_status wd_set_prefetch(wd_ctx *c, wd_prec prec, int on) {
    if (!c) return WD_ERR_ARG;
    if ((int)prec < 0 || (int)prec >= kNumPrec) return fail(c, WD_ERR_ARG, "wd_set_prefetch: bad precision");
    if (on && prec != WD_F32) return fail(c, WD_ERR_ARG, "wd_set_prefetch: the FP32 operator only");
    if (on && (c->g.eo_parity >= 0 || c->g.split_t))
        return fail(c, WD_ERR_ARG, "wd_set_prefetch: full, unsplit lattices only");
    c->prefetch[prec] = on != 0;
    return WD_OK;
}

wd_status wd_staging_error(wd_ctx *c, unsigned *err) {
    if (!c || !err) return WD_ERR_ARG;
    *err = 0;
    wd_status s = staged_error_word(c);
    if (s != WD_OK) return s;
    WD_CUDA(c, cudaStreamSynchronize(c->stream));
    WD_CUDA(c, cudaMemcpy(err, c->staged_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    WD_CUDA(c, cudaMemset(c->staged_err, 0, sizeof(unsigned)));
    return WD_OK;
}

}  // extern "C"
