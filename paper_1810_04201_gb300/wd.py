"""ctypes binding of libwd (include/wd.h): argument marshalling only.

Every step of the computation runs in the library's CUDA kernels; this module
converts Python arguments into C arguments, uses torch for device memory and
for the current CUDA stream, and turns status codes into exceptions.  There is
no CPU fallback: creating a Lattice (or calling cg_batched) loads
``_build/libwd.so`` and raises if it is missing.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libwd.so")

WD_F64, WD_F32, WD_F16, WD_DF32 = 0, 1, 2, 3
PRECS = {"f64": WD_F64, "f32": WD_F32, "f16": WD_F16, "df32": WD_DF32}
STATUS = {0: "WD_OK", 1: "WD_ERR_ARG", 2: "WD_ERR_CUDA", 3: "WD_ERR_OOM", 4: "WD_ERR_NOT_CONVERGED",
          5: "WD_ERR_BREAKDOWN", 6: "WD_ERR_NONFINITE", 7: "WD_ERR_TIMEOUT", 8: "WD_ERR_STATE"}
MAX_RHS = 16


class CGParams(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("inner_prec", ctypes.c_int),
                ("delta", ctypes.c_double), ("nrhs", ctypes.c_int), ("block", ctypes.c_int),
                ("rhs_tile", ctypes.c_int), ("normal_eq", ctypes.c_int), ("precondition", ctypes.c_int),
                ("stop_rule", ctypes.c_int)]


class CGResult(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("true_rel_resid", ctypes.c_double),
                ("true_rel_resid_b", ctypes.c_double), ("seconds", ctypes.c_double), ("status", ctypes.c_int),
                ("inner_corrections", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXCHANGE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int)


class Comm(ctypes.Structure):
    """wd_comm: the callbacks through which a split solve reaches other processes."""
    _fields_ = [("user", ctypes.c_void_p), ("exchange", EXCHANGE_FN), ("allreduce", ALLREDUCE_FN)]


class WDError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libwd.so and declare the C signatures (raises if the library is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libwd.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    PP = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "wd_create": ([ctypes.POINTER(P), ctypes.POINTER(I), I, P], I),
        "wd_destroy": ([P], I),
        "wd_set_stream": ([P, P], I),
        "wd_set_gauge": ([P, P, I, I], I),
        "wd_set_link_compression": ([P, I, I], I),
        "wd_debug_word": ([P, ctypes.POINTER(ctypes.c_uint), ctypes.POINTER(I)], I),
        "wd_field_bytes": ([P, I, I], S),
        "wd_pack": ([P, P, I, P, I, I], I),
        "wd_unpack": ([P, P, I, I, P, I], I),
        "wd_apply": ([P, D, P, P, I, I], I),
        "wd_apply_dagger": ([P, D, P, P, I, I], I),
        "wd_normal_apply": ([P, D, P, P, I, I], I),
        "wd_normal_apply_noalloc": ([P, D, P, P, I, I], I),
        "wd_apply_schur": ([P, D, P, P, I], I),
        "wd_cg_solve": ([P, D, P, P, ctypes.POINTER(CGParams), ctypes.POINTER(CGResult)], I),
        "wd_cg_solve_canonical": ([P, D, P, P, I, ctypes.POINTER(CGParams), ctypes.POINTER(CGResult)], I),
        "wd_cg_solve_batched": ([PP, ctypes.POINTER(D), PP, PP, I, ctypes.POINTER(CGParams),
                                 ctypes.POINTER(CGResult)], I),
        "wd_autotune": ([P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "wd_set_tiles": ([P, I, I, I, I], I),
        "wd_autotune_cg": ([P, I, I, ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "wd_set_staging": ([P, I, I, I], I),
        "wd_get_tiles": ([P, I, I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)], I),
        "wd_set_rhs_per_thread": ([P, I, I, I], I),
        "wd_staging_error": ([P, ctypes.POINTER(ctypes.c_uint)], I),
        "wd_set_prefetch": ([P, I, I], I),
        "wd_kernel_launches": ([P], ctypes.c_longlong),
        "wd_measure_fp64_rate": ([ctypes.POINTER(D)], I),
        "wd_create_split": ([ctypes.POINTER(P), ctypes.POINTER(I), I, I, I, P], I),
        "wd_face_bytes": ([P, I, I], S),
        "wd_face_pack": ([P, P, P, P, I, I, I], I),
        "wd_apply_interior": ([P, D, P, P, I, I, I], I),
        "wd_apply_faces": ([P, D, P, P, P, I, I, I], I),
        "wd_cg_solve_split": ([PP, I, D, PP, PP, ctypes.POINTER(CGParams), ctypes.POINTER(CGResult),
                               ctypes.POINTER(Comm)], I),
        "wd_status_string": ([I], ctypes.c_char_p),
        "wd_last_error": ([P], ctypes.c_char_p),
    }
    for name, (args, res) in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Lattice:
    """One lattice (dims, boundary, gauge field) bound to a library context.

    Fields are torch uint8 device tensors of ``field_bytes(prec, nrhs)`` bytes in the
    library's layout; canonical spinors are complex128 arrays (nrhs, V, 4, 3) and
    canonical links complex128 (4, V, 3, 3).
    """

    def __init__(self, dims, antiperiodic_t=True, stream=None):
        self.lib = load_library()
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.ctx = ctypes.c_void_p()
        self.recon = 18
        self.recon_p = {}
        d = (ctypes.c_int * 4)(*self.dims)
        st = self.lib.wd_create(ctypes.byref(self.ctx), d, int(bool(antiperiodic_t)), _stream_ptr(stream))
        if st != 0:
            raise WDError(st, "wd_create failed")

    # ------------------------------------------------------------------ plumbing
    def _check(self, st, what):
        if st != 0:
            msg = self.lib.wd_last_error(self.ctx).decode()
            raise WDError(st, f"{what}: {msg}")

    def close(self):
        if self.ctx:
            self.lib.wd_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream=None):
        self._check(self.lib.wd_set_stream(self.ctx, _stream_ptr(stream)), "wd_set_stream")

    @property
    def launches(self) -> int:
        return int(self.lib.wd_kernel_launches(self.ctx))

    def field_bytes(self, prec=WD_F64, nrhs=1) -> int:
        return int(self.lib.wd_field_bytes(self.ctx, prec, nrhs))

    def new_field(self, prec=WD_F64, nrhs=1, zero=True):
        n = self.field_bytes(prec, nrhs)
        return torch.zeros(n, dtype=torch.uint8, device="cuda") if zero else \
            torch.empty(n, dtype=torch.uint8, device="cuda")

    # ------------------------------------------------------------------ gauge / layout
    def set_gauge(self, U, recon=18):
        """U: canonical links, numpy complex128 (4, V, 3, 3) or a complex128 cuda tensor."""
        if isinstance(U, torch.Tensor) and U.is_cuda:
            t = U.contiguous()
            self._check(self.lib.wd_set_gauge(self.ctx, ctypes.c_void_p(t.data_ptr()), 1, recon), "wd_set_gauge")
            torch.cuda.current_stream().synchronize()
        else:
            a = np.ascontiguousarray(U, dtype=np.complex128)
            assert a.shape == (4, self.V, 3, 3)
            self._check(self.lib.wd_set_gauge(self.ctx, a.ctypes.data_as(ctypes.c_void_p), 0, recon),
                        "wd_set_gauge")
        self.recon = int(recon)
        self.recon_p = {}

    def debug_word(self):
        """(first out-of-range index record or 0, debug build?) -- see wd_debug_word."""
        w, d = ctypes.c_uint(), ctypes.c_int()
        self._check(self.lib.wd_debug_word(self.ctx, ctypes.byref(w), ctypes.byref(d)), "wd_debug_word")
        return w.value, bool(d.value)

    def set_link_compression(self, prec, recon):
        """Store the links of one precision with recon 18, 12 or 8 (until the next set_gauge)."""
        self._check(self.lib.wd_set_link_compression(self.ctx, prec, recon), "wd_set_link_compression")
        self.recon_p[int(prec)] = int(recon)

    def pack(self, psi, prec=WD_F64, out=None):
        """Canonical spinor(s) (numpy or cuda complex128, (V,4,3) or (nrhs,V,4,3)) -> field."""
        nrhs = 1 if (psi.ndim == 3) else psi.shape[0]
        if out is None:
            out = self.new_field(prec, nrhs, zero=False)
        if isinstance(psi, torch.Tensor) and psi.is_cuda:
            t = psi.contiguous()
            st = self.lib.wd_pack(self.ctx, ctypes.c_void_p(t.data_ptr()), 1, ctypes.c_void_p(out.data_ptr()), prec,
                                  nrhs)
        else:
            a = np.ascontiguousarray(psi, dtype=np.complex128)
            st = self.lib.wd_pack(self.ctx, a.ctypes.data_as(ctypes.c_void_p), 0, ctypes.c_void_p(out.data_ptr()),
                                  prec, nrhs)
        self._check(st, "wd_pack")
        return out

    def unpack(self, field, prec=WD_F64, nrhs=1, squeeze=True):
        """Field -> canonical numpy complex128 (nrhs, V, 4, 3) (squeezed for nrhs = 1)."""
        out = np.empty((nrhs, self.V, 4, 3), dtype=np.complex128)
        self._check(self.lib.wd_unpack(self.ctx, ctypes.c_void_p(field.data_ptr()), prec, nrhs,
                                       out.ctypes.data_as(ctypes.c_void_p), 0), "wd_unpack")
        return out[0] if (squeeze and nrhs == 1) else out

    # ------------------------------------------------------------------ operators
    def apply(self, kappa, src, dst, prec=WD_F64, nrhs=1, dagger=False):
        fn = self.lib.wd_apply_dagger if dagger else self.lib.wd_apply
        self._check(fn(self.ctx, float(kappa), ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                       prec, nrhs), "wd_apply_dagger" if dagger else "wd_apply")
        return dst

    def normal_apply(self, kappa, src, dst, prec=WD_F64, nrhs=1):
        self._check(self.lib.wd_normal_apply(self.ctx, float(kappa), ctypes.c_void_p(src.data_ptr()),
                                             ctypes.c_void_p(dst.data_ptr()), prec, nrhs), "wd_normal_apply")
        return dst

    def apply_schur(self, kappa, src, dst, dagger=False):
        """Even sites of dst = (1 - kappa^2 H_eo H_oe) src_e (or its adjoint), odd sites = 0 (FP64)."""
        self._check(self.lib.wd_apply_schur(self.ctx, float(kappa), ctypes.c_void_p(src.data_ptr()),
                                            ctypes.c_void_p(dst.data_ptr()), int(bool(dagger))), "wd_apply_schur")
        return dst

    def normal_apply_noalloc(self, kappa, src, dst, prec=WD_F64, nrhs=1):
        """D^dag D through the entry point that allocates no device memory (fixed 16 MiB scratch)."""
        self._check(self.lib.wd_normal_apply_noalloc(self.ctx, float(kappa), ctypes.c_void_p(src.data_ptr()),
                                                     ctypes.c_void_p(dst.data_ptr()), prec, nrhs),
                    "wd_normal_apply_noalloc")
        return dst

    # ------------------------------------------------------------------ solvers
    @staticmethod
    def params(tol=1e-10, max_iter=10000, inner=WD_F64, delta=0.0, nrhs=1, block=0, rhs_tile=0, normal_eq=0,
               precondition=0, stop_rule=0):
        return CGParams(tol, max_iter, inner, delta, nrhs, block, rhs_tile, normal_eq, precondition, stop_rule)

    def cg(self, kappa, b, x, tol=1e-10, max_iter=10000, inner=WD_F64, delta=0.0, nrhs=1, block=0,
           raise_on_fail=True, normal_eq=0, precondition=0, stop_rule=0):
        """Solve D x = b on device fields (x holds the start vector). Returns the per-RHS results.
        normal_eq=1 selects CGNE (D D^dag y = b, x = D^dag y); precondition=1 even-odd;
        stop_rule=1 applies tol to |b - D x| / |b| instead of the normal residual."""
        p = self.params(tol, max_iter, inner, delta, nrhs, block, 0, normal_eq, precondition, stop_rule)
        res = (CGResult * nrhs)()
        st = self.lib.wd_cg_solve(self.ctx, float(kappa), ctypes.c_void_p(b.data_ptr()),
                                  ctypes.c_void_p(x.data_ptr()), ctypes.byref(p), res)
        if raise_on_fail:
            self._check(st, "wd_cg_solve")
        return [r.as_dict() for r in res], st

    def cg_canonical(self, kappa, b, x, tol=1e-10, max_iter=10000, inner=WD_F64, delta=0.0, nrhs=1,
                     raise_on_fail=True, precondition=0, stop_rule=0):
        """End-to-end solve on canonical host arrays (numpy complex128, pinned torch CPU tensors
        allowed) or device tensors; x is overwritten with the solution."""
        p = self.params(tol, max_iter, inner, delta, nrhs, 0, 0, 0, precondition, stop_rule)
        res = (CGResult * nrhs)()
        if isinstance(b, torch.Tensor):
            on_dev = int(b.is_cuda)
            bp, xp = ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr())
        else:
            on_dev = 0
            bp, xp = b.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p)
        st = self.lib.wd_cg_solve_canonical(self.ctx, float(kappa), bp, xp, on_dev, ctypes.byref(p), res)
        if raise_on_fail:
            self._check(st, "wd_cg_solve_canonical")
        return [r.as_dict() for r in res], st

    def autotune(self, prec=WD_F64, nrhs=1, cache=None):
        """Time the launch shapes (wd_autotune) and keep the fastest.  With a cache path
        (or WD_TILE_CACHE set), a shape found before for the same lattice, precision, link
        compression, nrhs and device is reused without timing, and new results are added."""
        path = cache or os.environ.get("WD_TILE_CACHE")
        key = None
        if path:
            key = tile_cache_key(self.dims, prec, self.recon_p.get(int(prec), self.recon), nrhs, device_tag())
            hit = TileCache(path).get(key)
            if hit is not None:
                self.set_tiles(prec, nrhs, *hit)
                return hit
        st_, rt = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wd_autotune(self.ctx, prec, nrhs, ctypes.byref(st_), ctypes.byref(rt)), "wd_autotune")
        if path:
            TileCache(path).put(key, (st_.value, rt.value))
        return st_.value, rt.value

    def autotune_cg(self, prec=WD_F64, nrhs=1):
        """Tune the launch shape of the solver's fused kernels for inner precision prec
        (wd_autotune_cg); returns (site_tile, rhs_tile)."""
        st_, rt = ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wd_autotune_cg(self.ctx, prec, nrhs, ctypes.byref(st_), ctypes.byref(rt)),
                    "wd_autotune_cg")
        return st_.value, rt.value

    def tiles(self, prec=WD_F64, nrhs=1):
        """(site_tile, rhs_tile, rhs_per_thread) the plain operators of (prec, nrhs) use."""
        a, b, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.wd_get_tiles(self.ctx, prec, nrhs, ctypes.byref(a), ctypes.byref(b), ctypes.byref(k)),
                    "wd_get_tiles")
        return a.value, b.value, k.value

    def set_rhs_per_thread(self, prec, nrhs, k):
        self._check(self.lib.wd_set_rhs_per_thread(self.ctx, prec, nrhs, int(k)), "wd_set_rhs_per_thread")

    def set_staging(self, prec, rows, stages=2):
        """Plain operators of precision prec through the staged kernel (rows > 0) or the
        direct-load one (rows = 0)."""
        self._check(self.lib.wd_set_staging(self.ctx, prec, int(rows), int(stages)), "wd_set_staging")

    def set_prefetch(self, prec, on=True):
        """The plain FP32 operator through the cp.async-prefetch kernel (on) or the direct one."""
        self._check(self.lib.wd_set_prefetch(self.ctx, prec, int(bool(on))), "wd_set_prefetch")

    def staging_error(self) -> int:
        w = ctypes.c_uint()
        self._check(self.lib.wd_staging_error(self.ctx, ctypes.byref(w)), "wd_staging_error")
        return int(w.value)

    def set_tiles(self, prec, nrhs, site_tile, rhs_tile):
        self._check(self.lib.wd_set_tiles(self.ctx, prec, nrhs, site_tile, rhs_tile), "wd_set_tiles")


class TSplit:
    """A lattice split along t into nranks sub-lattices (section 2.3): which global t-slices
    each rank owns, its neighbours, the sign of the global antiperiodic boundary on what it
    receives, and the face exchange and global sums over torch.distributed.  Host logic
    only: the faces themselves are packed and applied by the library's kernels."""

    def __init__(self, dims, nranks):
        self.dims = tuple(int(d) for d in dims)
        self.nranks = int(nranks)
        if self.nranks < 2 or self.dims[3] % self.nranks:
            raise ValueError("the t extent must split into nranks >= 2 equal blocks")
        self.lt = self.dims[3] // self.nranks
        self.vf = self.dims[0] * self.dims[1] * self.dims[2]  # sites of one t-slice (a face)

    def t_range(self, rank):
        """Global t-slices [t0, t1) of rank."""
        return rank * self.lt, (rank + 1) * self.lt

    def neighbours(self, rank):
        """(previous, next) rank along t, periodic."""
        return (rank - 1) % self.nranks, (rank + 1) % self.nranks

    def receive_signs(self, rank, antiperiodic=True):
        """Signs on what rank receives from (previous, next): -1 across the global boundary
        t = T-1 <-> 0 of an antiperiodic lattice."""
        s = -1.0 if antiperiodic else 1.0
        return (s if rank == 0 else 1.0), (s if rank == self.nranks - 1 else 1.0)

    def local_sites(self, rank):
        """Global site indices of rank's sub-lattice, in its local order (x fastest, t slowest)."""
        t0, t1 = self.t_range(rank)
        return np.arange(t0 * self.vf, t1 * self.vf)

    def local_field(self, psi, rank):
        """Rank's part of a canonical global field (..., V, 4, 3)."""
        t0, t1 = self.t_range(rank)
        return np.ascontiguousarray(psi[..., t0 * self.vf:t1 * self.vf, :, :])

    def local_links(self, U, rank):
        """Rank's links U_mu(n) for its own sites n, (4, V_local, 3, 3)."""
        t0, t1 = self.t_range(rank)
        return np.ascontiguousarray(U[:, t0 * self.vf:t1 * self.vf])

    @staticmethod
    def exchange(dist, rank, prev, nxt, send_prev, recv_prev, send_next, recv_next, group=None):
        """Faces between neighbouring processes, in two shifts so that every message pairs
        with its receive even when prev == next (two processes): first each process sends
        send_next forward and receives recv_prev from behind, then send_prev backward and
        recv_next from ahead.  Tensors (CPU for gloo, CUDA for NCCL)."""
        if prev == rank and nxt == rank:
            recv_prev.copy_(send_next)
            recv_next.copy_(send_prev)
            return
        for snd, dst, rcv, src in ((send_next, nxt, recv_prev, prev), (send_prev, prev, recv_next, nxt)):
            if dist.get_backend(group) == "nccl":
                ops = [dist.P2POp(dist.isend, snd, dst, group), dist.P2POp(dist.irecv, rcv, src, group)]
                for w in dist.batch_isend_irecv(ops):
                    w.wait()
            else:
                ws = [dist.isend(snd, dst, group=group), dist.irecv(rcv, src, group=group)]
                for w in ws:
                    w.wait()

    @staticmethod
    def allreduce_sum(dist, t, group=None):
        """In-place sum of a tensor over all processes."""
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        return t


class SplitLattice(Lattice):
    """The sub-lattice of one rank of a lattice split along t (wd_create_split)."""

    def __init__(self, dims, nranks, rank, antiperiodic_t=True, stream=None):
        self.lib = load_library()
        self.split = TSplit(dims, nranks)
        self.rank = int(rank)
        self.dims = self.split.dims[:3] + (self.split.lt,)
        self.global_dims = self.split.dims
        self.V = int(np.prod(self.dims))
        self.ctx = ctypes.c_void_p()
        self.recon = 18
        self.recon_p = {}
        d = (ctypes.c_int * 4)(*self.global_dims)
        st = self.lib.wd_create_split(ctypes.byref(self.ctx), d, int(nranks), int(rank), int(bool(antiperiodic_t)),
                                      _stream_ptr(stream))
        if st != 0:
            raise WDError(st, "wd_create_split failed")

    def face_bytes(self, prec=WD_F64, nrhs=1) -> int:
        return int(self.lib.wd_face_bytes(self.ctx, prec, nrhs))

    def new_face(self, prec=WD_F64, nrhs=1):
        return torch.zeros(self.face_bytes(prec, nrhs), dtype=torch.uint8, device="cuda")

    def face_pack(self, src, to_prev, to_next, prec=WD_F64, nrhs=1, dagger=False):
        self._check(self.lib.wd_face_pack(self.ctx, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(to_prev.data_ptr()),
                                          ctypes.c_void_p(to_next.data_ptr()), prec, nrhs, int(bool(dagger))),
                    "wd_face_pack")

    def apply_interior(self, kappa, src, dst, prec=WD_F64, nrhs=1, dagger=False):
        self._check(self.lib.wd_apply_interior(self.ctx, float(kappa), ctypes.c_void_p(src.data_ptr()),
                                               ctypes.c_void_p(dst.data_ptr()), prec, nrhs, int(bool(dagger))),
                    "wd_apply_interior")
        return dst

    def apply_faces(self, kappa, from_prev, from_next, dst, prec=WD_F64, nrhs=1, dagger=False):
        self._check(self.lib.wd_apply_faces(self.ctx, float(kappa), ctypes.c_void_p(from_prev.data_ptr()),
                                            ctypes.c_void_p(from_next.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                            prec, nrhs, int(bool(dagger))), "wd_apply_faces")
        return dst


def _cuda_bytes(ptr, n):
    """A torch uint8 CUDA tensor over n bytes of device memory at ptr (no copy)."""
    class _Arr:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": "|u1", "data": (int(ptr), False), "version": 3}
    return torch.as_tensor(_Arr(), device="cuda")


class DistComm:
    """wd_comm over torch.distributed for split solves spread over processes (one
    sub-lattice block per process): faces through TSplit.exchange, sums through all_reduce.
    With NCCL the faces go device to device; with gloo (which sends host tensors) they are
    staged through host memory on the library's work stream, which must be torch's current
    stream (the default for SplitLattice).  Keeps its ctypes callbacks alive while it exists."""

    def __init__(self, dist, split: TSplit, first_rank, last_rank, proc_of_rank, group=None):
        self.dist, self.split, self.group = dist, split, group
        me = dist.get_rank(group)
        self.me = me
        self.prev = proc_of_rank(split.neighbours(first_rank)[0])
        self.next = proc_of_rank(split.neighbours(last_rank)[1])

        def exchange(user, send_prev, recv_prev, send_next, recv_next, nbytes, stream):
            try:
                t = [_cuda_bytes(p, nbytes) for p in (send_prev, recv_prev, send_next, recv_next)]
                if self.dist.get_backend(self.group) == "nccl":
                    TSplit.exchange(self.dist, self.me, self.prev, self.next, t[0], t[1], t[2], t[3], self.group)
                else:
                    h = [x.cpu() for x in t]  # waits for the packed faces on the current stream
                    TSplit.exchange(self.dist, self.me, self.prev, self.next, h[0], h[1], h[2], h[3], self.group)
                    t[1].copy_(h[1])
                    t[3].copy_(h[3])
                return 0
            except Exception:  # a failed exchange is reported through the status, never raised through C
                return 1

        def allreduce(user, vals, n):
            try:
                dev = "cuda" if self.dist.get_backend(self.group) == "nccl" else "cpu"
                t = torch.tensor([vals[i] for i in range(n)], dtype=torch.float64, device=dev)
                TSplit.allreduce_sum(self.dist, t, self.group)
                for i, v in enumerate(t.cpu().tolist()):
                    vals[i] = v
                return 0
            except Exception:
                return 1

        self._cb = (EXCHANGE_FN(exchange), ALLREDUCE_FN(allreduce))
        self.struct = Comm(None, self._cb[0], self._cb[1])


def cg_split(lattices, kappa, bs, xs, tol=1e-10, max_iter=10000, comm=None):
    """CGNR on a lattice split along t (wd_cg_solve_split): lattices are this process's
    SplitLattice blocks (consecutive ranks); comm a DistComm when other processes hold the rest."""
    lib = load_library()
    n = len(lattices)
    ctxs = (ctypes.c_void_p * n)(*[L.ctx.value for L in lattices])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    p = CGParams(tol, max_iter, WD_F64, 0.0, 1, 0, 0, 0, 0, 0)
    res = CGResult()
    st = lib.wd_cg_solve_split(ctxs, n, float(kappa), bp, xp, ctypes.byref(p), ctypes.byref(res),
                               ctypes.byref(comm.struct) if comm is not None else None)
    return res.as_dict(), st


def measure_fp64_rate() -> float:
    """GFLOP/s of independent FP64 multiply-add chains on the current device (wd_measure_fp64_rate)."""
    lib = load_library()
    g = ctypes.c_double()
    st = lib.wd_measure_fp64_rate(ctypes.byref(g))
    if st != 0:
        raise WDError(st, "wd_measure_fp64_rate failed")
    return float(g.value)


def device_tag() -> str:
    """Name and compute capability of the current CUDA device."""
    i = torch.cuda.current_device()
    major, minor = torch.cuda.get_device_capability(i)
    return f"{torch.cuda.get_device_name(i)}|sm_{major}{minor}"


def tile_cache_key(dims, prec, recon, nrhs, device) -> str:
    return f"{'x'.join(str(int(d)) for d in dims)}|prec{int(prec)}|recon{int(recon)}|nrhs{int(nrhs)}|{device}"


class TileCache:
    """Autotuned launch shapes on disk: a JSON object {key: [site_tile, rhs_tile]}.
    Writes go to a temporary file that replaces the old one, so a reader never sees a
    partial file; an unreadable file counts as empty."""

    def __init__(self, path):
        self.path = os.fspath(path)

    def load(self) -> dict:
        try:
            with open(self.path) as f:
                d = json.load(f)
            return d if isinstance(d, dict) else {}
        except (OSError, ValueError):
            return {}

    def get(self, key):
        v = self.load().get(key)
        if isinstance(v, list) and len(v) == 2 and all(isinstance(t, int) for t in v):
            return int(v[0]), int(v[1])
        return None

    def put(self, key, tiles) -> None:
        d = self.load()
        d[key] = [int(tiles[0]), int(tiles[1])]
        tmp = f"{self.path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def cg_batched(lattices, kappas, bs, xs, tol=1e-10, max_iter=10000, inner=WD_F32, delta=0.0):
    """Solve many independent lattices in one persistent launch (wd_cg_solve_batched)."""
    lib = load_library()
    n = len(lattices)
    ctxs = (ctypes.c_void_p * n)(*[L.ctx.value for L in lattices])
    ks = (ctypes.c_double * n)(*[float(k) for k in kappas])
    bp = (ctypes.c_void_p * n)(*[b.data_ptr() for b in bs])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    p = CGParams(tol, max_iter, inner, delta, 1, 0, 0, 0, 0, 0)
    res = (CGResult * n)()
    st = lib.wd_cg_solve_batched(ctxs, ks, bp, xp, n, ctypes.byref(p), res)
    return [r.as_dict() for r in res], st
