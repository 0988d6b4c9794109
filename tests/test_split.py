"""Domain decomposition along t (section 2.3: sub-lattices with copies of their
neighbours' boundary sites, global scalar products in CG).

GPU (one device, all sub-lattices in one process): the split operator -- faces packed,
exchanged by device copies, interior and face launches -- against the oracle's unsplit D
and D^dag; the decomposed CG against the oracle's solution.  GPU, two processes sharing the
device: the decomposed CG with the faces and sums through DistComm's callbacks over gloo.

CPU (world_size-2 gloo ranks): the host-side logic of the split -- which slices each rank
owns, who its neighbours are, the face exchange in both directions, the sign of the global
antiperiodic boundary and the global sums -- reproduces the unsplit oracle: each rank
evaluates the oracle's operator on its own sites of a sub-lattice extended by the slices it
received.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1810_04201_gb300 import gen
from paper_1810_04201_gb300.wd import TSplit

TOL = {0: 1e-13, 1: 2e-6}


# ----------------------------------------------------------------------------- host logic
def test_tsplit_partition_and_neighbours():
    sp = TSplit((4, 6, 2, 12), 4)
    owned = np.concatenate([sp.local_sites(r) for r in range(4)])
    np.testing.assert_array_equal(owned, np.arange(4 * 6 * 2 * 12))
    assert [sp.t_range(r) for r in range(4)] == [(0, 3), (3, 6), (6, 9), (9, 12)]
    assert sp.neighbours(0) == (3, 1) and sp.neighbours(3) == (2, 0)
    assert sp.receive_signs(0) == (-1.0, 1.0) and sp.receive_signs(3) == (1.0, -1.0)
    assert sp.receive_signs(1) == (1.0, 1.0) and sp.receive_signs(0, antiperiodic=False) == (1.0, 1.0)
    with pytest.raises(ValueError):
        TSplit((4, 4, 4, 6), 4)
    with pytest.raises(ValueError):
        TSplit((4, 4, 4, 6), 1)


def extended_operator_at_local_sites(U, psi, kappa, sp, rank, halo_prev, halo_next, link_prev, dagger):
    """The oracle's operator at rank's own sites, evaluated on the sub-lattice extended by one
    received slice on each side (periodic in x, y, z; the extension keeps every t neighbour of
    an owned site inside it, so its own wrap is never used)."""
    vf, lt = sp.vf, sp.lt
    dims_ext = sp.dims[:3] + (lt + 2,)
    psi_ext = np.concatenate([halo_prev, sp.local_field(psi, rank), halo_next])
    U_ext = np.zeros((4, vf * (lt + 2), 3, 3), complex)
    U_ext[:, :, 0, 0] = U_ext[:, :, 1, 1] = U_ext[:, :, 2, 2] = 1.0  # links no owned site reads
    U_ext[:, vf:vf * (lt + 1)] = sp.local_links(U, rank)
    U_ext[3, :vf] = link_prev  # U_t(n - t) of the first owned slice
    sites = np.arange(vf, vf * (lt + 1))
    return oracle.apply_D_sites(U_ext, psi_ext, kappa, dims_ext, sites, antiperiodic_t=False, dagger=dagger)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gloo_rank(rank, world, port, dims, kappa, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sp = TSplit(dims, world)
        U = gen.haar_links(dims, seed=61)
        psi = gen.gaussian_source(dims, seed=62)
        prev, nxt = sp.neighbours(rank)
        loc = sp.local_field(psi, rank)
        vf = sp.vf
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.float64).copy())
        send_prev, send_next = t(loc[:vf]), t(loc[-vf:])
        recv_prev, recv_next = torch.empty_like(send_prev), torch.empty_like(send_next)
        TSplit.exchange(dist, rank, prev, nxt, send_prev, recv_prev, send_next, recv_next)
        # the t links of the last slice travel forward once (the backward hop of the next rank)
        lk = t(sp.local_links(U, rank)[3, -vf:])
        lk_prev, dummy = torch.empty_like(lk), torch.empty_like(lk)
        TSplit.exchange(dist, rank, prev, nxt, lk.clone(), lk_prev, lk, dummy)
        s_prev, s_next = sp.receive_signs(rank, antiperiodic=True)
        c = lambda x, shape: x.numpy().view(np.complex128).reshape(shape)
        halo_prev = s_prev * c(recv_prev, (vf, 4, 3))
        halo_next = s_next * c(recv_next, (vf, 4, 3))
        res = {}
        for dagger in (False, True):
            mine = extended_operator_at_local_sites(U, psi, kappa, sp, rank, halo_prev, halo_next,
                                                    c(lk_prev, (vf, 3, 3)), dagger)
            want = oracle.apply_D(U, psi, kappa, dims, antiperiodic_t=True, dagger=dagger)[sp.local_sites(rank)]
            n2 = torch.tensor([float(np.vdot(mine, mine).real)], dtype=torch.float64)
            TSplit.allreduce_sum(dist, n2)
            full = oracle.apply_D(U, psi, kappa, dims, antiperiodic_t=True, dagger=dagger)
            res[dagger] = (oracle.rel_err(mine, want), float(n2.item()), float(np.vdot(full, full).real))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dims", [(4, 4, 2, 4), (2, 4, 4, 6)])
def test_gloo_two_ranks_exchange_matches_unsplit_oracle(dims):
    """Two gloo processes, one sub-lattice each (so each process is both the other's previous
    and next neighbour): the exchanged faces, with the boundary sign, give each rank the
    unsplit operator on its sites, and the global sum of |D psi|^2 is the unsplit one."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_gloo_rank, args=(r, 2, port, dims, 0.12, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=240) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        for dagger, (err, n2, n2_full) in got[rank].items():
            assert err < 1e-14, (rank, dagger, err)
            assert n2 == pytest.approx(n2_full, rel=1e-12)


# ----------------------------------------------------------------------------- GPU
@pytest.fixture(scope="module")
def wd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import wd as _wd
    return _wd


def split_blocks(wd, dims, nranks, U, antiperiodic=True, recon=18):
    blocks = []
    for r in range(nranks):
        b = wd.SplitLattice(dims, nranks, r, antiperiodic_t=antiperiodic)
        b.set_gauge(b.split.local_links(U, r), recon=recon)
        blocks.append(b)
    return blocks


def split_apply(blocks, kappa, fields, prec, dagger, nrhs=1):
    """D (or D^dag) on every block: faces packed, exchanged by device copies, interior and faces."""
    n = len(blocks)
    to_prev = [b.new_face(prec, nrhs) for b in blocks]
    to_next = [b.new_face(prec, nrhs) for b in blocks]
    for b, f, tp, tn in zip(blocks, fields, to_prev, to_next):
        b.face_pack(f, tp, tn, prec, nrhs=nrhs, dagger=dagger)
    outs = []
    for k, (b, f) in enumerate(zip(blocks, fields)):
        o = b.new_field(prec, nrhs)
        b.apply_interior(kappa, f, o, prec, nrhs=nrhs, dagger=dagger)
        b.apply_faces(kappa, to_next[(k - 1) % n].clone(), to_prev[(k + 1) % n].clone(), o, prec, nrhs=nrhs,
                      dagger=dagger)
        outs.append(o)
    return outs


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nranks", [((4, 4, 4, 8), 2), ((4, 6, 2, 8), 4), ((6, 4, 4, 6), 3), ((4, 2, 4, 4), 4),
                                         ((5, 3, 4, 6), 2)])
@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("dagger", [False, True])
def test_split_operator_matches_unsplit_oracle(wd, dims, nranks, prec, dagger):
    """Sub-lattices of 1 to 4 slices (one slice: both faces on the same slice), odd extents."""
    kappa = 0.124
    U = gen.haar_links(dims, seed=71)
    psi = gen.gaussian_source(dims, seed=72)
    blocks = split_blocks(wd, dims, nranks, U)
    fields = [b.pack(b.split.local_field(psi, r), prec) for r, b in enumerate(blocks)]
    outs = split_apply(blocks, kappa, fields, prec, dagger)
    torch.cuda.synchronize()
    got = np.concatenate([b.unpack(o, prec) for b, o in zip(blocks, outs)])
    want = oracle.apply_D(U, psi, kappa, dims, antiperiodic_t=True, dagger=dagger)
    assert oracle.rel_err(got, want) < TOL[prec]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_split_operator_multi_rhs(wd, prec):
    """Several right-hand sides per launch on sub-lattices, with the launch shape the autotuner
    picks; the FP32 kernel with several right-hand sides per thread (which has no sub-lattice
    form) is neither tuned nor accepted there."""
    dims, nranks, kappa, nrhs = (4, 6, 4, 8), 2, 0.124, 4
    U = gen.haar_links(dims, seed=81)
    psis = np.stack([gen.gaussian_source(dims, seed=82 + j) for j in range(nrhs)])
    blocks = split_blocks(wd, dims, nranks, U)
    for b in blocks:
        b.autotune(prec, nrhs)
        assert b.tiles(prec, nrhs)[2] == 1
    if prec == 1:
        with pytest.raises(wd.WDError):
            blocks[0].set_rhs_per_thread(prec, nrhs, 2)
    fields = [b.pack(np.stack([b.split.local_field(p, r) for p in psis]), prec) for r, b in enumerate(blocks)]
    for dagger in (False, True):
        outs = split_apply(blocks, kappa, fields, prec, dagger, nrhs)
        torch.cuda.synchronize()
        got = np.concatenate([b.unpack(o, prec, nrhs, squeeze=False) for b, o in zip(blocks, outs)], axis=1)
        for j in range(nrhs):
            want = oracle.apply_D(U, psis[j], kappa, dims, antiperiodic_t=True, dagger=dagger)
            assert oracle.rel_err(got[j], want) < TOL[prec], (j, dagger)


@pytest.mark.gpu
@pytest.mark.parametrize("antiperiodic,recon", [(False, 18), (True, 12), (True, 8)])
def test_split_operator_boundary_and_compression(wd, antiperiodic, recon):
    dims, nranks, kappa = (4, 4, 6, 8), 4, 0.11
    U = gen.haar_links(dims, seed=73)
    psi = gen.gaussian_source(dims, seed=74)
    blocks = split_blocks(wd, dims, nranks, U, antiperiodic, recon)
    fields = [b.pack(b.split.local_field(psi, r)) for r, b in enumerate(blocks)]
    for dagger in (False, True):
        outs = split_apply(blocks, kappa, fields, 0, dagger)
        got = np.concatenate([b.unpack(o) for b, o in zip(blocks, outs)])
        want = oracle.apply_D(U, psi, kappa, dims, antiperiodic_t=antiperiodic, dagger=dagger)
        assert oracle.rel_err(got, want) < 1e-13


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nranks", [((8, 8, 8, 8), 2), ((6, 4, 6, 8), 4)])
def test_split_cg_matches_oracle_solution(wd, dims, nranks):
    """The decomposed CG (faces between the sub-lattices by device copies on a side stream,
    every scalar product summed over all of them) gives the oracle's solution."""
    kappa = 0.12
    U = gen.haar_links(dims, seed=75)
    b = gen.gaussian_source(dims, seed=76)
    blocks = split_blocks(wd, dims, nranks, U)
    bs = [blk.pack(blk.split.local_field(b, r)) for r, blk in enumerate(blocks)]
    xs = [blk.new_field() for blk in blocks]
    res, st = wd.cg_split(blocks, kappa, bs, xs, tol=1e-10)
    assert st == 0 and res["status"] == 0, res
    x = np.concatenate([blk.unpack(f) for blk, f in zip(blocks, xs)])
    x_ref, info = oracle.cgnr(U, b, kappa, dims, tol=1e-13)
    assert oracle.rel_err(x, x_ref) < 1e-9
    # the residuals it reports are those of its x, through the oracle's unsplit operator
    r = b - oracle.apply_D(U, x, kappa, dims)
    rn = np.linalg.norm(oracle.apply_Ddag(U, r, kappa, dims)) / np.linalg.norm(oracle.apply_Ddag(U, b, kappa, dims))
    assert res["true_rel_resid"] == pytest.approx(rn, rel=1e-4) and rn <= 1.01e-10
    assert res["true_rel_resid_b"] == pytest.approx(np.linalg.norm(r) / np.linalg.norm(b), rel=1e-4)
    # same recursion as the unsplit oracle CG to 1e-10: the same iteration count, within one
    _, i10 = oracle.cgnr(U, b, kappa, dims, tol=1e-10)
    assert abs(res["iters"] - i10["iters"]) <= 1
    # a start vector: the solve resumes from it
    xs2 = [blk.pack(blk.split.local_field(0.5 * x_ref, r)) for r, blk in enumerate(blocks)]
    res2, st2 = wd.cg_split(blocks, kappa, bs, xs2, tol=1e-10)
    assert st2 == 0 and res2["iters"] <= res["iters"]
    x2 = np.concatenate([blk.unpack(f) for blk, f in zip(blocks, xs2)])
    assert oracle.rel_err(x2, x_ref) < 1e-9


@pytest.mark.gpu
def test_split_refusals(wd):
    dims = (4, 4, 4, 8)
    U = gen.haar_links(dims, seed=77)
    blocks = split_blocks(wd, dims, 2, U)
    b0 = blocks[0]
    f = b0.new_field()
    with pytest.raises(wd.WDError) as e:  # the plain operator would miss the faces
        b0.apply(0.12, f, b0.new_field())
    assert e.value.status == 8
    _, st = b0.cg(0.12, f, b0.new_field(), raise_on_fail=False)
    assert st == 8
    with pytest.raises(wd.WDError) as e:  # FP16 faces are not built
        b0.face_pack(b0.new_field(2), b0.new_face(), b0.new_face(), prec=2)
    assert e.value.status == 1
    assert b0.face_bytes(2) == 0 and b0.face_bytes(0) == 6 * 64 * 16
    # one of two sub-lattices in this process and no callbacks: refused
    res, st = wd.cg_split(blocks[:1], 0.12, [f], [b0.new_field()])
    assert st == 1
    with pytest.raises(ValueError):
        wd.SplitLattice((4, 4, 4, 6), 4, 0)
    lib = wd.load_library()
    import ctypes
    ctx = ctypes.c_void_p()
    assert lib.wd_create_split(ctypes.byref(ctx), (ctypes.c_int * 4)(4, 4, 4, 6), 4, 0, 1, None) == 1
    # an ordinary context is not split
    plain = wd.Lattice(dims)
    plain.set_gauge(U)
    assert int(lib.wd_face_bytes(plain.ctx, 0, 1)) == 0


def _split_solve_rank(rank, world, port, dims, kappa, out):
    """One process of a two-process split solve on one GPU: its own sub-lattice and context,
    faces and scalar products through DistComm over gloo (host-staged faces)."""
    import datetime
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        import __graft_entry__  # noqa: F401  (puts the repository on the path)
        from paper_1810_04201_gb300 import wd
        torch.cuda.set_device(0)
        U = gen.haar_links(dims, seed=75)
        b = gen.gaussian_source(dims, seed=76)
        lat = wd.SplitLattice(dims, world, rank)
        lat.set_gauge(lat.split.local_links(U, rank))
        fb = lat.pack(lat.split.local_field(b, rank))
        fx = lat.new_field()
        comm = wd.DistComm(dist, lat.split, rank, rank, lambda k: k)
        res, st = wd.cg_split([lat], kappa, [fb], [fx], tol=1e-10, comm=comm)
        out.put((rank, st, res, lat.unpack(fx)))
    except Exception as e:  # reported to the parent, which fails the test
        out.put((rank, -1, repr(e), None))
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_split_cg_two_processes_gloo(wd):
    """The decomposed CG across two processes sharing one GPU: each process holds one sub-lattice,
    the library calls DistComm's callbacks for the face exchange and the global sums (gloo, faces
    staged through host memory; no kernel waits on the other process), and the joined solution is
    the oracle's, with the iteration count of the one-process split solve."""
    dims, kappa = (6, 4, 6, 8), 0.12
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_solve_rank, args=(r, 2, port, dims, kappa, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r[0], r[1:]) for r in (q.get(timeout=300) for _ in range(2)))
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
        assert p.exitcode == 0
    for rank in (0, 1):
        assert got[rank][0] == 0, got[rank]
    x = np.concatenate([got[0][2], got[1][2]])
    U = gen.haar_links(dims, seed=75)
    b = gen.gaussian_source(dims, seed=76)
    x_ref, _ = oracle.cgnr(U, b, kappa, dims, tol=1e-13)
    assert oracle.rel_err(x, x_ref) < 1e-9
    assert got[0][1]["iters"] == got[1][1]["iters"]
    assert got[0][1]["true_rel_resid"] == pytest.approx(got[1][1]["true_rel_resid"], rel=1e-12)
    blocks = split_blocks(wd, dims, 2, U)
    res1, st1 = wd.cg_split(blocks, kappa, [blk.pack(blk.split.local_field(b, r)) for r, blk in enumerate(blocks)],
                            [blk.new_field() for blk in blocks], tol=1e-10)
    assert st1 == 0 and abs(res1["iters"] - got[0][1]["iters"]) <= 1
