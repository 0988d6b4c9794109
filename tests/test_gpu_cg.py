"""GPU CG solvers against the CPU oracle (through the C ABI).

Bar: true FP64 normal residual <= 1e-10 recomputed by the library, and the
solution within 1e-9 (relative 2-norm) of the oracle solution iterated to
1e-13, on lattices whose condition number keeps that bound (Haar links,
kappa <= 0.125: cond(D) about 4).
"""
import numpy as np
import pytest

import oracle
from paper_1810_04201_gb300 import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def wd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import wd as _wd
    return _wd


def ref_solution(U, b, kappa, dims):
    x, info = oracle.cgnr(U, b, kappa, dims, tol=1e-13, max_iter=20000)
    assert info["converged"]
    return x, info


@pytest.mark.parametrize("inner", [0, 1, 2, 3])
def test_cg_4x4(wd, inner):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=1)
    x_ref, info = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner)
    r = res[0]
    assert st == 0 and r["status"] == 0
    assert r["true_rel_resid"] <= 1e-10
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9
    if inner == 0:
        _, i10 = oracle.cgnr(U, b, kappa, dims, tol=1e-10)
        assert abs(r["iters"] - i10["iters"]) <= 1
    else:
        assert r["reliable_updates"] >= 1


@pytest.mark.parametrize("inner", [0, 1, 2, 3])
@pytest.mark.parametrize("recon", [18, 12, 8])
def test_cg_odd_shapes(wd, inner, recon):
    dims, kappa = (6, 6, 6, 8), 0.124
    U = gen.haar_links(dims, seed=3)
    b = gen.gaussian_source(dims, seed=4)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=recon)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner)
    assert st == 0 and res[0]["true_rel_resid"] <= 1e-10
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9


def test_cg_dense_lu_2x4(wd):
    """On 2^4 (each neighbour reached twice) the solution matches LAPACK's LU solve."""
    dims, kappa = (2, 2, 2, 2), 0.12
    U = gen.haar_links(dims, seed=21)
    b = gen.gaussian_source(dims, seed=22)
    xd = oracle.dense_solve(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-12)
    assert st == 0
    assert oracle.rel_err(lat.unpack(fx), xd) < 1e-10


@pytest.mark.parametrize("inner", [0, 1, 2, 3])
def test_cg_multi_rhs_point_sources(wd, inner):
    dims, kappa = (4, 4, 4, 8), 0.12
    U = gen.haar_links(dims, seed=7)
    B = gen.propagator_sources(dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(B), lat.new_field(nrhs=12)
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, nrhs=12)
    assert st == 0
    X = lat.unpack(fx, nrhs=12)
    for k in (0, 5, 11):
        x_ref, _ = ref_solution(U, B[k], kappa, dims)
        assert oracle.rel_err(X[k], x_ref) < 1e-9
    assert all(r["true_rel_resid"] <= 1e-10 for r in res)


def test_cg_initial_guess_and_zero_source(wd):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=2)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    r1, _ = lat.cg(kappa, fb, fx, tol=1e-10)
    r2, st = lat.cg(kappa, fb, fx, tol=1e-10)  # resume from the converged solution
    assert st == 0 and r2[0]["iters"] == 0
    z = lat.pack(np.zeros_like(b))
    fz = lat.new_field()
    r3, st = lat.cg(kappa, z, fz, tol=1e-10)
    assert st == 0 and r3[0]["iters"] == 0
    assert not lat.unpack(fz).any()


@pytest.mark.parametrize("inner,eo", [(0, 0), (1, 0), (0, 1), (2, 1)])
def test_start_vector_zero_and_nearly_zero(wd, inner, eo):
    """A zero start vector skips the D x0 work; a start vector with one tiny nonzero
    entry (and the same vector in another right-hand side) takes the full setup.  All
    reach the oracle solution."""
    dims, kappa = (4, 4, 4, 6), 0.12
    U = gen.haar_links(dims, seed=31)
    b = gen.gaussian_source(dims, seed=32)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb = lat.pack(b)
    x0 = np.zeros_like(b)
    x0[7, 2, 1] = 1e-300
    for start in (np.zeros_like(b), x0, 0.5 * x_ref):
        fx = lat.pack(start)
        res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, precondition=eo)
        assert st == 0 and res[0]["true_rel_resid"] <= 1e-10
        assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9
    B = np.stack([b, b])
    X0 = np.stack([np.zeros_like(b), x0])
    fX = lat.pack(X0)
    res, st = lat.cg(kappa, lat.pack(B), fX, tol=1e-10, inner=inner, nrhs=2, precondition=eo)
    assert st == 0
    X = lat.unpack(fX, nrhs=2, squeeze=False)
    assert all(oracle.rel_err(X[j], x_ref) < 1e-9 for j in range(2))


def test_cg_failure_statuses(wd):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=2)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, max_iter=3, raise_on_fail=False)
    assert st == 4 and res[0]["iters"] == 3
    bn = b.copy()
    bn[5, 1, 2] = np.nan
    res, st = lat.cg(kappa, lat.pack(bn), lat.new_field(), tol=1e-10, raise_on_fail=False)
    assert st == 6
    res, st = lat.cg(kappa, lat.pack(bn), lat.new_field(), tol=1e-10, inner=1, raise_on_fail=False)
    assert st == 6


def test_cg_canonical_host_buffers(wd):
    import torch
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=1)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    bt = torch.from_numpy(b.copy()).pin_memory()
    xt = torch.zeros_like(bt).pin_memory()
    res, st = lat.cg_canonical(kappa, bt, xt, tol=1e-10)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    assert st == 0 and oracle.rel_err(xt.numpy(), x_ref) < 1e-9


@pytest.mark.parametrize("k,recon,seed", [(12, 18, 7), (5, 12, 8), (1, 18, 9), (4, 8, 10)])
def test_block_cg(wd, k, recon, seed):
    """Block CG over k right-hand sides: every column matches the oracle solution."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = gen.haar_links(dims, seed=seed)
    B = gen.propagator_sources(dims)[:k] if k == 12 else gen.gaussian_source(dims, seed=seed, nrhs=k)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=recon)
    fb, fx = lat.pack(B), lat.new_field(nrhs=k)
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, nrhs=k, block=1)
    assert st == 0, res
    X = lat.unpack(fx, nrhs=k, squeeze=False)
    for j in sorted({0, k // 2, k - 1}):
        x_ref, _ = ref_solution(U, B[j], kappa, dims)
        assert oracle.rel_err(X[j], x_ref) < 1e-9
    assert all(r["true_rel_resid"] <= 1e-10 for r in res)
    if k == 12:
        fy = lat.new_field(nrhs=k)
        res1, _ = lat.cg(kappa, fb, fy, tol=1e-10, nrhs=k, block=0)
        assert res[0]["iters"] < max(r["iters"] for r in res1)


@pytest.mark.parametrize("inner", [0, 1, 2])
def test_host_loop_matches_graph(wd, inner, monkeypatch):
    """The host-driven loop (WD_CG_LOOP=host) launches the same kernels: same result, bit for bit."""
    dims, kappa = (4, 4, 6, 4), 0.12
    U = gen.haar_links(dims, seed=3)
    b = gen.gaussian_source(dims, seed=4)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb = lat.pack(b)
    fx1, fx2 = lat.new_field(), lat.new_field()
    r1, _ = lat.cg(kappa, fb, fx1, tol=1e-10, inner=inner)
    monkeypatch.setenv("WD_CG_LOOP", "host")
    r2, _ = lat.cg(kappa, fb, fx2, tol=1e-10, inner=inner)
    assert r1[0]["iters"] == r2[0]["iters"]
    np.testing.assert_array_equal(lat.unpack(fx1), lat.unpack(fx2))


def test_autotune_keeps_results(wd):
    dims, kappa = (8, 8, 8, 8), 0.12
    U = gen.haar_links(dims, seed=5)
    psi = gen.gaussian_source(dims, seed=6, nrhs=4)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    f = lat.pack(psi)
    o1 = lat.new_field(nrhs=4)
    lat.apply(kappa, f, o1, nrhs=4)
    st, rt = lat.autotune(0, 4)
    assert st in (16, 32, 64, 128, 256) and 1 <= rt <= 4 and (st * rt) % 32 == 0
    o2 = lat.new_field(nrhs=4)
    lat.apply(kappa, f, o2, nrhs=4)
    # the per-site arithmetic does not depend on the launch shape
    np.testing.assert_array_equal(lat.unpack(o1, nrhs=4), lat.unpack(o2, nrhs=4))


@pytest.mark.parametrize("inner", [0, 1, 3])
def test_cgne_paper_form(wd, inner):
    """CGNE (the paper's listing: D D^dag y = b, x = D^dag y) gives the oracle's solution."""
    dims, kappa = (4, 4, 6, 4), 0.12
    U = gen.haar_links(dims, seed=13)
    b = gen.gaussian_source(dims, seed=14)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    _, ine = oracle.cgne(U, b, kappa, dims, tol=1e-10)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, normal_eq=1)
    assert st == 0
    assert res[0]["true_rel_resid_b"] <= 1e-10 * 1.01
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9
    if inner == 0:
        assert abs(res[0]["iters"] - ine["iters"]) <= 1


def _parity(dims):
    V = int(np.prod(dims))
    n = np.arange(V)
    c = []
    for L in dims:
        c.append(n % L)
        n = n // L
    return (sum(c) % 2).astype(bool)


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 6, 8), (8, 6, 4, 2)])
@pytest.mark.parametrize("dagger", [False, True])
def test_schur_operator_matches_oracle(wd, dims, dagger):
    """(1 - k^2 H_eo H_oe) x_e equals the even part of D (x_e, kappa H_oe x_e), built from the oracle's D."""
    kappa = 0.12
    U = gen.haar_links(dims, seed=17)
    psi = gen.gaussian_source(dims, seed=18)
    odd = _parity(dims)
    xe = psi.copy()
    xe[odd] = 0
    y = oracle.apply_D(U, xe, kappa, dims, dagger=dagger)   # odd sites: -kappa H_oe x_e
    z = xe.copy()
    z[odd] = -y[odd]                                        # x_o = kappa H_oe x_e
    ref = oracle.apply_D(U, z, kappa, dims, dagger=dagger)
    ref[odd] = 0
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    out = lat.new_field()
    lat.apply_schur(kappa, lat.pack(psi), out, dagger=dagger)
    assert oracle.rel_err(lat.unpack(out), ref) < 1e-13


@pytest.mark.parametrize("inner,recon", [(0, 18), (1, 18), (2, 12), (3, 18), (0, 8), (1, 8)])
def test_even_odd_cg(wd, inner, recon):
    """Even-odd preconditioned CGNR: same solution as the oracle, about half the iterations."""
    dims, kappa = (4, 6, 4, 8), 0.124
    U = gen.haar_links(dims, seed=19)
    b = gen.gaussian_source(dims, seed=20)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=recon)
    fb = lat.pack(b)
    fx, fy = lat.new_field(), lat.new_field()
    r_eo, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, precondition=1)
    assert st == 0
    assert r_eo[0]["true_rel_resid"] <= 1e-10
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9
    r_full, _ = lat.cg(kappa, fb, fy, tol=1e-10, inner=inner)
    assert r_eo[0]["iters"] < 0.8 * r_full[0]["iters"]


def test_even_odd_rejects_odd_extents(wd):
    lat = wd.Lattice((3, 4, 4, 4))
    lat.set_gauge(gen.unit_links((3, 4, 4, 4)))
    b = lat.pack(gen.gaussian_source((3, 4, 4, 4), 1))
    res, st = lat.cg(0.12, b, lat.new_field(), precondition=1, raise_on_fail=False)
    assert st == 1


def test_max_rhs_and_side_stream(wd):
    """16 right-hand sides (the maximum) on a non-default stream."""
    import torch
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=23)
    B = gen.gaussian_source(dims, seed=24, nrhs=16)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        lat = wd.Lattice(dims)
        lat.set_gauge(U)
        fb, fx = lat.pack(B), lat.new_field(nrhs=16)
        res, st = lat.cg(kappa, fb, fx, tol=1e-10, nrhs=16, inner=1)
        X = lat.unpack(fx, nrhs=16, squeeze=False)
    assert st == 0 and all(r["true_rel_resid"] <= 1e-10 for r in res)
    for j in (0, 15):
        x_ref, _ = ref_solution(U, B[j], kappa, dims)
        assert oracle.rel_err(X[j], x_ref) < 1e-9
    with pytest.raises(wd.WDError):
        lat.cg(kappa, fb, fx, nrhs=17)


def test_canonical_pageable_host_buffers(wd):
    dims, kappa = (4, 4, 2, 4), 0.12
    U = gen.haar_links(dims, seed=25)
    b = gen.gaussian_source(dims, seed=26)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    x = np.zeros_like(b)
    res, st = lat.cg_canonical(kappa, b, x, tol=1e-10, precondition=1)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    assert st == 0 and oracle.rel_err(x, x_ref) < 1e-9


def test_corrupted_inputs_give_statuses_not_hangs(wd):
    """A NaN link or an infinite source entry ends the solve with WD_ERR_NONFINITE in
    every inner precision (and in the batched solver), never with a hang."""
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=2)
    Ubad = U.copy()
    Ubad[2, 17, 1, 0] = np.nan
    lat = wd.Lattice(dims)
    lat.set_gauge(Ubad)
    for inner in (0, 1, 2, 3):
        res, st = lat.cg(kappa, lat.pack(b), lat.new_field(), tol=1e-10, inner=inner, raise_on_fail=False)
        assert st == 6 and res[0]["status"] == 6, inner
    lat.set_gauge(U)
    binf = b.copy()
    binf[3, 0, 0] = np.inf
    res, st = lat.cg(kappa, lat.pack(binf), lat.new_field(), tol=1e-10, raise_on_fail=False)
    assert st == 6
    res, st = wd.cg_batched([lat], [kappa], [lat.pack(binf)], [lat.new_field()], tol=1e-10)
    assert res[0]["status"] == 6


def test_autotune_cache_file(wd, tmp_path):
    """Tiles tuned once are stored under (lattice, precision, links, nrhs, device) and
    reused by a later context without timing."""
    import json
    dims = (8, 8, 8, 8)
    path = tmp_path / "tiles.json"
    lat = wd.Lattice(dims)
    lat.set_gauge(gen.haar_links(dims, seed=3), recon=12)
    t1 = lat.autotune(1, 4, cache=path)
    key = wd.tile_cache_key(dims, 1, 12, 4, wd.device_tag())
    assert json.loads(path.read_text())[key] == list(t1)
    lat2 = wd.Lattice(dims)
    lat2.set_gauge(gen.haar_links(dims, seed=3), recon=12)
    before = lat2.launches
    assert lat2.autotune(1, 4, cache=path) == t1
    assert lat2.launches == before  # no timing launches
    assert lat2.autotune(1, 2, cache=path) != () and len(json.loads(path.read_text())) == 2


@pytest.mark.parametrize("inner,rin,eo", [(1, 12, 1), (2, 8, 0), (1, 8, 1), (3, 12, 0)])
def test_whole_fp64_links_with_compressed_inner_links(wd, inner, rin, eo):
    """FP64 links kept whole (18) beside recon-12/8 links of the inner precision: the
    operators of both precisions and the mixed solve agree with the oracle."""
    dims, kappa = (4, 6, 4, 8), 0.124
    U = gen.haar_links(dims, seed=41)
    b = gen.gaussian_source(dims, seed=42)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=18)
    lat.set_link_compression(inner, rin)
    tol = {1: 2e-6, 2: 4e-3, 3: 1e-13}[inner]
    for prec, t in ((0, 1e-13), (inner, tol)):
        o = lat.new_field(prec)
        lat.apply(kappa, lat.pack(b, prec), o, prec)
        assert oracle.rel_err(lat.unpack(o, prec), oracle.apply_D(U, b, kappa, dims)) < t
    fx = lat.new_field()
    res, st = lat.cg(kappa, lat.pack(b), fx, tol=1e-10, inner=inner, precondition=eo)
    assert st == 0 and res[0]["true_rel_resid"] <= 1e-10
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9


@pytest.mark.parametrize("r16,r32,eo", [(12, 12, 0), (12, 12, 1), (8, 8, 0), (12, 18, 1), (12, 8, 0)])
def test_fp16_iteration_fp32_corrections(wd, r16, r32, eo):
    """FP16 inner iterations corrected in FP32 between the FP64 reliable updates, on FP32
    links compressed as the FP64 copy (18) or as the FP16 copy; with a third compression
    on the FP32 copy there are no corrections.  Every variant reaches the oracle's solution."""
    dims, kappa = (6, 4, 4, 8), 0.124
    U = gen.haar_links(dims, seed=45)
    b = gen.gaussian_source(dims, seed=46)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=18)
    lat.set_link_compression(2, r16)
    if r32 != 18:
        lat.set_link_compression(1, r32)
    fx = lat.new_field()
    res, st = lat.cg(kappa, lat.pack(b), fx, tol=1e-10, inner=2, precondition=eo)
    assert st == 0 and res[0]["true_rel_resid"] <= 1e-10 and res[0]["reliable_updates"] >= 1
    assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9
    assert (res[0]["inner_corrections"] > 0) == (r32 in (18, r16))


def test_link_compression_rules(wd):
    dims, kappa = (4, 4, 4, 4), 0.12
    U = gen.haar_links(dims, seed=43)
    b = gen.gaussian_source(dims, seed=44)
    lat = wd.Lattice(dims)
    with pytest.raises(wd.WDError) as e:
        lat.set_link_compression(1, 12)  # no gauge field yet
    assert e.value.status == 8
    lat.set_gauge(U, recon=12)
    with pytest.raises(wd.WDError) as e:
        lat.set_link_compression(1, 10)
    assert e.value.status == 1
    lat.set_link_compression(1, 18)  # compressed FP64 links with whole inner links: refused by the solver
    res, st = lat.cg(kappa, lat.pack(b), lat.new_field(), tol=1e-10, inner=1, raise_on_fail=False)
    assert st == 1
    res, st = lat.cg(kappa, lat.pack(b), lat.new_field(), tol=1e-10, inner=0)  # plain FP64 is fine
    assert st == 0
    res, st = wd.cg_batched([lat], [kappa], [lat.pack(b)], [lat.new_field()], tol=1e-10, inner=1)
    assert st == 1
    lat.set_gauge(U, recon=12)  # resets every precision
    assert lat.cg(kappa, lat.pack(b), lat.new_field(), tol=1e-10, inner=1)[1] == 0
    ul = wd.Lattice(dims)
    ul.set_gauge(gen.unit_links(dims))
    with pytest.raises(wd.WDError) as e:
        ul.set_link_compression(1, 8)
    assert e.value.status == 1
    ul.set_link_compression(1, 12)
    o = ul.new_field(1)
    ul.apply(kappa, ul.pack(b, 1), o, 1)
    assert oracle.rel_err(ul.unpack(o, 1), oracle.apply_D(gen.unit_links(dims), b, kappa, dims)) < 2e-6


def test_multi_rhs_with_compressed_inner_links(wd):
    """Three right-hand sides, FP32 inner CG with recon-12 links beside whole FP64 links,
    with and without even-odd: every column reaches the oracle solution."""
    dims, kappa = (4, 4, 6, 4), 0.12
    U = gen.haar_links(dims, seed=45)
    B = gen.gaussian_source(dims, seed=46, nrhs=3)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    lat.set_link_compression(1, 12)
    for eo in (0, 1):
        fx = lat.new_field(nrhs=3)
        res, st = lat.cg(kappa, lat.pack(B), fx, tol=1e-10, inner=1, nrhs=3, precondition=eo)
        assert st == 0 and all(r["true_rel_resid"] <= 1e-10 for r in res)
        X = lat.unpack(fx, nrhs=3, squeeze=False)
        for j in range(3):
            x_ref, _ = ref_solution(U, B[j], kappa, dims)
            assert oracle.rel_err(X[j], x_ref) < 1e-9, (eo, j)


def oracle_residuals(U, b, x, kappa, dims):
    """(||b - D x|| / ||b||, ||D^dag (b - D x)|| / ||D^dag b||) with the oracle's operator."""
    r = b - oracle.apply_D(U, x, kappa, dims)
    db = oracle.apply_Ddag(U, b, kappa, dims)
    return (float(np.linalg.norm(r) / np.linalg.norm(b)),
            float(np.linalg.norm(oracle.apply_Ddag(U, r, kappa, dims)) / np.linalg.norm(db)))


@pytest.mark.parametrize("inner", [1, 2, 3])
@pytest.mark.parametrize("max_iter", [10000, 7])
def test_mixed_reported_residuals_are_those_of_x(wd, inner, max_iter):
    """Mixed precision on the full lattice: when every right-hand side stops at a reliable
    update, that update is the final check.  The residuals reported must still be those of
    the returned x, recomputed here with the oracle's operator; a zero source among the rows
    (stopped at the setup) makes the final check run for all of them."""
    dims, kappa = (4, 6, 4, 8), 0.12
    U = gen.haar_links(dims, seed=21)
    B = gen.gaussian_source(dims, seed=22, nrhs=3)
    B[2] = 0.0
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    for rows in (2, 3):
        fb, fx = lat.pack(B[:rows]), lat.new_field(nrhs=rows)
        res, st = lat.cg(kappa, fb, fx, tol=1e-10, nrhs=rows, inner=inner, max_iter=max_iter,
                         raise_on_fail=False)
        X = lat.unpack(fx, nrhs=rows, squeeze=False)
        assert st == (0 if max_iter > 100 else 4), res
        for j in range(2):
            rb, rn = oracle_residuals(U, B[j], X[j], kappa, dims)
            tol = 1e-3 if max_iter > 100 else 1e-6
            assert res[j]["true_rel_resid"] == pytest.approx(rn, rel=tol), (rows, j)
            assert res[j]["true_rel_resid_b"] == pytest.approx(rb, rel=tol), (rows, j)
            if max_iter > 100:
                assert rn <= 1.01e-10
        if rows == 3:
            assert not X[2].any() and res[2]["true_rel_resid"] == 0.0


@pytest.mark.parametrize("inner", [0, 1, 2, 3])
@pytest.mark.parametrize("eo", [0, 1])
def test_system_residual_stop_rule(wd, inner, eo):
    """stop_rule = 1: tol applies to ||b - D x|| / ||b|| (the residual of the paper's listing,
    section 2.2).  The reported residual is that of the returned x (recomputed here with the
    oracle's operator) and meets tol; the solution matches the oracle's."""
    dims, kappa = (6, 4, 6, 8), 0.124
    U = gen.smoothed_links(dims, seed=23, eps=0.4)
    b = gen.gaussian_source(dims, seed=24)
    x_ref, _ = ref_solution(U, b, kappa, dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(b), lat.new_field()
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, precondition=eo, stop_rule=1)
    assert st == 0, res
    x = lat.unpack(fx)
    rb, rn = oracle_residuals(U, b, x, kappa, dims)
    assert res[0]["true_rel_resid_b"] == pytest.approx(rb, rel=1e-3)
    assert rb <= 1.01e-10
    assert oracle.rel_err(x, x_ref) < 1e-9


def test_stop_rule_arguments(wd):
    dims = (4, 4, 4, 4)
    lat = wd.Lattice(dims)
    lat.set_gauge(gen.haar_links(dims, seed=1))
    b = lat.pack(gen.gaussian_source(dims, seed=2))
    _, st = lat.cg(0.12, b, lat.new_field(), stop_rule=2, raise_on_fail=False)
    assert st == 1
    _, st = lat.cg(0.12, b, lat.new_field(), block=1, stop_rule=1, raise_on_fail=False)
    assert st == 1
    # CGNE already iterates b - D x: the rule changes nothing there
    fx1, fx2 = lat.new_field(), lat.new_field()
    r1, _ = lat.cg(0.12, b, fx1, normal_eq=1)
    r2, _ = lat.cg(0.12, b, fx2, normal_eq=1, stop_rule=1)
    assert r1[0]["iters"] == r2[0]["iters"]
    assert np.array_equal(lat.unpack(fx1), lat.unpack(fx2))


def test_kappa_scan_keeps_graph_cache_bounded(wd):
    """kappa is part of a solver graph's signature: a scan over 20 values (more than the 16
    graphs a context keeps) evicts the least recently used graphs and every solve still
    gives the oracle's solution, also a kappa whose graph was evicted and is rebuilt."""
    dims = (4, 4, 4, 4)
    U = gen.haar_links(dims, seed=81)
    b = gen.gaussian_source(dims, seed=82)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb = lat.pack(b)
    kappas = [0.10 + 0.00125 * i for i in range(20)] + [0.10]
    for k in kappas:
        fx = lat.new_field()
        res, st = lat.cg(k, fb, fx, tol=1e-10)
        assert st == 0 and res[0]["true_rel_resid"] <= 1e-10
        x_ref, _ = ref_solution(U, b, k, dims)
        assert oracle.rel_err(lat.unpack(fx), x_ref) < 1e-9, k


@pytest.mark.parametrize("inner,nrhs", [(0, 1), (1, 1), (1, 3)])
def test_autotune_cg_keeps_solutions(wd, inner, nrhs):
    """The solver autotuner picks a valid launch shape for the fused CG kernels; solves with
    it give the oracle's solutions, and the plain operator's shape is left as it was."""
    dims, kappa = (8, 8, 4, 8), 0.12
    U = gen.haar_links(dims, seed=83)
    B = gen.gaussian_source(dims, seed=84, nrhs=nrhs)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    plain = lat.autotune(inner, nrhs)
    st_, rt = lat.autotune_cg(inner, nrhs)
    assert st_ in (16, 32, 64, 128, 256) and 1 <= rt <= nrhs and (st_ * rt) % 32 == 0 and st_ * rt <= 256
    assert plain[0] in (16, 32, 64, 128, 256)
    fx = lat.new_field(nrhs=nrhs)
    res, st = lat.cg(kappa, lat.pack(B if nrhs > 1 else B[0]), fx, tol=1e-10, inner=inner, nrhs=nrhs)
    assert st == 0
    X = lat.unpack(fx, nrhs=nrhs, squeeze=False)
    for j in range(nrhs):
        x_ref, _ = ref_solution(U, B[j], kappa, dims)
        assert oracle.rel_err(X[j], x_ref) < 1e-9


def test_fixed_rhs_tile_in_solver(wd):
    """params.rhs_tile fixes the right-hand-side tile of the solver's kernels: same solutions."""
    dims, kappa = (4, 4, 4, 8), 0.12
    U = gen.haar_links(dims, seed=85)
    B = gen.gaussian_source(dims, seed=86, nrhs=5)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb = lat.pack(B)
    xs = {}
    for rt in (0, 1, 2, 5):
        fx = lat.new_field(nrhs=5)
        p = lat.params(tol=1e-10, nrhs=5, rhs_tile=rt, inner=1)
        res = (wd.CGResult * 5)()
        import ctypes
        st = lat.lib.wd_cg_solve(lat.ctx, kappa, ctypes.c_void_p(fb.data_ptr()), ctypes.c_void_p(fx.data_ptr()),
                                 ctypes.byref(p), res)
        assert st == 0 and all(r.true_rel_resid <= 1e-10 for r in res)
        xs[rt] = lat.unpack(fx, nrhs=5, squeeze=False)
    for rt in (1, 2, 5):
        assert oracle.rel_err(xs[rt], xs[0]) < 1e-9
