"""The batched persistent solver: many lattices of uneven size and kappa in one
cooperative launch, each solution checked against the oracle."""
import numpy as np
import pytest

import oracle
from paper_1810_04201_gb300 import gen

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (4, 4, 4, 8), (6, 6, 6, 6), (4, 6, 4, 8), (8, 8, 8, 8), (2, 4, 4, 4), (6, 6, 6, 8)]


@pytest.fixture(scope="module")
def wd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import wd as _wd
    return _wd


def make_batch(wd, recon=18):
    kappas = [0.10 + 0.025 * u for u in gen.uniform(5, 5, 0, len(SHAPES))]
    lats, bs, xs, inputs = [], [], [], []
    for i, dims in enumerate(SHAPES):
        U = gen.haar_links(dims, seed=100 + i)
        b = gen.gaussian_source(dims, seed=200 + i)
        lat = wd.Lattice(dims)
        lat.set_gauge(U, recon=recon)
        lats.append(lat)
        bs.append(lat.pack(b))
        xs.append(lat.new_field())
        inputs.append((U, b))
    return lats, kappas, bs, xs, inputs


@pytest.mark.parametrize("inner,recon", [(1, 18), (2, 18), (1, 12), (1, 8)])
def test_batched_matches_oracle(wd, inner, recon):
    lats, kappas, bs, xs, inputs = make_batch(wd, recon)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=inner)
    assert st == 0, res
    for i, (lat, (U, b)) in enumerate(zip(lats, inputs)):
        assert res[i]["status"] == 0 and res[i]["true_rel_resid"] <= 1e-10
        x_ref, _ = oracle.cgnr(U, b, kappas[i], lat.dims, tol=1e-13)
        assert oracle.rel_err(lat.unpack(xs[i]), x_ref) < 1e-9, i
    # uneven work: the lattices needed different iteration counts
    assert len({r["iters"] for r in res}) > 1


def test_batched_same_as_single_solves(wd):
    """A lattice solved in the batch converges like the same lattice solved alone."""
    lats, kappas, bs, xs, inputs = make_batch(wd)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 0
    for i in (0, 4):
        x1 = lats[i].new_field()
        r1, st1 = lats[i].cg(kappas[i], bs[i], x1, tol=1e-10, inner=1)
        assert st1 == 0
        assert oracle.rel_err(lats[i].unpack(xs[i]), lats[i].unpack(x1)) < 1e-9


def test_batched_wait_timeout_is_reported(wd, monkeypatch):
    """A wait that nothing ends runs out: every lattice gets WD_ERR_TIMEOUT, the context stays usable."""
    lats, kappas, bs, xs, inputs = make_batch(wd)
    monkeypatch.setenv("WD_BATCH_STALL_TEST", "1")
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 7 and all(r["status"] == 7 for r in res)
    monkeypatch.delenv("WD_BATCH_STALL_TEST")
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 0


def test_batched_argument_errors(wd):
    lats, kappas, bs, xs, _ = make_batch(wd)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=0)
    assert st == 1
    lats[1].set_gauge(gen.haar_links(lats[1].dims, 3), recon=12)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 1


@pytest.mark.parametrize("inner,rin", [(1, 12), (1, 8), (2, 12)])
def test_batched_whole_fp64_links_compressed_inner(wd, inner, rin):
    """Whole FP64 links beside compressed inner links in the persistent kernel: same solutions."""
    lats, kappas, bs, xs, inputs = make_batch(wd)
    for lat in lats:
        lat.set_link_compression(inner, rin)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=inner)
    assert st == 0, res
    for i, (lat, (U, b)) in enumerate(zip(lats, inputs)):
        assert res[i]["status"] == 0 and res[i]["true_rel_resid"] <= 1e-10
        x_ref, _ = oracle.cgnr(U, b, kappas[i], lat.dims, tol=1e-13)
        assert oracle.rel_err(lat.unpack(xs[i]), x_ref) < 1e-9, i


def test_batched_link_compression_rules(wd):
    """Compressed FP64 links need the same inner compression; every context the same pair."""
    lats, kappas, bs, xs, _ = make_batch(wd, recon=12)
    for lat in lats:
        lat.set_link_compression(1, 18)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 1
    lats, kappas, bs, xs, _ = make_batch(wd)
    lats[2].set_link_compression(1, 12)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 1
    lats[2].set_link_compression(1, 18)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 0


def oracle_residuals(U, b, x, kappa, dims):
    """(||b - D x|| / ||b||, ||D^dag (b - D x)|| / ||D^dag b||) with the oracle's operator."""
    r = b - oracle.apply_D(U, x, kappa, dims)
    db = oracle.apply_Ddag(U, b, kappa, dims)
    return (float(np.linalg.norm(r) / np.linalg.norm(b)),
            float(np.linalg.norm(oracle.apply_Ddag(U, r, kappa, dims)) / np.linalg.norm(db)))


def test_batched_mixed_start_vectors(wd):
    """Zero and nonzero start vectors in one batch: each lattice takes its own setup path,
    converges to the oracle's solution, and reports the oracle's residuals of its x."""
    lats, kappas, bs, xs, inputs = make_batch(wd)
    starts = {}
    for i in (1, 4, 6):
        U, b = inputs[i]
        x_ref, _ = oracle.cgnr(U, b, kappas[i], lats[i].dims, tol=1e-13)
        starts[i] = 0.5 * x_ref if i != 6 else gen.gaussian_source(lats[i].dims, seed=300)
        xs[i] = lats[i].pack(starts[i])
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 0, res
    for i, (lat, (U, b)) in enumerate(zip(lats, inputs)):
        x = lat.unpack(xs[i])
        x_ref, _ = oracle.cgnr(U, b, kappas[i], lat.dims, tol=1e-13)
        assert oracle.rel_err(x, x_ref) < 1e-9, i
        rb, rn = oracle_residuals(U, b, x, kappas[i], lat.dims)
        assert res[i]["true_rel_resid"] == pytest.approx(rn, rel=1e-3), i
        assert res[i]["true_rel_resid_b"] == pytest.approx(rb, rel=1e-3), i
    # a start at half the solution needs fewer iterations than the zero start of the same lattice
    lats2, kappas2, bs2, xs2, _ = make_batch(wd)
    res0, _ = wd.cg_batched(lats2, kappas2, bs2, xs2, tol=1e-10, inner=1)
    assert res[1]["iters"] <= res0[1]["iters"] and res[4]["iters"] <= res0[4]["iters"]


def test_batched_iteration_limit_reports_residual_of_x(wd):
    """Stopped by max_iter: WD_ERR_NOT_CONVERGED, and the reported residuals are those of
    the returned x (the stopping reliable update doubles as the final check)."""
    lats, kappas, bs, xs, inputs = make_batch(wd)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, max_iter=6, inner=1)
    assert st == 4
    for i, (lat, (U, b)) in enumerate(zip(lats, inputs)):
        assert res[i]["status"] == 4 and res[i]["iters"] == 6 and res[i]["reliable_updates"] >= 1
        rb, rn = oracle_residuals(U, b, lat.unpack(xs[i]), kappas[i], lat.dims)
        assert rn > 1e-10
        assert res[i]["true_rel_resid"] == pytest.approx(rn, rel=1e-6), i
        assert res[i]["true_rel_resid_b"] == pytest.approx(rb, rel=1e-6), i


@pytest.mark.parametrize("rin", [18, 12])
def test_batched_full_c5_workload(wd, rin):
    """The 64-lattice uneven workload the bench times (shapes from {8^4, 8^3x16, 12^4, 12^3x24,
    16^4}, kappa in [0.10, 0.125], per-lattice seeds 100 + i; 1.86 M sites, many tiles per
    lattice), in its launch configuration: FP32 inner iterations, whole FP64 links, inner links
    whole or recon-12.  Every lattice's solution is checked through the oracle's operator (the
    residuals b - D x and D^dag (b - D x) recomputed on the host, which must be the ones the
    library reports and meet the tolerance), and two of them, a 16^4 and a 12^3 x 24, element by
    element against the oracle's own CG solution."""
    shapes, kappas, seeds = gen.batch_workload(64)
    lats, bs, xs, inputs = [], [], [], []
    for dims, seed in zip(shapes, seeds):
        U = gen.haar_links(dims, seed)
        b = gen.gaussian_source(dims, seed)
        lat = wd.Lattice(dims)
        lat.set_gauge(U)
        if rin != 18:
            lat.set_link_compression(1, rin)
        lats.append(lat)
        bs.append(lat.pack(b))
        xs.append(lat.new_field())
        inputs.append((U, b))
    assert sum(l.V for l in lats) > 1_500_000 and {(16, 16, 16, 16), (12, 12, 12, 24)} <= set(shapes)
    res, st = wd.cg_batched(lats, kappas, bs, xs, tol=1e-10, inner=1)
    assert st == 0, [r for r in res if r["status"] != 0][:3]
    for i, (lat, (U, b)) in enumerate(zip(lats, inputs)):
        x = lat.unpack(xs[i])
        rb, rn = oracle_residuals(U, b, x, kappas[i], lat.dims)
        assert res[i]["status"] == 0 and rn <= 1.01e-10, (i, rn)
        assert res[i]["true_rel_resid"] == pytest.approx(rn, rel=1e-3), i
        assert res[i]["true_rel_resid_b"] == pytest.approx(rb, rel=1e-3), i
    for dims in ((16, 16, 16, 16), (12, 12, 12, 24)):
        i = shapes.index(dims)
        U, b = inputs[i]
        x_ref, _ = oracle.cgnr(U, b, kappas[i], dims, tol=1e-13)
        assert oracle.rel_err(lats[i].unpack(xs[i]), x_ref) < 1e-9, (i, dims)
    assert len({r["iters"] for r in res}) > 1
