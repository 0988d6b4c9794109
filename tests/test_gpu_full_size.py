"""Solvers on the full-size workloads, in the launch configuration bench.py times.

The GPU solutions are checked against the oracle: on 16^4 against the oracle's own CG
solution (element by element, the 1e-9 solution bar), on the larger lattices through the
oracle's operator (the true residual b - D x recomputed on the host, and the normal-equation
residual D^dag (b - D x) that CGNR stops on), which holds at any size.

  16^4      Haar links, kappa = 0.12, Gaussian source, plain FP64 CGNR (the default bench)
  32^3x64   smoothed links exp(i 0.4 H), kappa = 0.124: FP32-inner and FP16-storage CG with
            even-odd preconditioning (the fastest mixed-precision variants)
  24^3x48   Haar links, kappa = 0.12: the 12 spin-colour point sources in one multi-RHS solve
"""
import os

import numpy as np
import pytest

import oracle
from paper_1810_04201_gb300 import gen

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def wd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import wd as _wd
    return _wd


def normal_residual(U, b, x, kappa, dims):
    """(||b - D x|| / ||b||, ||D^dag (b - D x)|| / ||D^dag b||) with the oracle's operator."""
    r = b - oracle.apply_D(U, x, kappa, dims)
    rn = oracle.apply_Ddag(U, r, kappa, dims)
    db = oracle.apply_Ddag(U, b, kappa, dims)
    return (float(np.linalg.norm(r) / np.linalg.norm(b)), float(np.linalg.norm(rn) / np.linalg.norm(db)))


def test_c2_fp64_cg_matches_oracle_solution(wd):
    dims, kappa = (16, 16, 16, 16), 0.12
    U = gen.haar_links(dims, 2)
    b = gen.gaussian_source(dims, 2)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    lat.autotune(0, 1)
    fx = lat.new_field()
    res, st = lat.cg(kappa, lat.pack(b), fx, tol=1e-10)
    assert st == 0 and res[0]["true_rel_resid"] <= 1e-10
    x = lat.unpack(fx)
    x_ref, _ = oracle.cgnr(U, b, kappa, dims, tol=1e-13)
    assert oracle.rel_err(x, x_ref) < 1e-9
    _, rn = normal_residual(U, b, x, kappa, dims)
    assert rn <= 1.01e-10


@pytest.mark.parametrize("inner", [1, 2])
def test_c3_mixed_even_odd_residual(wd, inner):
    dims, kappa = (32, 32, 32, 64), 0.124
    U = gen.smoothed_links(dims, 6, eps=0.4)
    b = gen.gaussian_source(dims, 6)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fx = lat.new_field()
    res, st = lat.cg(kappa, lat.pack(b), fx, tol=1e-10, inner=inner, precondition=1)
    assert st == 0 and res[0]["true_rel_resid"] <= 1e-10 and res[0]["reliable_updates"] >= 1
    _, rn = normal_residual(U, b, lat.unpack(fx), kappa, dims)
    assert rn <= 1.01e-10


def test_c4_multi_rhs_point_sources_residual(wd):
    dims, kappa = (24, 24, 24, 48), 0.12
    U = gen.haar_links(dims, 7)
    B = gen.propagator_sources(dims)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb, fx = lat.pack(B), lat.new_field(nrhs=12)
    res, st = lat.cg(kappa, fb, fx, tol=1e-10, nrhs=12, inner=1)
    assert st == 0 and all(r["true_rel_resid"] <= 1e-10 for r in res)
    X = lat.unpack(fx, nrhs=12, squeeze=False)
    for j in (0, 5, 11):
        _, rn = normal_residual(U, B[j], X[j], kappa, dims)
        assert rn <= 1.01e-10, j


def read_c3_reference():
    """The oracle's 32^3 x 64 solution at sampled sites and its error-bound data
    (tests/golden/c3_oracle_reference.txt, written by make_c3_reference.py there)."""
    meta, sites, vals = {}, [], []
    for line in open(os.path.join(GOLDEN, "c3_oracle_reference.txt")):
        if line.startswith("#") or not line.strip():
            continue
        parts = line.split()
        if parts[0] == "site":
            sites.append(int(parts[1]))
            r = np.array(parts[2:], dtype=np.float64)
            vals.append((r[0::2] + 1j * r[1::2]).reshape(4, 3))
        else:
            meta[parts[0]] = float(parts[1])
    return meta, np.array(sites), np.array(vals)


# (inner precision, even-odd, inner-precision link compression); inner 0 is plain FP64 CG
C3_VARIANTS = [(0, 0, 18), (1, 0, 18), (2, 0, 18), (3, 0, 18), (0, 1, 18), (1, 1, 18), (2, 1, 18), (3, 1, 18),
               (1, 1, 12)]


def test_c3_variants_against_oracle_solution(wd):
    """Each 32^3 x 64 solver variant, run with the system-residual stopping rule
    (||b - D x|| <= 1e-10 ||b||), against the oracle's solution (CG to 1e-13): the error at the
    sampled sites, over the norm of the whole oracle solution, stays below the forward-error
    bound cond(D) ||b - D x|| / ||b|| (cond(D) from the oracle's Lanczos estimate of the spectrum
    of D^dag D), and its estimate for the whole field (scaled by sqrt(V / sites)) meets the 1e-9
    solution bar."""
    meta, sites, xref = read_c3_reference()
    dims, kappa = (32, 32, 32, 64), 0.124
    U = gen.smoothed_links(dims, 6, eps=0.4)
    b = gen.gaussian_source(dims, 6)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    fb = lat.pack(b)
    scale = np.sqrt(lat.V / len(sites))
    for inner, eo, rin in C3_VARIANTS:
        if inner:
            lat.set_link_compression(inner, rin)
        fx = lat.new_field()
        res, st = lat.cg(kappa, fb, fx, tol=1e-10, inner=inner, precondition=eo, stop_rule=1)
        assert st == 0 and res[0]["true_rel_resid_b"] <= 1e-10
        x = lat.unpack(fx)
        err = float(np.linalg.norm(x[sites] - xref) / meta["x_norm"])
        bound = meta["cond_D"] * res[0]["true_rel_resid_b"]
        print(f"C3 inner={inner} eo={eo} recon_inner={rin}: ||b-Dx||/||b|| {res[0]['true_rel_resid_b']:.3e}, "
              f"iterations {res[0]['iters']}, sampled relative error {err * scale:.3e} (estimate), "
              f"bound {bound:.3e}")
        assert err <= bound, (inner, eo, rin, err, bound)
        assert err * scale <= 1e-9, (inner, eo, rin, err * scale)
        if inner:
            lat.set_link_compression(inner, 18)
