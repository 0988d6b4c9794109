"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks a printed
value (the gamma matrices of Appendix A), a closed form (free-field plane
waves and spectrum), an invariant (gamma5-hermiticity, adjointness, gauge
covariance, the staggered-sign identity, hermiticity and positivity of
D^dag D), a special case (kappa = 0, locality) or a textbook library routine
(dense LU through LAPACK) -- chosen so that a dropped term, a wrong sign, a
wrong link index or a transposed operand fails at least one of them.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1810_04201_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_gammas():
    """Parse the Appendix A matrices stored in tests/golden."""
    tok = {"0": 0, "1": 1, "-1": -1, "i": 1j, "-i": -1j}
    mats, cur, key = {}, None, None
    for line in open(os.path.join(GOLDEN, "gamma_appendix_A.txt")):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("gamma"):
            key = int(line.split()[1])
            cur = []
            mats[key] = cur
        else:
            cur.append([tok[t] for t in line.split()])
    return {k: np.array(v, dtype=np.complex128) for k, v in mats.items()}


def coords(dims):
    v = int(np.prod(dims))
    n = np.arange(v)
    c = []
    for L in dims:
        c.append(n % L)
        n = n // L
    return np.stack(c, axis=1)


def inner(a, b):
    return np.vdot(np.ravel(a), np.ravel(b))


# --------------------------------------------------------------------- gamma table
def test_gamma_table_is_appendix_A():
    g = paper_gammas()
    for mu in (0, 1, 2, 3, 5):
        np.testing.assert_array_equal(oracle.gamma(mu), g[mu])


def test_clifford_algebra_and_gamma5():
    g = [oracle.gamma(mu) for mu in range(4)]
    I4 = np.eye(4)
    for a in range(4):
        np.testing.assert_allclose(g[a], g[a].conj().T, atol=0)  # hermitian
        for b in range(4):
            np.testing.assert_allclose(g[a] @ g[b] + g[b] @ g[a], 2 * (a == b) * I4, atol=1e-15)
    np.testing.assert_allclose(g[0] @ g[1] @ g[2] @ g[3], oracle.gamma(5), atol=1e-15)


def test_projectors_have_rank_two():
    # section 2.1: lower spin components are a rescaling of the upper ones, so 1 +- gamma_mu has rank 2
    for mu in range(4):
        for s in (+1, -1):
            P = np.eye(4) + s * oracle.gamma(mu)
            assert np.linalg.matrix_rank(P) == 2
            np.testing.assert_allclose((P / 2) @ (P / 2), P / 2, atol=1e-15)


# --------------------------------------------------------------------- free field
@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (3, 2, 5, 6), (2, 6, 4, 2)])
@pytest.mark.parametrize("antiperiodic", [True, False])
@pytest.mark.parametrize("dagger", [False, True])
def test_free_field_plane_wave(dims, antiperiodic, dagger):
    """U = 1: D e^{ipx} u = [(1 - 2k sum cos p) + 2ik sum gamma sin p] e^{ipx} u (D^dag: -2ik...)."""
    kappa = 0.137
    g = paper_gammas()
    c = coords(dims)
    U = gen.unit_links(dims)
    rng = np.random.default_rng(7)
    for trial in range(3):
        k = [rng.integers(0, L) for L in dims]
        p = [2 * np.pi * k[mu] / dims[mu] for mu in range(3)]
        p.append((2 * k[3] + (1 if antiperiodic else 0)) * np.pi / dims[3])
        u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
        phase = np.exp(1j * (c @ np.array(p)))
        psi = phase[:, None, None] * u[None]
        out = oracle.apply_D(U, psi, kappa, dims, antiperiodic, dagger)
        M = (1 - 2 * kappa * sum(np.cos(x) for x in p)) * np.eye(4)
        sgn = -1 if dagger else 1
        M = M + sgn * 2j * kappa * sum(g[mu] * np.sin(p[mu]) for mu in range(4))
        expect = phase[:, None, None] * (M @ u)[None]
        np.testing.assert_allclose(out, expect, atol=1e-13)


def test_free_field_spectrum():
    """Eigenvalues 1 - 2k sum cos p +- 2ik sqrt(sum sin^2 p), each six times (basis independent)."""
    dims, kappa = (2, 4, 2, 4), 0.12
    U = gen.unit_links(dims)
    ev = np.linalg.eigvals(oracle.dense_matrix(U, kappa, dims))
    expect = []
    for k0 in range(dims[0]):
        for k1 in range(dims[1]):
            for k2 in range(dims[2]):
                for k3 in range(dims[3]):
                    p = [2 * np.pi * k0 / dims[0], 2 * np.pi * k1 / dims[1], 2 * np.pi * k2 / dims[2],
                         (2 * k3 + 1) * np.pi / dims[3]]
                    re = 1 - 2 * kappa * sum(np.cos(x) for x in p)
                    im = 2 * kappa * np.sqrt(sum(np.sin(x) ** 2 for x in p))
                    expect += [re + 1j * im] * 6 + [re - 1j * im] * 6
    expect = np.array(expect)
    key = lambda z: (np.round(z.real, 9), np.round(z.imag, 9))
    a = np.array(sorted(ev, key=key))
    b = np.array(sorted(expect, key=key))
    np.testing.assert_allclose(a, b, atol=1e-10)


# --------------------------------------------------------------------- invariants
DIMS = (4, 6, 2, 4)


@pytest.fixture(scope="module")
def field():
    U = gen.haar_links(DIMS, seed=11)
    psi = gen.gaussian_source(DIMS, seed=12)
    phi = gen.gaussian_source(DIMS, seed=13)
    return U, psi, phi


def test_gamma5_hermiticity(field):
    # section 2.2: gamma5 D gamma5 = D^dag
    U, psi, _ = field
    g5 = np.array([1, 1, -1, -1], dtype=float)[None, :, None]
    lhs = g5 * oracle.apply_D(U, g5 * psi, 0.12, DIMS)
    rhs = oracle.apply_Ddag(U, psi, 0.12, DIMS)
    assert oracle.rel_err(lhs, rhs) < 1e-15


def test_adjointness(field):
    U, psi, phi = field
    a = inner(phi, oracle.apply_D(U, psi, 0.12, DIMS))
    b = inner(oracle.apply_Ddag(U, phi, 0.12, DIMS), psi)
    assert abs(a - b) < 1e-12 * abs(a)


@pytest.mark.parametrize("antiperiodic", [True, False])
def test_gauge_covariance(field, antiperiodic):
    U, psi, _ = field
    G = gen.gauge_transform(DIMS, seed=5)
    c = coords(DIMS)
    V = len(c)
    Up = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % DIMS[mu]
        nf = cf[:, 0] + DIMS[0] * (cf[:, 1] + DIMS[1] * (cf[:, 2] + DIMS[2] * cf[:, 3]))
        Up[mu] = G @ U[mu] @ np.conj(np.swapaxes(G[nf], 1, 2))
    psip = np.einsum("nab,nsb->nsa", G, psi)
    lhs = oracle.apply_D(Up, psip, 0.12, DIMS, antiperiodic)
    rhs = np.einsum("nab,nsb->nsa", G, oracle.apply_D(U, psi, 0.12, DIMS, antiperiodic))
    assert oracle.rel_err(lhs, rhs) < 1e-14
    assert V == int(np.prod(DIMS))


def test_staggered_sign_identity(field):
    """eps D(kappa) eps = D(-kappa), eps(n) = (-1)^(x+y+z+t): the paper's +kappa form (Eq. 1)."""
    U, psi, _ = field
    eps = ((-1.0) ** coords(DIMS).sum(axis=1))[:, None, None]
    lhs = eps * oracle.apply_D(U, eps * psi, 0.12, DIMS)
    rhs = oracle.apply_D(U, psi, -0.12, DIMS)
    assert oracle.rel_err(lhs, rhs) < 1e-15


def test_kappa_zero_is_identity(field):
    U, psi, _ = field
    np.testing.assert_array_equal(oracle.apply_D(U, psi, 0.0, DIMS), psi)


def test_locality(field):
    """A delta source reaches only its 8 neighbours; one changed link U_mu(m) changes only sites m, m+mu."""
    U, _, _ = field
    V = int(np.prod(DIMS))
    c = coords(DIMS)
    s = 37
    delta = np.zeros((V, 4, 3), complex)
    delta[s] = np.arange(12).reshape(4, 3) + 1j
    out = oracle.apply_D(U, delta, 0.12, DIMS)
    nz = set(np.nonzero(np.abs(out).sum(axis=(1, 2)) > 0)[0].tolist())
    expect = {s}
    for mu in range(4):
        for d in (1, -1):
            cc = c[s].copy()
            cc[mu] = (cc[mu] + d) % DIMS[mu]
            expect.add(int(cc[0] + DIMS[0] * (cc[1] + DIMS[1] * (cc[2] + DIMS[2] * cc[3]))))
    assert nz == expect
    psi = gen.gaussian_source(DIMS, seed=3)
    m, mu = 29, 2
    U2 = U.copy()
    U2[mu, m] = gen.haar_su3(77, 1)[0]
    diff = np.abs(oracle.apply_D(U2, psi, 0.12, DIMS) - oracle.apply_D(U, psi, 0.12, DIMS)).sum(axis=(1, 2))
    cc = c[m].copy()
    cc[mu] = (cc[mu] + 1) % DIMS[mu]
    mf = int(cc[0] + DIMS[0] * (cc[1] + DIMS[1] * (cc[2] + DIMS[2] * cc[3])))
    assert set(np.nonzero(diff > 0)[0].tolist()) == {m, mf}


def test_normal_operator_hermitian_positive(field):
    U, psi, phi = field
    a = inner(phi, oracle.apply_normal(U, psi, 0.12, DIMS))
    b = np.conj(inner(psi, oracle.apply_normal(U, phi, 0.12, DIMS)))
    assert abs(a - b) < 1e-12 * abs(a)
    q = inner(psi, oracle.apply_normal(U, psi, 0.12, DIMS))
    assert abs(q.imag) < 1e-12 * q.real and q.real > 0
    dpsi = oracle.apply_D(U, psi, 0.12, DIMS)
    assert abs(q.real - np.vdot(dpsi, dpsi).real) < 1e-12 * q.real


def test_apply_sites_matches_full(field):
    U, psi, _ = field
    full = oracle.apply_D(U, psi, 0.12, DIMS)
    sites = [0, 5, 77, int(np.prod(DIMS)) - 1]
    np.testing.assert_array_equal(oracle.apply_D_sites(U, psi, 0.12, DIMS, sites), full[sites])


# --------------------------------------------------------------------- solvers
@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_cgnr_matches_dense_lu_small(dims):
    U = gen.haar_links(dims, seed=21)
    b = gen.gaussian_source(dims, seed=22)
    x, info = oracle.cgnr(U, b, 0.12, dims, tol=1e-12)
    assert info["converged"] and info["true_normal_rel"] < 2e-12
    xd = oracle.dense_solve(U, b, 0.12, dims)
    assert oracle.rel_err(x, xd) < 1e-10
    assert info["true_rel"] < 1e-10


@pytest.mark.slow
def test_cgnr_matches_dense_lu_4x4():
    dims = (4, 4, 4, 4)
    U = gen.haar_links(dims, seed=1)
    b = gen.gaussian_source(dims, seed=1)
    x, info = oracle.cgnr(U, b, 0.12, dims, tol=1e-10)
    assert info["converged"] and info["true_normal_rel"] <= 1e-10 * 1.01
    xd = oracle.dense_solve(U, b, 0.12, dims)
    assert oracle.rel_err(x, xd) < 1e-9


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4), (4, 4, 2, 2)])
def test_cg_within_chebyshev_bound(dims):
    """CG on D^dag D reaches |r_k|/|r_0| <= eps within ln(2 sqrt(K)/eps) / ln((sqrt(K)+1)/(sqrt(K)-1))
    iterations, K = cond(D^dag D) = (s_max / s_min)^2 from LAPACK's SVD of the assembled D."""
    U = gen.haar_links(dims, seed=21)
    b = gen.gaussian_source(dims, seed=22)
    _, info = oracle.cgnr(U, b, 0.12, dims, tol=1e-12)
    sv = np.linalg.svd(oracle.dense_matrix(U, 0.12, dims), compute_uv=False)
    rk = sv[0] / sv[-1]
    bound = np.log(2 * rk / 1e-12) / np.log((rk + 1) / (rk - 1))
    assert info["converged"] and info["iters"] <= np.ceil(bound)


def test_cgne_equals_cgnr():
    dims = (4, 2, 4, 4)
    U = gen.haar_links(dims, seed=31)
    b = gen.gaussian_source(dims, seed=32)
    x1, i1 = oracle.cgnr(U, b, 0.11, dims, tol=1e-12)
    x2, i2 = oracle.cgne(U, b, 0.11, dims, tol=1e-12)
    assert i1["converged"] and i2["converged"]
    assert oracle.rel_err(x1, x2) < 1e-10
    assert i2["true_rel"] < 1e-11


def test_cgnr_initial_guess_resume():
    dims = (2, 2, 4, 4)
    U = gen.haar_links(dims, seed=41)
    b = gen.gaussian_source(dims, seed=42)
    xa, _ = oracle.cgnr(U, b, 0.12, dims, tol=1e-4)
    xb, ib = oracle.cgnr(U, b, 0.12, dims, tol=1e-12, x0=xa)
    xc, ic = oracle.cgnr(U, b, 0.12, dims, tol=1e-12)
    assert ib["iters"] < ic["iters"]
    assert oracle.rel_err(xb, xc) < 1e-10


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
@pytest.mark.parametrize("case", ["cgnr_start_vector", "cgnr_three_steps", "cgne_three_steps"])
def test_recomputed_residuals_match_dense_matrix(dims, case):
    """The residuals the solvers report for the x they return (section 2.2: r = b - D x for the
    system, D^dag r for the normal equations) against numpy on the assembled matrix M:
    ||b - M x|| / ||b|| and ||M^H (b - M x)|| / ||M^H b||.  The x is far from converged (a random
    start vector with no iteration, or three iterations), so the two residuals are O(1) and differ."""
    kappa = 0.12
    U = gen.haar_links(dims, seed=51)
    b = gen.gaussian_source(dims, seed=52)
    if case == "cgnr_start_vector":
        x0 = gen.gaussian_source(dims, seed=53)
        x, info = oracle.cgnr(U, b, kappa, dims, tol=1e-14, max_iter=0, x0=x0)
        np.testing.assert_array_equal(x, x0)
    elif case == "cgnr_three_steps":
        x, info = oracle.cgnr(U, b, kappa, dims, tol=1e-14, max_iter=3)
    else:
        x, info = oracle.cgne(U, b, kappa, dims, tol=1e-14, max_iter=3)
    assert not info["converged"]
    M = oracle.dense_matrix(U, kappa, dims)
    bf, xf = b.reshape(-1), x.reshape(-1)
    r = bf - M @ xf
    want_rel = np.linalg.norm(r) / np.linalg.norm(bf)
    want_normal = np.linalg.norm(M.conj().T @ r) / np.linalg.norm(M.conj().T @ bf)
    assert want_rel > 1e-3 and want_normal > 1e-3 and abs(want_rel / want_normal - 1) > 1e-3
    assert info["true_rel"] == pytest.approx(want_rel, rel=1e-12)
    assert info["true_normal_rel"] == pytest.approx(want_normal, rel=1e-12)


def test_cg_zero_source():
    dims = (2, 2, 2, 2)
    U = gen.haar_links(dims, seed=1)
    x, info = oracle.cgnr(U, np.zeros((16, 4, 3), complex), 0.12, dims)
    assert info["iters"] == 0 and np.all(x == 0)


def test_paper_stencil_byte_count():
    """Section 2.4: 8 links and 9 spinors per stencil are (9*24 + 8*18) * 8 = 2880 input bytes."""
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_counts.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    spinor_reals, link_reals = 4 * 3 * 2, 3 * 3 * 2
    assert (9 * spinor_reals + 8 * link_reals) * 8 == vals["stencil_input_bytes"]
    # 16 SU(3) x colour-vector products, each 9 complex multiply-adds of 8 flops (section 6.4, stage 3)
    assert 16 * 9 * 8 == vals["su3_mult_flops"]


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (2, 2, 2, 4)])
def test_lanczos_extremes_match_dense_spectrum(dims):
    """The Lanczos estimate of the extreme eigenvalues of D^dag D (the condition-number
    bound on CG solution errors) against LAPACK's eigenvalues of the assembled D^dag D:
    exact once the steps reach the dimension, and inside the spectrum before that
    (Ritz values interlace)."""
    U = gen.haar_links(dims, seed=31)
    M = oracle.dense_matrix(U, 0.12, dims)
    ev = np.linalg.eigvalsh(M.conj().T @ M)
    n = M.shape[0]
    lo, hi, k = oracle.normal_extreme_eigs(U, 0.12, dims, steps=n, seed=5)
    assert k == n
    assert lo == pytest.approx(ev[0], rel=1e-8) and hi == pytest.approx(ev[-1], rel=1e-10)
    lo, hi, k = oracle.normal_extreme_eigs(U, 0.12, dims, steps=n // 6, seed=5)
    assert ev[0] * (1 - 1e-12) <= lo and hi <= ev[-1] * (1 + 1e-12)
    assert hi > 0.9 * ev[-1]
