"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle's C source (a flipped
projector sign, U where U^dag belongs, a transposed link, a dropped
antiperiodic sign, a wrong link site, a dropped hop, a wrong kappa sign, a typo
in a gamma matrix, norms where squared norms belong in CG, D where D^dag belongs
in the recomputed normal residual, that residual divided by |b|), builds it, and
checks that at least one of the pins used in test_oracle_pins fails for it.
The unmodified source passes all of them.  The Lanczos estimate of the
spectrum of D^dag D (Python) gets the same treatment with its own pin.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_1810_04201_gb300 import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "wilson_oracle.c")

MUTATIONS = {
    "clean": None,
    "forward_projector_sign": ("cplx Pf = (alpha == beta ? 1.0 : 0.0) - sign * GAMMA",
                               "cplx Pf = (alpha == beta ? 1.0 : 0.0) + sign * GAMMA"),
    "U_instead_of_Udag": ("conj(Ub[3 * B + A])", "Ub[3 * A + B]"),
    "transposed_forward_link": ("Uf[3 * A + B]", "Uf[3 * B + A]"),
    "no_antiperiodic_sign": ("double bf = (mu == 3 && antiperiodic_t && c[3] == L[3] - 1) ? -1.0 : 1.0;",
                             "double bf = 1.0;"),
    "backward_link_at_n": ("const cplx *Ub = link(U, L, mu, nb);", "const cplx *Ub = link(U, L, mu, n);"),
    "dropped_backward_hop": ("s += bb * Pb * conj(Ub[3 * B + A]) * pb[3 * beta + B];", ""),
    "kappa_sign": ("p0[3 * alpha + A] - kappa * hop[alpha][A]", "p0[3 * alpha + A] + kappa * hop[alpha][A]"),
    "gamma2_typo": ("{{0, 0, I, 0}, {0, 0, 0, -I}, {-I, 0, 0, 0}, {0, I, 0, 0}}",
                    "{{0, 0, I, 0}, {0, 0, 0, I}, {-I, 0, 0, 0}, {0, I, 0, 0}}"),
    "cg_unsquared_norms": ("double alpha = rho / norm2(q, N);", "double alpha = sqrt(rho) / sqrt(norm2(q, N));"),
    "residual_D_instead_of_Ddag": ("oracle_wilson_apply(L, ap, kappa, U, e, De, 1);",
                                   "oracle_wilson_apply(L, ap, kappa, U, e, De, 0);"),
    "normal_residual_over_norm_b": ("info->true_normal_rel = ndb > 0 ? sqrt(nde / ndb) : sqrt(nde);",
                                    "info->true_normal_rel = nb > 0 ? sqrt(nde / nb) : sqrt(nde);"),
}


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("iter_resid", ctypes.c_double),
                ("true_normal_rel", ctypes.c_double), ("true_rel", ctypes.c_double)]


def build_variant(tmp_path, name, mut):
    src = open(SRC).read()
    if mut is not None:
        assert mut[0] in src, name
        src = src.replace(mut[0], mut[1])
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", str(c), "-o", str(so),
                    "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.oracle_wilson_apply.argtypes = [P, I, D, P, P, P, I]
    lib.oracle_gamma.argtypes = [I, P]
    lib.oracle_cgnr.argtypes = [P, I, D, P, P, P, D, I, ctypes.POINTER(Info)]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def apply(lib, U, psi, kappa, dims, ap=True, dagger=False):
    out = np.empty_like(psi)
    lib.oracle_wilson_apply((ctypes.c_int * 4)(*dims), int(ap), kappa, _p(U), _p(psi), _p(out), int(dagger))
    return out


def coords(dims):
    n = np.arange(int(np.prod(dims)))
    c = []
    for L in dims:
        c.append(n % L)
        n = n // L
    return np.stack(c, axis=1)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def pins_pass(lib):
    """True when every pin holds for this compiled copy of the oracle."""
    from test_oracle_pins import paper_gammas
    g = paper_gammas()
    out = np.zeros(32)
    for mu in (0, 1, 2, 3, 5):
        lib.oracle_gamma(mu, _p(out))
        if not np.array_equal((out[0::2] + 1j * out[1::2]).reshape(4, 4), g[mu]):
            return False
    # free-field plane waves, both boundary conditions and both operators
    dims, kappa = (4, 2, 6, 4), 0.13
    c = coords(dims)
    U1 = gen.unit_links(dims)
    rng = np.random.default_rng(3)
    for ap in (True, False):
        for dag in (False, True):
            k = [1, 1, 2, 1]
            p = [2 * np.pi * k[m] / dims[m] for m in range(3)] + [(2 * k[3] + ap) * np.pi / dims[3]]
            u = rng.normal(size=(4, 3)) + 1j * rng.normal(size=(4, 3))
            ph = np.exp(1j * (c @ np.array(p)))
            psi = np.ascontiguousarray(ph[:, None, None] * u[None])
            M = (1 - 2 * kappa * sum(np.cos(x) for x in p)) * np.eye(4) + \
                (-1 if dag else 1) * 2j * kappa * sum(g[m] * np.sin(p[m]) for m in range(4))
            if not np.allclose(apply(lib, U1, psi, kappa, dims, ap, dag), ph[:, None, None] * (M @ u)[None],
                               atol=1e-12):
                return False
    # interacting invariants
    U = gen.haar_links(dims, 11)
    psi = gen.gaussian_source(dims, 12)
    g5 = np.array([1, 1, -1, -1.0])[None, :, None]
    if rel(g5 * apply(lib, U, np.ascontiguousarray(g5 * psi), kappa, dims), apply(lib, U, psi, kappa, dims,
                                                                                    dagger=True)) > 1e-14:
        return False
    G = gen.gauge_transform(dims, 5)
    Up = np.empty_like(U)
    for mu in range(4):
        cf = c.copy()
        cf[:, mu] = (cf[:, mu] + 1) % dims[mu]
        nf = cf[:, 0] + dims[0] * (cf[:, 1] + dims[1] * (cf[:, 2] + dims[2] * cf[:, 3]))
        Up[mu] = G @ U[mu] @ np.conj(np.swapaxes(G[nf], 1, 2))
    psip = np.ascontiguousarray(np.einsum("nab,nsb->nsa", G, psi))
    if rel(apply(lib, np.ascontiguousarray(Up), psip, kappa, dims),
           np.einsum("nab,nsb->nsa", G, apply(lib, U, psi, kappa, dims))) > 1e-13:
        return False
    # CG against LAPACK on 2^4
    d2 = (2, 2, 2, 2)
    U2 = gen.haar_links(d2, 21)
    b2 = gen.gaussian_source(d2, 22)
    x = np.zeros_like(b2)
    info = Info()
    lib.oracle_cgnr((ctypes.c_int * 4)(*d2), 1, 0.12, _p(U2), _p(b2), _p(x), 1e-12, 500, ctypes.byref(info))
    n = b2.size
    Mat = np.empty((n, n), complex)
    e = np.zeros_like(b2)
    for j in range(n):
        e.reshape(-1)[j] = 1
        Mat[:, j] = apply(lib, U2, e, 0.12, d2).reshape(-1)
        e.reshape(-1)[j] = 0
    # the operator itself must also be the true one: compare the dense solve with the CG result
    xd = np.linalg.solve(Mat, b2.reshape(-1)).reshape(b2.shape)
    if not (info.converged and rel(x, xd) < 1e-9):
        return False
    # the recomputed residuals of a far-from-converged x (three iterations) against numpy on Mat
    x3 = np.zeros_like(b2)
    i3 = Info()
    lib.oracle_cgnr((ctypes.c_int * 4)(*d2), 1, 0.12, _p(U2), _p(b2), _p(x3), 1e-14, 3, ctypes.byref(i3))
    r3 = b2.reshape(-1) - Mat @ x3.reshape(-1)
    want_rel = np.linalg.norm(r3) / np.linalg.norm(b2)
    want_normal = np.linalg.norm(Mat.conj().T @ r3) / np.linalg.norm(Mat.conj().T @ b2.reshape(-1))
    if not (np.isclose(i3.true_rel, want_rel, rtol=1e-12) and np.isclose(i3.true_normal_rel, want_normal,
                                                                          rtol=1e-12)):
        return False
    # CG's convergence bound: |r_k| / |r_0| <= 2 sqrt(K) ((sqrt(K) - 1) / (sqrt(K) + 1))^k, K = cond(D^dag D)
    sv = np.linalg.svd(Mat, compute_uv=False)
    rk = sv[0] / sv[-1]
    bound = np.log(2 * rk / 1e-12) / np.log((rk + 1) / (rk - 1))
    return info.iters <= np.ceil(bound)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutation_is_caught(tmp_path, name, monkeypatch):
    monkeypatch.syspath_prepend(os.path.dirname(os.path.abspath(__file__)))
    lib = build_variant(tmp_path, name, MUTATIONS[name])
    ok = pins_pass(lib)
    if name == "clean":
        assert ok
    else:
        assert not ok, f"mutation {name} passed every pin"


# The same for the oracle's Lanczos estimate of the spectrum of D^dag D: each case plants one
# mistake in a copy of the Python function and checks that its pin (the extreme eigenvalues
# of the assembled D^dag D from LAPACK) fails.
LANCZOS_MUTATIONS = {
    "clean": None,
    "two_term_recurrence": ("w -= alpha * q + beta * q_prev", "w -= alpha * q"),
    "shifted_offdiagonal": ("np.array(betas[:len(alphas) - 1])", "np.array(betas[1:len(alphas)])"),
    "unnormalised_vector": ("q_prev, q = q, w / beta", "q_prev, q = q, w"),
}


def lanczos_variant(mut):
    import inspect
    import oracle
    src = inspect.getsource(oracle.normal_extreme_eigs)
    if mut is not None:
        assert mut[0] in src
        src = src.replace(mut[0], mut[1])
    ns = dict(vars(oracle))
    exec(src, ns)
    return ns["normal_extreme_eigs"]


@pytest.mark.parametrize("name", list(LANCZOS_MUTATIONS))
def test_lanczos_mutation_is_caught(name):
    import oracle
    fn = lanczos_variant(LANCZOS_MUTATIONS[name])
    dims = (2, 2, 2, 2)
    U = gen.haar_links(dims, seed=31)
    M = oracle.dense_matrix(U, 0.12, dims)
    ev = np.linalg.eigvalsh(M.conj().T @ M)
    with np.errstate(all="ignore"):
        lo, hi, _ = fn(U, 0.12, dims, steps=M.shape[0], seed=5)
    ok = bool(np.isclose(lo, ev[0], rtol=1e-8) and np.isclose(hi, ev[-1], rtol=1e-10))
    if name == "clean":
        assert ok
    else:
        assert not ok, f"mutation {name} passed the pin"
