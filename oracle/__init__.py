"""CPU oracle for the Wilson-Dirac operator and its CG solvers.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU
baseline use this package; the CUDA library never does and shares no code
with it.  The arithmetic lives in ``wilson_oracle.c`` (plain C99, FP64,
complex.h); this module compiles it with gcc, loads it through ctypes and adds
the dense-matrix checks (numpy / LAPACK) and a Lanczos estimate of the extreme
eigenvalues of D^dag D (the condition number that bounds solution errors).

Paper passages followed (arXiv:1810.04201):
  * section 2.1, Eq. (1)-(3): the operator D, kappa, the projectors 1 +- gamma_mu;
  * section 2.2: gamma5-hermiticity, the normal equations and the CG listing;
  * Appendix A: the gamma matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wilson_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2, no fast-math, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-fno-fast-math",
               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class CGInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("iter_resid", ctypes.c_double),
                ("true_normal_rel", ctypes.c_double), ("true_rel", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
            lib.oracle_gamma.argtypes = [I, P]
            lib.oracle_wilson_apply.argtypes = [P, I, D, P, P, P, I]
            lib.oracle_wilson_apply_sites.argtypes = [P, I, D, P, P, I, P, ctypes.c_longlong, P]
            lib.oracle_normal_apply.argtypes = [P, I, D, P, P, P, P]
            lib.oracle_cgnr.argtypes = [P, I, D, P, P, P, D, I, ctypes.POINTER(CGInfo)]
            lib.oracle_cgne.argtypes = [P, I, D, P, P, P, D, I, ctypes.POINTER(CGInfo)]
            lib.oracle_cgnr.restype = I
            lib.oracle_cgne.restype = I
            lib.oracle_set_threads.argtypes = [I]
            lib.oracle_get_threads.restype = I
            lib.oracle_set_threads(os.cpu_count() or 1)
            _lib = lib
    return _lib


def set_threads(n: int) -> None:
    _load().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(_load().oracle_get_threads())


def _dims(dims):
    return (ctypes.c_int * 4)(*[int(d) for d in dims])


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def gamma(mu: int) -> np.ndarray:
    """The oracle's gamma_mu table (mu = 0..3) or gamma_5 (mu = 5), 4x4 complex."""
    out = np.zeros(32)
    _load().oracle_gamma(int(mu), _ptr(out))
    return (out[0::2] + 1j * out[1::2]).reshape(4, 4)


def apply_D(U, psi, kappa, dims, antiperiodic_t=True, dagger=False):
    """D psi (or D^dag psi): section 2.1, Eq. (1), hopping term with -kappa."""
    U = _c128(U)
    psi = _c128(psi)
    v = int(np.prod(dims))
    assert U.shape == (4, v, 3, 3) and psi.shape == (v, 4, 3)
    out = np.empty_like(psi)
    _load().oracle_wilson_apply(_dims(dims), int(bool(antiperiodic_t)), float(kappa), _ptr(U), _ptr(psi),
                                _ptr(out), int(bool(dagger)))
    return out


def apply_Ddag(U, psi, kappa, dims, antiperiodic_t=True):
    return apply_D(U, psi, kappa, dims, antiperiodic_t, dagger=True)


def apply_D_sites(U, psi, kappa, dims, sites, antiperiodic_t=True, dagger=False):
    """(D psi)(n) at the listed sites only, shape (len(sites), 4, 3)."""
    U = _c128(U)
    psi = _c128(psi)
    s = np.ascontiguousarray(sites, dtype=np.int64)
    out = np.empty((len(s), 4, 3), dtype=np.complex128)
    _load().oracle_wilson_apply_sites(_dims(dims), int(bool(antiperiodic_t)), float(kappa), _ptr(U), _ptr(psi),
                                      int(bool(dagger)), _ptr(s), len(s), _ptr(out))
    return out


def apply_normal(U, psi, kappa, dims, antiperiodic_t=True):
    """D^dag D psi."""
    U = _c128(U)
    psi = _c128(psi)
    out = np.empty_like(psi)
    tmp = np.empty_like(psi)
    _load().oracle_normal_apply(_dims(dims), int(bool(antiperiodic_t)), float(kappa), _ptr(U), _ptr(psi),
                                _ptr(out), _ptr(tmp))
    return out


def _solve(fn, U, b, kappa, dims, tol, max_iter, x0, antiperiodic_t):
    U = _c128(U)
    b = _c128(b)
    x = np.zeros_like(b) if x0 is None else _c128(x0).copy()
    info = CGInfo()
    fn(_dims(dims), int(bool(antiperiodic_t)), float(kappa), _ptr(U), _ptr(b), _ptr(x), float(tol), int(max_iter),
       ctypes.byref(info))
    return x, {"iters": info.iters, "converged": bool(info.converged), "iter_resid": info.iter_resid,
               "true_normal_rel": info.true_normal_rel, "true_rel": info.true_rel}


def cgnr(U, b, kappa, dims, tol=1e-10, max_iter=10000, x0=None, antiperiodic_t=True):
    """Solve D^dag D x = D^dag b by CG (section 2.2, normal equations)."""
    return _solve(_load().oracle_cgnr, U, b, kappa, dims, tol, max_iter, x0, antiperiodic_t)


def cgne(U, b, kappa, dims, tol=1e-10, max_iter=10000, antiperiodic_t=True):
    """Solve D D^dag y = b by CG, x = D^dag y (the paper's listing, section 2.2)."""
    return _solve(_load().oracle_cgne, U, b, kappa, dims, tol, max_iter, None, antiperiodic_t)


def dense_matrix(U, kappa, dims, antiperiodic_t=True, dagger=False):
    """D as an explicit (12V x 12V) matrix, assembled column by column from unit vectors."""
    v = int(np.prod(dims))
    n = 12 * v
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros((v, 4, 3), dtype=np.complex128)
    flat = e.reshape(-1)
    for j in range(n):
        flat[j] = 1.0
        M[:, j] = apply_D(U, e, kappa, dims, antiperiodic_t, dagger).reshape(-1)
        flat[j] = 0.0
    return M


def dense_solve(U, b, kappa, dims, antiperiodic_t=True):
    """x = D^{-1} b by LU (LAPACK zgesv through numpy), for lattices up to a few thousand unknowns."""
    M = dense_matrix(U, kappa, dims, antiperiodic_t)
    x = np.linalg.solve(M, _c128(b).reshape(-1))
    return x.reshape(np.shape(b))


def normal_extreme_eigs(U, kappa, dims, steps, seed=0, antiperiodic_t=True):
    """Estimates of the smallest and largest eigenvalues of D^dag D (hermitian, positive;
    section 2.2), which bound the error of a CG solution: ||x - x*|| / ||x*|| <=
    cond(D) ||b - D x|| / ||b||, cond(D) = sqrt(lambda_max / lambda_min).

    Plain Lanczos without reorthogonalisation from a seeded Gaussian start vector: the
    extreme eigenvalues of the k-step tridiagonal matrix (diagonal alpha_j, off-diagonal
    beta_j) approach those of D^dag D from inside as k grows; lost orthogonality only adds
    copies of eigenvalues that have already converged.  Returns (lambda_min, lambda_max,
    steps taken)."""
    from scipy.linalg import eigh_tridiagonal
    v = int(np.prod(dims))
    rng = np.random.default_rng(seed)
    q = rng.standard_normal((v, 4, 3)) + 1j * rng.standard_normal((v, 4, 3))
    q /= np.linalg.norm(q)
    q_prev = np.zeros_like(q)
    beta = 0.0
    alphas, betas = [], []
    for _ in range(steps):
        w = apply_normal(U, q, kappa, dims, antiperiodic_t)
        alpha = float(np.vdot(q, w).real)
        w -= alpha * q + beta * q_prev
        alphas.append(alpha)
        beta = float(np.linalg.norm(w))
        if beta == 0.0:
            break
        betas.append(beta)
        q_prev, q = q, w / beta
    ev = eigh_tridiagonal(np.array(alphas), np.array(betas[:len(alphas) - 1]), eigvals_only=True)
    return float(ev[0]), float(ev[-1]), len(alphas)


def rel_err(a, b) -> float:
    """||a - b|| / ||b|| (per-field 2-norm)."""
    nb = np.linalg.norm(np.ravel(b))
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / (nb if nb > 0 else 1.0))
