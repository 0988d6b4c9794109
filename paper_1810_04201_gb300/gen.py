"""Seeded synthetic inputs for the Wilson-Dirac operator and its solvers.

This module is the one piece of code that both the CPU oracle's tests and the
CUDA path use.  It holds no arithmetic of the method itself (no Dirac operator,
no projector, no solver step): it only draws gauge links and sources.

Random numbers come from a counter-based generator so that any slice of a
stream can be regenerated independently and identically on every machine:

* SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
  generators", OOPSLA 2014) maps the 64-bit counter ``key + (i + 1) * GOLDEN``
  to a 64-bit output ``z`` through the published finaliser
  ``z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27;
  z *= 0x94D049BB133111EB; z ^= z >> 31``.
* A uniform double in (0, 1) is ``((z >> 11) + 0.5) * 2**-53``.
* Normal deviates use the Box-Muller transform on consecutive uniform pairs.

Streams are keyed by ``(seed, stream)``; each stream id below names one kind of
draw, so links and sources of the same seed are independent.

Layouts (canonical, the library's boundary layout):

* links ``U[mu][n][A][B]``: complex128 array of shape ``(4, V, 3, 3)``, row A,
  column B, ``U_mu(n)`` sits on the edge from ``n`` to ``n + mu`` (the paper's
  section 2.1, links on the forward edges);
* spinors ``psi[n][alpha][A]``: complex128 array of shape ``(V, 4, 3)``
  (spin-major, colour-minor, the ``su3_spinor`` structure of section 6.1);
* site index ``n = x + Lx * (y + Ly * (z + Lz * t))``, mu = 0, 1, 2, 3 = x, y, z, t.

Workload recipes (inputs shaped like the paper's single-node lattices):

* Haar-random SU(3) links: 3x3 complex Gaussian -> Gram-Schmidt (positive
  diagonal of R) -> divide by the principal cube root of the determinant.
* Smoothed links ``U = exp(i eps H)``, ``H = sum_a w_a lambda_a / 2`` with
  ``w_a ~ N(0, 1)`` and the eight Gell-Mann matrices ``lambda_a``.
* Gaussian sources: real and imaginary parts ~ N(0, 1/2) per component.
* Point sources: one non-zero entry (section 2.3: "a single non-zero entry set
  to one").
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids
STREAM_HAAR = 1
STREAM_ALGEBRA = 2
STREAM_SOURCE = 3
STREAM_GAUGE_TRANSFORM = 4
STREAM_MISC = 5

_CHUNK = 1 << 20  # matrices per generation chunk (bounds host memory)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    a = np.array([(int(seed) * 0x100000001B3 + int(stream) * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix64(a)[0]


def uniform(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Uniform doubles in (0, 1) for counters ``start .. start + n - 1``."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = _key(seed, stream) + i * _GOLDEN
        z = _mix64(z)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, stream: int, start: int, n: int) -> np.ndarray:
    """Standard normal deviates; deviate k uses uniforms 2k and 2k+1 of the stream."""
    k0 = start // 2
    m = (start + n + 1) // 2 - k0 + 1
    u = uniform(seed, stream, 2 * k0, 2 * m)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    g = np.empty(2 * m)
    g[0::2] = r * np.cos(2.0 * np.pi * u2)
    g[1::2] = r * np.sin(2.0 * np.pi * u2)
    off = start - 2 * k0
    return g[off:off + n]


def volume(dims) -> int:
    d = [int(v) for v in dims]
    return d[0] * d[1] * d[2] * d[3]


def _complex_normal(seed, stream, start, n, var=1.0):
    g = normal(seed, stream, 2 * start, 2 * n)
    s = np.sqrt(var / 2.0)
    return (g[0::2] + 1j * g[1::2]) * s


def _gram_schmidt_rows(z: np.ndarray) -> np.ndarray:
    def proj(u, w):
        return np.sum(np.conj(u) * w, axis=1, keepdims=True) * u

    def unit(u):
        return u / np.linalg.norm(u, axis=1, keepdims=True)

    v0 = unit(z[:, 0, :])
    v1 = z[:, 1, :] - proj(v0, z[:, 1, :])
    v1 = unit(v1 - proj(v0, v1))
    v2 = z[:, 2, :] - proj(v0, z[:, 2, :]) - proj(v1, z[:, 2, :])
    v2 = unit(v2 - proj(v0, v2) - proj(v1, v2))
    return np.stack([v0, v1, v2], axis=1)


def _haar_su3_chunk(seed: int, start: int, n: int) -> np.ndarray:
    """Gram-Schmidt on the rows (re-orthogonalised once; positive R diagonal => Haar on U(3)),
    then removal of the determinant phase by its principal cube root."""
    z = _complex_normal(seed, STREAM_HAAR, 9 * start, 9 * n).reshape(n, 3, 3)
    q = _gram_schmidt_rows(z)
    det = np.linalg.det(q)
    phase = np.exp(-1j * np.angle(det) / 3.0)
    return q * phase[:, None, None]


def haar_su3(seed: int, n: int) -> np.ndarray:
    """``n`` Haar-random SU(3) matrices, shape (n, 3, 3)."""
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        out[s:s + m] = _haar_su3_chunk(seed, s, m)
    return out


def gell_mann() -> np.ndarray:
    """The eight Gell-Mann matrices, shape (8, 3, 3)."""
    lam = np.zeros((8, 3, 3), dtype=np.complex128)
    lam[0][0, 1] = lam[0][1, 0] = 1
    lam[1][0, 1], lam[1][1, 0] = -1j, 1j
    lam[2][0, 0], lam[2][1, 1] = 1, -1
    lam[3][0, 2] = lam[3][2, 0] = 1
    lam[4][0, 2], lam[4][2, 0] = -1j, 1j
    lam[5][1, 2] = lam[5][2, 1] = 1
    lam[6][1, 2], lam[6][2, 1] = -1j, 1j
    lam[7][0, 0] = lam[7][1, 1] = 1 / np.sqrt(3)
    lam[7][2, 2] = -2 / np.sqrt(3)
    return lam


def smoothed_su3(seed: int, n: int, eps: float) -> np.ndarray:
    """``n`` matrices exp(i eps H), H = sum_a w_a lambda_a / 2, w_a ~ N(0,1)."""
    lam = gell_mann()
    out = np.empty((n, 3, 3), dtype=np.complex128)
    for s in range(0, n, _CHUNK):
        m = min(_CHUNK, n - s)
        w = normal(seed, STREAM_ALGEBRA, 8 * s, 8 * m).reshape(m, 8)
        h = np.einsum("ma,aij->mij", w, lam) * 0.5
        h = 0.5 * (h + np.conj(np.swapaxes(h, 1, 2)))
        ev, vec = np.linalg.eigh(h)
        ph = np.exp(1j * eps * ev)
        out[s:s + m] = np.einsum("mij,mj,mkj->mik", vec, ph, np.conj(vec))
    return out


def unit_links(dims) -> np.ndarray:
    v = volume(dims)
    u = np.zeros((4, v, 3, 3), dtype=np.complex128)
    u[:, :, 0, 0] = u[:, :, 1, 1] = u[:, :, 2, 2] = 1.0
    return u


def haar_links(dims, seed: int) -> np.ndarray:
    """Gauge field of Haar-random SU(3) links, shape (4, V, 3, 3)."""
    v = volume(dims)
    return haar_su3(seed, 4 * v).reshape(4, v, 3, 3)


def smoothed_links(dims, seed: int, eps: float = 0.4) -> np.ndarray:
    """Gauge field of smoothed links exp(i eps H), shape (4, V, 3, 3)."""
    v = volume(dims)
    return smoothed_su3(seed, 4 * v, eps).reshape(4, v, 3, 3)


def gaussian_source(dims, seed: int, nrhs: int = 0) -> np.ndarray:
    """Complex-normal spinor field(s): (V, 4, 3), or (nrhs, V, 4, 3) when nrhs > 0."""
    v = volume(dims)
    k = max(nrhs, 1)
    b = _complex_normal(seed, STREAM_SOURCE, 0, k * v * 12).reshape(k, v, 4, 3)
    return b if nrhs > 0 else b[0]


def point_source(dims, site: int, spin: int, colour: int) -> np.ndarray:
    v = volume(dims)
    b = np.zeros((v, 4, 3), dtype=np.complex128)
    b[site, spin, colour] = 1.0
    return b


def propagator_sources(dims, site: int = 0) -> np.ndarray:
    """The 12 spin-colour point sources at one site, shape (12, V, 4, 3)."""
    v = volume(dims)
    b = np.zeros((12, v, 4, 3), dtype=np.complex128)
    for s in range(4):
        for c in range(3):
            b[3 * s + c, site, s, c] = 1.0
    return b


def gauge_transform(dims, seed: int) -> np.ndarray:
    """One Haar SU(3) matrix per site, shape (V, 3, 3) (for covariance tests)."""
    v = volume(dims)
    return haar_su3(seed + 0x5EED, v)


# Batched uneven workload: 64 lattices drawn from five shapes, kappa ~ U[0.10, 0.125].
BATCH_SHAPES = ((8, 8, 8, 8), (8, 8, 8, 16), (12, 12, 12, 12), (12, 12, 12, 24), (16, 16, 16, 16))


def batch_workload(n: int = 64, seed: int = 99):
    """Shapes and kappas of the batched uneven workload (per-lattice seeds 100 + i)."""
    u = uniform(seed, STREAM_MISC, 0, 2 * n)
    shapes = [BATCH_SHAPES[min(int(u[2 * i] * len(BATCH_SHAPES)), len(BATCH_SHAPES) - 1)] for i in range(n)]
    kappas = [0.10 + 0.025 * float(u[2 * i + 1]) for i in range(n)]
    seeds = [100 + i for i in range(n)]
    return shapes, kappas, seeds
