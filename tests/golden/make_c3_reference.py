"""Write c3_oracle_reference.txt: the oracle's solution of the 32^3 x 64 mixed-precision
workload at sampled sites, with the condition-number estimate that bounds solution errors.

Workload: smoothed links exp(i 0.4 H) (seed 6), kappa = 0.124, Gaussian source (seed 6),
antiperiodic t.  The oracle solves D^dag D x = D^dag b by CG (section 2.2) to a normal
residual of 1e-13; the extreme eigenvalues of D^dag D come from the oracle's Lanczos
estimate.  Every value written here comes from oracle/ (no GPU involved).

Run from the repository root (about an hour on 8 cores):
    python tests/golden/make_c3_reference.py
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1810_04201_gb300 import gen  # noqa: E402

DIMS, KAPPA, SEED, EPS = (32, 32, 32, 64), 0.124, 6, 0.4
LANCZOS_STEPS = 600
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c3_oracle_reference.txt")


def sample_sites(v: int) -> np.ndarray:
    """First and last 16 sites and 32 seeded ones (the GPU test uses the same list)."""
    rnd = (gen.uniform(11, 3, 0, 32) * v).astype(np.int64)
    return np.unique(np.concatenate([np.arange(16), v - 16 + np.arange(16), rnd]))


def main() -> None:
    t0 = time.time()
    U = gen.smoothed_links(DIMS, SEED, eps=EPS)
    b = gen.gaussian_source(DIMS, SEED)
    x, info = oracle.cgnr(U, b, KAPPA, DIMS, tol=1e-13, max_iter=20000)
    assert info["converged"], info
    t1 = time.time()
    lo_half, hi_half, _ = oracle.normal_extreme_eigs(U, KAPPA, DIMS, LANCZOS_STEPS // 2, seed=SEED)
    lo, hi, k = oracle.normal_extreme_eigs(U, KAPPA, DIMS, LANCZOS_STEPS, seed=SEED)
    t2 = time.time()
    v = int(np.prod(DIMS))
    sites = sample_sites(v)
    with open(OUT, "w") as f:
        f.write("# Oracle reference of the 32^3 x 64 workload: smoothed links exp(i 0.4 H) seed 6, kappa 0.124,\n")
        f.write("# Gaussian source seed 6, antiperiodic t.  Written by tests/golden/make_c3_reference.py from\n")
        f.write("# oracle.cgnr (tol 1e-13) and oracle.normal_extreme_eigs (plain Lanczos on D^dag D).\n")
        f.write(f"cg_iters {info['iters']}\n")
        f.write(f"true_normal_rel {info['true_normal_rel']:.6e}\n")
        f.write(f"true_rel {info['true_rel']:.6e}\n")
        f.write(f"x_norm {np.linalg.norm(x):.17e}\n")
        f.write(f"lanczos_steps {k}\n")
        f.write(f"lambda_min {lo:.10e}\n")
        f.write(f"lambda_max {hi:.10e}\n")
        f.write(f"lambda_min_half_steps {lo_half:.10e}\n")
        f.write(f"lambda_max_half_steps {hi_half:.10e}\n")
        f.write(f"cond_D {np.sqrt(hi / lo):.6e}\n")
        f.write(f"# sites: index, then the 12 components (spin-major, colour-minor) as re im pairs\n")
        for s in sites:
            vals = " ".join(f"{z.real:.17e} {z.imag:.17e}" for z in x[s].reshape(-1))
            f.write(f"site {int(s)} {vals}\n")
    print(f"cg {t1 - t0:.0f} s, lanczos {t2 - t1:.0f} s, cond(D) {np.sqrt(hi / lo):.4e}, wrote {OUT}")


if __name__ == "__main__":
    main()
