"""The index-checking debug build (-DWD_DEBUG, in place of a memory checker, which is
closed on this pool): every Dslash neighbour and checkerboard index is checked against its
field on small, odd-shaped and 2-extent lattices, through the operators and the solvers,
and no kernel may leave an out-of-range record.  Runs in a child process that loads the
debug library."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = textwrap.dedent("""
    import sys
    import numpy as np
    import oracle
    from paper_1810_04201_gb300 import build, gen, wd
    wd.load_library(build.build(debug=True))
    kappa = 0.12
    tol = {0: 1e-13, 1: 2e-6, 2: 4e-3, 3: 1e-13}
    for dims in [(2, 2, 2, 2), (3, 5, 4, 6), (4, 4, 2, 8), (6, 4, 4, 4)]:
        U = gen.haar_links(dims, seed=5)
        psi = gen.gaussian_source(dims, seed=6, nrhs=3)
        lat = wd.Lattice(dims)
        word, dbg = lat.debug_word()
        assert dbg and word == 0
        for recon in (18, 12, 8):
            lat.set_gauge(U, recon=recon)
            for prec in (0, 1, 2, 3):
                f = lat.pack(psi, prec)
                for dag in (False, True):
                    o = lat.new_field(prec, 3)
                    lat.apply(kappa, f, o, prec, nrhs=3, dagger=dag)
                    got = lat.unpack(o, prec, 3)
                    for r in range(3):
                        ref = oracle.apply_D(U, psi[r], kappa, dims, dagger=dag)
                        assert oracle.rel_err(got[r], ref) < tol[prec], (dims, recon, prec, dag)
            assert lat.debug_word()[0] == 0, (dims, recon, hex(lat.debug_word()[0]))
        lat.set_gauge(U)
        for inner in (0, 1, 3):
            res, st = lat.cg(kappa, lat.pack(psi[0]), lat.new_field(), tol=1e-10, inner=inner)
            assert st == 0
            if all(d % 2 == 0 for d in dims):
                res, st = lat.cg(kappa, lat.pack(psi), lat.new_field(nrhs=3), tol=1e-10, inner=inner, nrhs=3,
                                 precondition=1)
                assert st == 0
                o = lat.new_field()
                lat.apply_schur(kappa, lat.pack(psi[0]), o)
        res, st = wd.cg_batched([lat], [kappa], [lat.pack(psi[0])], [lat.new_field()], tol=1e-10)
        assert st == 0
        assert lat.debug_word()[0] == 0, (dims, hex(lat.debug_word()[0]))
    print("DEBUG-BUILD-OK")
""")


def test_debug_build_has_no_out_of_range_index():
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, capture_output=True, text=True, timeout=1500)
    assert r.returncode == 0 and "DEBUG-BUILD-OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
