"""Checks of the seeded input generators (not of the method)."""
import numpy as np

from paper_1810_04201_gb300 import gen


def test_splitmix64_reference_value():
    # The published SplitMix64 sequence started from state 0 begins with 0xE220A8397B1DCDAF.
    z = gen._mix64(np.array([0x9E3779B97F4A7C15], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF


def test_streams_are_reproducible_and_sliceable():
    a = gen.normal(5, 1, 0, 1000)
    b = gen.normal(5, 1, 0, 1000)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(gen.normal(5, 1, 301, 50), a[301:351])
    np.testing.assert_array_equal(gen.uniform(5, 2, 17, 10), gen.uniform(5, 2, 0, 40)[17:27])
    assert not np.allclose(gen.normal(5, 2, 0, 10), a[:10])


def test_normal_moments():
    g = gen.normal(1, 1, 0, 200000)
    assert abs(g.mean()) < 0.01 and abs(g.var() - 1) < 0.01


def test_haar_su3_is_special_unitary_and_haar():
    U = gen.haar_su3(3, 20000)
    I = np.eye(3)
    err = np.abs(U @ np.conj(np.swapaxes(U, 1, 2)) - I).max()
    assert err < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    tr = np.trace(U, axis1=1, axis2=2)
    # Haar moments on SU(3): E[tr U] = 0, E[|tr U|^2] = 1
    assert abs(tr.mean()) < 0.03
    assert abs(np.mean(np.abs(tr) ** 2) - 1) < 0.05


def test_gell_mann_and_smoothed_links():
    lam = gen.gell_mann()
    for a in range(8):
        assert abs(np.trace(lam[a])) < 1e-15
        np.testing.assert_allclose(lam[a], lam[a].conj().T)
        for b in range(8):
            assert abs(np.trace(lam[a] @ lam[b]) - 2 * (a == b)) < 1e-14
    U = gen.smoothed_su3(4, 5000, 0.4)
    assert np.abs(U @ np.conj(np.swapaxes(U, 1, 2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-13
    U0 = gen.smoothed_su3(4, 100, 1e-9)
    assert np.abs(U0 - np.eye(3)).max() < 1e-8
    # smoothed links stay near the identity: Re tr U / 3 well above the Haar value 0
    assert np.real(np.trace(U, axis1=1, axis2=2)).mean() / 3 > 0.8


def test_sources():
    b = gen.gaussian_source((2, 2, 2, 4), 1)
    assert b.shape == (32, 4, 3)
    assert abs(np.mean(np.abs(gen.gaussian_source((8, 8, 8, 8), 2)) ** 2) - 1) < 0.02
    P = gen.propagator_sources((2, 2, 2, 2), site=3)
    assert P.shape == (12, 16, 4, 3)
    assert np.count_nonzero(P) == 12 and P[7, 3, 2, 1] == 1


def test_batch_workload():
    shapes, kappas, seeds = gen.batch_workload()
    assert len(shapes) == 64 and set(shapes) <= set(gen.BATCH_SHAPES)
    assert min(kappas) >= 0.10 and max(kappas) <= 0.125
    assert seeds[0] == 100 and seeds[-1] == 163
