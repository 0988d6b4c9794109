"""GPU parity of the Dslash kernels against the CPU oracle (through the C ABI).

Tolerances (relative per-field 2-norm):
  * FP64: 1e-13 (the operator is exact up to rounding; FMA contraction and the
    half-spinor form change the rounding order only, ~1e-16 per site);
  * FP32: 2e-6 (single-precision storage of inputs and links, about 40 rounding
    steps per output component at 6e-8 each);
  * FP16 storage: 4e-3 (half-precision storage, 2^-11 relative to the per-site
    scale, FP32 arithmetic);
  * DF32 (pairs of floats, 48-bit significand): the FP64 tolerance, 1e-13 (inputs
    rounded to 2^-49 relative, about 40 operations per output at ~2^-47 each).
"""
import numpy as np
import pytest

import oracle
from paper_1810_04201_gb300 import gen

pytestmark = pytest.mark.gpu

TOL = {0: 1e-13, 1: 2e-6, 2: 4e-3, 3: 1e-13}
KAPPA = 0.12


@pytest.fixture(scope="module")
def wd():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1810_04201_gb300 import wd as _wd
    return _wd


SHAPES = [(4, 4, 4, 4), (2, 2, 2, 2), (6, 6, 6, 8), (3, 5, 4, 6), (8, 8, 8, 12), (4, 6, 8, 10)]


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("recon", [18, 12, 8])
def test_dslash_parity(wd, dims, prec, recon):
    U = gen.haar_links(dims, seed=2)
    psi = gen.gaussian_source(dims, seed=3)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=recon)
    f = lat.pack(psi, prec)
    for dagger in (False, True):
        o = lat.new_field(prec)
        lat.apply(KAPPA, f, o, prec, dagger=dagger)
        got = lat.unpack(o, prec)
        ref = oracle.apply_D(U, psi, KAPPA, dims, dagger=dagger)
        assert oracle.rel_err(got, ref) < TOL[prec], (dagger, oracle.rel_err(got, ref))


@pytest.mark.parametrize("prec", [0, 1, 3])
def test_periodic_time_and_paper_sign(wd, prec):
    dims = (4, 4, 2, 6)
    U = gen.haar_links(dims, seed=8)
    psi = gen.gaussian_source(dims, seed=9)
    lat = wd.Lattice(dims, antiperiodic_t=False)
    lat.set_gauge(U)
    f = lat.pack(psi, prec)
    o = lat.new_field(prec)
    lat.apply(-KAPPA, f, o, prec)  # the paper's +kappa convention
    ref = oracle.apply_D(U, psi, -KAPPA, dims, antiperiodic_t=False)
    assert oracle.rel_err(lat.unpack(o, prec), ref) < TOL[prec]


@pytest.mark.parametrize("nrhs,tiles", [(3, (64, 1)), (5, (32, 4)), (12, (16, 12)), (12, (32, 8)), (7, (128, 2))])
def test_multi_rhs_parity(wd, nrhs, tiles):
    dims = (4, 4, 6, 4)
    U = gen.haar_links(dims, seed=4)
    psi = gen.gaussian_source(dims, seed=5, nrhs=nrhs)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    for prec in (0, 1):
        if prec == 0 and tiles[0] < 32:
            # FP64 runs two lanes per site: a block needs whole warps along the sites
            with pytest.raises(wd.WDError):
                lat.set_tiles(prec, nrhs, *tiles)
            continue
        lat.set_tiles(prec, nrhs, *tiles)
        f = lat.pack(psi, prec)
        o = lat.new_field(prec, nrhs)
        lat.apply(KAPPA, f, o, prec, nrhs=nrhs)
        got = lat.unpack(o, prec, nrhs)
        for r in range(nrhs):
            assert oracle.rel_err(got[r], oracle.apply_D(U, psi[r], KAPPA, dims)) < TOL[prec]


def test_normal_op_parity(wd):
    dims = (4, 4, 4, 8)
    U = gen.haar_links(dims, seed=6)
    psi = gen.gaussian_source(dims, seed=7)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    f = lat.pack(psi)
    o = lat.new_field()
    lat.normal_apply(KAPPA, f, o)
    assert oracle.rel_err(lat.unpack(o), oracle.apply_normal(U, psi, KAPPA, dims)) < 1e-13


def test_df32_pack_roundtrip_and_range(wd):
    """DF32 keeps 48 significand bits: a pack/unpack round trip is exact to 2^-48 relative."""
    dims = (4, 4, 4, 4)
    psi = gen.gaussian_source(dims, seed=2) * np.exp(np.linspace(-20, 20, 256 * 12)).reshape(256, 4, 3)
    lat = wd.Lattice(dims)
    back = lat.unpack(lat.pack(psi, 3), 3)
    assert np.max(np.abs(back - psi) / np.abs(psi)) < 2.0 ** -47


def test_pack_unpack_roundtrip_bit_exact(wd):
    dims = (3, 5, 4, 6)
    psi = gen.gaussian_source(dims, seed=1, nrhs=2)
    lat = wd.Lattice(dims)
    f = lat.pack(psi, 0)
    np.testing.assert_array_equal(lat.unpack(f, 0, 2), psi)


@pytest.mark.parametrize("dims", [(16, 16, 16, 16), (32, 32, 32, 64)])
def test_full_size_sampled(wd, dims):
    """Full-size lattices: GPU output compared with the oracle at sampled sites, every
    precision and link compression."""
    U = gen.haar_links(dims, seed=10) if dims[3] == 16 else gen.smoothed_links(dims, seed=6, eps=0.4)
    psi = gen.gaussian_source(dims, seed=11)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    V = int(np.prod(dims))
    sites = np.unique(np.concatenate([np.arange(64), V - 1 - np.arange(64),
                                      gen.uniform(3, 9, 0, 256).__mul__(V).astype(np.int64)]))
    for recon in (18, 12, 8):
        lat.set_gauge(U, recon=recon)
        for prec in (0, 1, 2, 3):
            f = lat.pack(psi, prec)
            o = lat.new_field(prec)
            for dagger in (False, True):
                lat.apply(KAPPA, f, o, prec, dagger=dagger)
                got = lat.unpack(o, prec)[sites]
                ref = oracle.apply_D_sites(U, psi, KAPPA, dims, sites, dagger=dagger)
                assert oracle.rel_err(got, ref) < TOL[prec], (recon, prec, dagger)


def test_argument_errors(wd):
    lat = wd.Lattice((4, 4, 4, 4))
    f = lat.new_field()
    with pytest.raises(wd.WDError) as e:
        lat.apply(KAPPA, f, lat.new_field())
    assert e.value.status == 8  # no gauge yet
    lat.set_gauge(gen.unit_links((4, 4, 4, 4)))
    with pytest.raises(wd.WDError) as e:
        lat.apply(KAPPA, f, f)
    assert e.value.status == 1
    with pytest.raises(wd.WDError):
        lat.apply(KAPPA, f, lat.new_field(), nrhs=17)
    with pytest.raises(wd.WDError):
        lat.set_tiles(0, 4, 48, 1)
    with pytest.raises(wd.WDError) as e:
        lat.set_gauge(gen.unit_links((4, 4, 4, 4)), recon=7)
    assert e.value.status == 1
    with pytest.raises(wd.WDError):
        wd.Lattice((4, 1, 4, 4))


def test_recon8_rejects_singular_links(wd):
    """The 8-real form divides by |U01|^2 + |U02|^2: unit links are refused, and the
    context then holds no gauge field until a valid one is set."""
    dims = (4, 4, 4, 4)
    lat = wd.Lattice(dims)
    with pytest.raises(wd.WDError) as e:
        lat.set_gauge(gen.unit_links(dims), recon=8)
    assert e.value.status == 1
    f = lat.pack(gen.gaussian_source(dims, 1))
    with pytest.raises(wd.WDError) as e:
        lat.apply(KAPPA, f, lat.new_field())
    assert e.value.status == 8
    U = gen.haar_links(dims, seed=6)
    U[1, 5] = np.eye(3)  # one unit link among Haar links
    with pytest.raises(wd.WDError):
        lat.set_gauge(U, recon=8)
    U = gen.haar_links(dims, seed=6)
    lat.set_gauge(U, recon=8)
    psi = gen.gaussian_source(dims, 2)
    o = lat.new_field()
    lat.apply(KAPPA, lat.pack(psi), o)
    assert oracle.rel_err(lat.unpack(o), oracle.apply_D(U, psi, KAPPA, dims)) < TOL[0]


@pytest.mark.parametrize("prec", [0, 1, 2, 3])
def test_recon8_smoothed_links(wd, prec):
    """Near-unit links (exp(i eps H), the mixed-precision workload) through recon 8."""
    dims = (6, 4, 4, 8)
    U = gen.smoothed_links(dims, eps=0.4, seed=12)
    psi = gen.gaussian_source(dims, seed=13)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=8)
    f = lat.pack(psi, prec)
    for dagger in (False, True):
        o = lat.new_field(prec)
        lat.apply(KAPPA, f, o, prec, dagger=dagger)
        ref = oracle.apply_D(U, psi, KAPPA, dims, dagger=dagger)
        assert oracle.rel_err(lat.unpack(o, prec), ref) < TOL[prec]


@pytest.mark.parametrize("recon", [18, 8])
def test_outputs_fully_written_over_nan_poison(wd, recon):
    """Output buffers filled with NaN bytes before each call: every site of every
    right-hand side is overwritten (no unwritten tail or tile)."""
    dims, nrhs = (6, 4, 4, 6), 3
    U = gen.haar_links(dims, seed=21)
    psi = gen.gaussian_source(dims, seed=22, nrhs=nrhs)
    lat = wd.Lattice(dims)
    lat.set_gauge(U, recon=recon)
    for prec in (0, 1, 2, 3):
        f = lat.pack(psi, prec)
        for call in (lat.apply, lat.normal_apply):
            o = lat.new_field(prec, nrhs)
            o.fill_(0xFF)
            call(KAPPA, f, o, prec, nrhs=nrhs)
            got = lat.unpack(o, prec, nrhs)
            assert np.isfinite(got).all(), (prec, call.__name__)
            for r in range(nrhs):
                ref = oracle.apply_D(U, psi[r], KAPPA, dims)
                if call == lat.normal_apply:
                    ref = oracle.apply_Ddag(U, ref, KAPPA, dims)
                assert oracle.rel_err(got[r], ref) < 4 * TOL[prec], (prec, call.__name__, r)


@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("dims,rows", [((8, 4, 4, 6), 1), ((8, 4, 4, 6), 2), ((8, 4, 4, 6), 4), ((16, 6, 2, 4), 3),
                                       ((32, 8, 4, 4), 4), ((4, 2, 2, 2), 2)])
def test_staged_dslash_matches_oracle(wd, prec, dims, rows):
    """The kernel that stages neighbour spinors through shared memory (bulk copies on an
    mbarrier, persistent blocks, several tiles in flight): D and D^dag in FP32 and FP16 against
    the oracle, two right-hand sides, recon-18 and recon-12, and against the direct kernel."""
    U = gen.haar_links(dims, seed=91)
    psi = gen.gaussian_source(dims, seed=92, nrhs=2)
    for recon in (18, 12):
        lat = wd.Lattice(dims)
        lat.set_gauge(U, recon=recon)
        f = lat.pack(psi, prec)
        direct = {}
        for staged in (0, rows):
            lat.set_staging(prec, staged, 3 if staged else 2)
            for dag in (False, True):
                o = lat.new_field(prec, nrhs=2)
                lat.apply(0.12, f, o, prec, nrhs=2, dagger=dag)
                got = lat.unpack(o, prec, nrhs=2)
                if not staged:
                    direct[dag] = got
                    continue
                for k in range(2):
                    want = oracle.apply_D(U, psi[k], 0.12, dims, dagger=dag)
                    assert oracle.rel_err(got[k], want) < TOL[prec], (recon, dag, k)
                # the same per-site arithmetic as the direct kernel, apart from the order of
                # FP32 sums the compiler chose
                assert oracle.rel_err(got, direct[dag]) < TOL[prec]
        assert lat.staging_error() == 0


def test_staged_dslash_rejects_unsuited_shapes(wd):
    lat = wd.Lattice((6, 4, 4, 4))
    lat.set_gauge(gen.haar_links((6, 4, 4, 4), seed=93))
    for prec, rows, stages in ((2, 1, 2), (1, 3, 2), (0, 1, 2), (1, 1, 5), (1, 1, 1)):
        with pytest.raises(wd.WDError) as e:  # FP16 with Lx % 4, rows not dividing Ly, FP64, stage counts
            lat.set_staging(prec, rows, stages)
        assert e.value.status == 1
    big = wd.Lattice((64, 8, 2, 2))
    with pytest.raises(wd.WDError):  # more than 256 sites per tile
        big.set_staging(1, 8, 2)
    lat.set_staging(1, 2, 2)
    lat.set_staging(1, 0)


@pytest.mark.parametrize("nrhs,site_tile,rhs_tile,k", [(3, 32, 3, 3), (8, 32, 8, 2), (8, 64, 4, 4), (12, 16, 8, 4),
                                                       (12, 32, 6, 3), (5, 64, 4, 2)])
def test_rhs_per_thread_matches_oracle(wd, nrhs, site_tile, rhs_tile, k):
    """FP32 with k right-hand sides per thread (each link loaded once for k): D and D^dag
    against the oracle, also with a partial last group of right-hand sides, and the same
    result as one right-hand side per thread."""
    dims = (6, 4, 4, 6)
    U = gen.haar_links(dims, seed=95)
    psi = gen.gaussian_source(dims, seed=96, nrhs=nrhs)
    for recon in (18, 12, 8):
        lat = wd.Lattice(dims)
        lat.set_gauge(U, recon=recon)
        f = lat.pack(psi, 1)
        lat.set_tiles(1, nrhs, site_tile, rhs_tile)
        outs = {}
        for kk in (1, k):
            lat.set_rhs_per_thread(1, nrhs, kk)
            assert lat.tiles(1, nrhs) == (site_tile, rhs_tile, kk)
            for dag in (False, True):
                o = lat.new_field(1, nrhs=nrhs)
                lat.apply(0.12, f, o, 1, nrhs=nrhs, dagger=dag)
                outs[kk, dag] = lat.unpack(o, 1, nrhs=nrhs)
        for dag in (False, True):
            for j in range(nrhs):
                want = oracle.apply_D(U, psi[j], 0.12, dims, dagger=dag)
                assert oracle.rel_err(outs[k, dag][j], want) < TOL[1], (recon, dag, j)
            assert oracle.rel_err(outs[k, dag], outs[1, dag]) < 1e-7
    with pytest.raises(wd.WDError):
        lat.set_rhs_per_thread(0, nrhs, 2)  # FP64: one right-hand side per thread


def test_staged_wait_timeout_is_reported(wd, monkeypatch):
    """A wait of the staged kernel that runs out (block 0 waits on an mbarrier that nothing
    completes) sets the context's staging error word instead of hanging; the block drains its
    copies in flight and leaves, and the context stays usable."""
    dims = (8, 4, 4, 6)
    U = gen.haar_links(dims, seed=97)
    psi = gen.gaussian_source(dims, seed=98)
    lat = wd.Lattice(dims)
    lat.set_gauge(U)
    f = lat.pack(psi, 1)
    lat.set_staging(1, 2, 2)
    monkeypatch.setenv("WD_STAGED_STALL_TEST", "1")
    lat.apply(0.12, f, lat.new_field(1), 1)
    assert lat.staging_error() == 1
    monkeypatch.delenv("WD_STAGED_STALL_TEST")
    o = lat.new_field(1)
    lat.apply(0.12, f, o, 1)
    assert lat.staging_error() == 0
    assert oracle.rel_err(lat.unpack(o, 1), oracle.apply_D(U, psi, 0.12, dims)) < TOL[1]


@pytest.mark.parametrize("dims,nrhs", [((8, 4, 6, 6), 1), ((6, 4, 4, 6), 3), ((5, 3, 4, 6), 2)])
def test_prefetch_dslash_matches_oracle(wd, dims, nrhs):
    """The FP32 kernel with per-thread cp.async prefetch of the neighbour spinors: D and D^dag,
    recon 18/12/8, against the oracle and the direct kernel."""
    U = gen.haar_links(dims, seed=99)
    psi = gen.gaussian_source(dims, seed=100, nrhs=nrhs)
    for recon in (18, 12, 8):
        lat = wd.Lattice(dims)
        lat.set_gauge(U, recon=recon)
        f = lat.pack(psi if nrhs > 1 else psi[0], 1)
        for dag in (False, True):
            outs = []
            for on in (False, True):
                lat.set_prefetch(1, on)
                o = lat.new_field(1, nrhs=nrhs)
                lat.apply(0.12, f, o, 1, nrhs=nrhs, dagger=dag)
                outs.append(lat.unpack(o, 1, nrhs=nrhs, squeeze=False))
            for j in range(nrhs):
                want = oracle.apply_D(U, psi[j], 0.12, dims, dagger=dag)
                assert oracle.rel_err(outs[1][j], want) < TOL[1], (recon, dag, j)
            assert oracle.rel_err(outs[1], outs[0]) < 1e-7
    with pytest.raises(wd.WDError):
        lat.set_prefetch(0, True)
