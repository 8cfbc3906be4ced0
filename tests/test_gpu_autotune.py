"""The launch-shape autotuner: it leaves the lattice as it found it, picks
block sizes from the candidate set, and any block size gives the same links
bit for bit (each thread owns one site or link; the reductions keep a fixed
shape)."""
import numpy as np
import pytest

from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


ADAPT = dict(eps=0.01, alpha=1.0, mode=cl.CL_D2_MEANABS, n_min=1, n_max=6, tol_rel=0.05)


def _lat(prec, theta=1.0, L=(6, 4, 4, 6)):
    return cl.Lattice(L, beta=6.0, theta=theta, prec=prec, seed=9, start=cl.CL_START_HOT,
                      gauge_sigma=0.05, own_stream=True)


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE, cl.CL_DF64])
def test_autotune_leaves_state_and_picks_candidates(prec):
    cp = cl.make_cool(**ADAPT)
    with _lat(prec) as a, _lat(prec) as b:
        a.step(0.01, 2)
        a.cool(cp)
        b.step(0.01, 2)
        b.cool(cp)
        U0, n0, r0 = a.links(), a.launches(), a.last_cool_report()
        blocks, table = a.autotune(0.01, cp, reps=2, use_cache=False, want_table=True)
        assert all(v in cl.TUNE_CANDIDATES for v in blocks)
        assert a.blocks() == blocks
        assert table.shape == (4, cl.CL_NTUNE) and np.all(table[:, [0, 1, 2]] > 0)
        for f in range(cl.CL_NTUNE):
            if np.all(table[:, f] > 0):
                assert table[cl.TUNE_CANDIDATES.index(blocks[f]), f] == table[:, f].min()
        assert a.launches() == n0 and a.step_count == 2
        assert np.array_equal(a.links(), U0)
        assert a.last_cool_report() == r0
        # the tuned lattice continues exactly like an untuned one
        for lat in (a, b):
            lat.step(0.01, 3)
            lat.cool(cp)
        assert np.array_equal(a.links(), b.links())


@pytest.mark.parametrize("prec,theta", [(cl.CL_FP64, 1.0), (cl.CL_FP32_STORAGE, 0.5),
                                        (cl.CL_FP64, 0.0), (cl.CL_DF64, 1.0), (cl.CL_DF64, 0.0)])
def test_every_block_size_gives_the_same_links(prec, theta):
    cp = cl.make_cool(**ADAPT)
    ref = None
    for bs in cl.TUNE_CANDIDATES:
        with _lat(prec, theta, L=(5, 4, 3, 7)) as lat:  # V = 420: ragged tail at every size
            lat.set_blocks([bs] * cl.CL_NTUNE)
            assert lat.blocks() == [bs] * cl.CL_NTUNE
            for _ in range(3):
                lat.step(0.01, 1)
                lat.cool(cp)
            U = lat.links()
        if ref is None:
            ref = U
        assert np.array_equal(U, ref), bs


def test_mixed_block_sizes_and_cache():
    cp = cl.make_cool(**ADAPT)
    with _lat(cl.CL_FP64) as a, _lat(cl.CL_FP64) as b:
        a.set_blocks([32, 256, 64, 128, 96])
        for lat in (a, b):
            lat.step(0.01, 2)
            lat.cool(cp)
        assert np.array_equal(a.links(), b.links())
        first, _ = a.autotune(0.01, cp, reps=1, use_cache=True)
        b.set_blocks([0] * cl.CL_NTUNE)
        again, _ = b.autotune(0.01, cp, reps=1, use_cache=True)  # same shape: from the cache
        assert again == first


def test_set_blocks_rejects_bad_sizes():
    with _lat(cl.CL_FP64) as lat:
        for bad in ([16] * 5, [512] * 5, [100] * 5, [-32] * 5):
            with pytest.raises(cl.CLError) as ei:
                lat.set_blocks(bad)
            assert ei.value.status == cl.CL_ERR_INVALID
        assert lat.blocks() == [128] * cl.CL_NTUNE
