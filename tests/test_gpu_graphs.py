"""Step graphs and batches of chains (cl_capture_step / cl_replay,
cl_batch_*): a replayed or batched step launches the same kernels in the same
order as the eager calls, and every reduction has a fixed order, so the links
must agree with the eager path bit for bit; the eager path itself is checked
against the oracle once more here."""
import numpy as np
import pytest

import oracle as O
from paper_1311_1056_gb300 import build, cl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    cl.load()


def _lat(L=(4, 4, 4, 6), beta=6.0, theta=1.0, prec=cl.CL_FP64, seed=3, sigma=0.05):
    return cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=seed, start=cl.CL_START_HOT,
                      gauge_sigma=sigma, own_stream=True)


ADAPT = dict(eps=0.01, alpha=1.0, mode=cl.CL_D2_MEANABS, n_min=1, n_max=6, tol_rel=0.05)


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE, cl.CL_DF64])
@pytest.mark.parametrize("cool", [None, ADAPT])
def test_replay_equals_eager(prec, cool):
    cp = cl.make_cool(**cool) if cool else None
    with _lat(prec=prec) as a, _lat(prec=prec) as b:
        b.capture_step(0.01, cp)
        assert b.step_count == 0  # capturing runs nothing
        for k in range(5):
            a.step(0.01, 1)
            if cp is not None:
                ra = a.cool(cp)
            b.replay(1)
            if cp is not None:
                rb = b.last_cool_report()
                assert ra == rb, k
        assert a.step_count == b.step_count == 5
        assert a.launches() == b.launches()
        assert np.array_equal(a.links(), b.links())
        assert a.observables() == b.observables()


def test_replay_against_oracle():
    L, beta, theta, eps, seed = (4, 4, 4, 6), 6.0, 1.0, 0.01, 3
    cpar = dict(eps=eps, alpha=1.0, mode=cl.CL_D1, forced_sweeps=2)
    U = O.random_gauge(L, O.hot_start(L, seed), seed, 0.05)
    with _lat() as lat:
        lat.capture_step(eps, cl.make_cool(**cpar))
        lat.replay(3)
        got = lat.links()
    for step in range(3):
        U = O.cl_step(L, U, beta, theta, eps, seed, step)
        U, _ = O.cool(L, U, O.cool_params(**cpar))
    assert np.abs(got - U).max() < 1e-12


def test_replay_mixed_with_eager_calls_and_set_step():
    cp = cl.make_cool(**ADAPT)
    with _lat() as a, _lat() as b:
        for lat in (a, b):
            cl.cl_set_step(lat.h, 7)
        b.capture_step(0.01, cp)
        for k in range(4):
            a.step(0.01, 1)
            a.cool(cp)
        b.replay(2)
        b.step(0.01, 1)
        b.cool(cp)
        b.replay(1)
        assert a.step_count == b.step_count == 11
        assert np.array_equal(a.links(), b.links())


def _chains():
    """Four unlike chains: sizes, couplings, theta, precision and rule differ."""
    return [
        dict(L=(4, 4, 4, 4), beta=5.6, theta=0.0, prec=cl.CL_FP64, seed=11),
        dict(L=(6, 4, 4, 4), beta=6.0, theta=0.5, prec=cl.CL_FP32_STORAGE, seed=12),
        dict(L=(4, 6, 4, 8), beta=6.2, theta=1.5, prec=cl.CL_FP64, seed=13),
        dict(L=(8, 8, 8, 8), beta=5.9, theta=2.0, prec=cl.CL_FP32_STORAGE, seed=14),
    ]


def test_batch_equals_each_chain_alone():
    chains = _chains()
    eps = [0.01, 0.005, 0.01, 0.008]
    cps = [cl.make_cool(**ADAPT), cl.make_cool(eps=0.005, alpha=1.0, mode=cl.CL_D1, forced_sweeps=2),
           cl.make_cool(eps=0.01, alpha=0.5, mode=cl.CL_D0, n_min=0, n_max=4, tol_rel=0.1),
           cl.make_cool(eps=0.008, alpha=1.0, mode=cl.CL_D2_RMS, n_min=1, n_max=5, tol_rel=0.05)]
    alone = []
    for c, e, cp in zip(chains, eps, cps):
        with _lat(**c) as lat:
            reps = []
            for _ in range(6):
                lat.step(e, 1)
                reps.append(lat.cool(cp))
            alone.append((lat.links(), reps[-1], lat.observables(), lat.launches()))
    lats = [_lat(**c) for c in chains]
    try:
        with cl.Batch(lats, eps, cps) as b:
            b.run(4)
            b.run(2)
            b.synchronize()
            for lat, (U, rep, obs, nl) in zip(lats, alone):
                assert lat.step_count == 6
                assert np.array_equal(lat.links(), U)
                assert lat.last_cool_report() == rep
                assert lat.observables() == obs
                assert lat.launches() == nl
    finally:
        for lat in lats:
            lat.close()


def test_batch_without_cooling_and_then_eager():
    chains = _chains()[:2]
    lats = [_lat(**c) for c in chains]
    refs = [_lat(**c) for c in chains]
    try:
        with cl.Batch(lats, 0.01) as b:
            b.run(3)
        for lat, ref in zip(lats, refs):
            ref.step(0.01, 4)
            lat.step(0.01, 1)  # eager calls after the batch is gone
            assert np.array_equal(lat.links(), ref.links())
    finally:
        for lat in lats + refs:
            lat.close()


def test_batch_refuses_a_chain_stepped_alone():
    lats = [_lat(**c) for c in _chains()[:2]]
    try:
        with cl.Batch(lats, 0.01) as b:
            b.run(1)
            lats[0].step(0.01, 1)
            with pytest.raises(cl.CLError) as ei:
                b.run(1)
            assert ei.value.status == cl.CL_ERR_INVALID
    finally:
        for lat in lats:
            lat.close()


def test_graph_argument_errors():
    with cl.Lattice((4, 4, 4, 4)) as lat:  # legacy default stream
        with pytest.raises(cl.CLError) as ei:
            lat.capture_step(0.01)
        assert ei.value.status == cl.CL_ERR_INVALID
        with pytest.raises(cl.CLError):
            lat.replay(1)  # nothing captured
    with _lat() as lat:
        with pytest.raises(cl.CLError):
            cl.cl_batch_create([lat.h, lat.h], 0.01)  # the same lattice twice
        with pytest.raises(cl.CLError):
            lat.capture_step(-1.0)


def test_batch_membership_changes():
    """Chains join and leave a batch between runs; each ends where it would
    alone after the same number of steps."""
    chains = _chains()[:3]
    cp = cl.make_cool(**ADAPT)
    lats = [_lat(**c) for c in chains]
    refs = [_lat(**c) for c in chains]
    try:
        with cl.Batch(lats[:2], 0.01, [cp, cp]) as b:
            b.run(2)
            b.add(lats[2], 0.01, cp)
            assert len(b) == 3
            b.run(3)
            b.remove(lats[0])
            b.run(2)
            with pytest.raises(cl.CLError):
                b.remove(lats[0])  # no longer a member
            with pytest.raises(cl.CLError):
                b.add(lats[1], 0.01, cp)  # already a member
        lats[0].step(0.01, 1)  # stepped on its own after leaving
        lats[0].cool(cp)
        for ref, n in zip(refs, (6, 7, 5)):
            for _ in range(n):
                ref.step(0.01, 1)
                ref.cool(cp)
        for lat, ref in zip(lats, refs):
            assert lat.step_count == ref.step_count
            assert np.array_equal(lat.links(), ref.links())
    finally:
        for lat in lats + refs:
            lat.close()


def _fused_chains(prec):
    """Unlike chains of one precision: sizes (ragged, not multiples of the
    block), couplings, theta = 0 and != 0, fixed and adaptive step size."""
    return [
        dict(L=(4, 4, 4, 4), beta=5.6, theta=0.0, prec=prec, seed=21, k_ref=0.0),
        dict(L=(6, 4, 4, 4), beta=6.0, theta=0.5, prec=prec, seed=22, k_ref=6.0),
        dict(L=(4, 6, 4, 8), beta=6.2, theta=1.5, prec=prec, seed=23, k_ref=0.0),
        dict(L=(3, 5, 4, 7), beta=5.9, theta=2.0, prec=prec, seed=24, k_ref=4.0),
        dict(L=(8, 8, 8, 8), beta=6.0, theta=1.0, prec=prec, seed=25, k_ref=0.0),
        dict(L=(2, 1, 3, 1), beta=6.0, theta=0.7, prec=prec, seed=26, k_ref=0.0),  # extents of 1
    ]


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32_STORAGE])
def test_fused_batch_equals_each_chain_alone(prec):
    """Fused mode: one launch per kernel family runs the blocks of every
    chain, each with its own geometry, buffers, noise and cooling rule -- the
    single-pass D_0 / D_1 sweeps and the four-kernel D_2 sweeps side by side,
    different sweep limits, theta = 0 and != 0, adaptive and fixed step size.
    Every chain must end where it ends alone, bit for bit."""
    chains = _fused_chains(prec)
    eps = [0.01, 0.005, 0.01, 0.008, 0.006, 0.01]
    cps = [cl.make_cool(**ADAPT), cl.make_cool(eps=0.005, alpha=1.0, mode=cl.CL_D1, forced_sweeps=2),
           cl.make_cool(eps=0.01, alpha=0.5, mode=cl.CL_D0, n_min=0, n_max=4, tol_rel=0.1),
           cl.make_cool(eps=0.008, alpha=1.0, mode=cl.CL_D2_RMS, n_min=1, n_max=5, tol_rel=0.05),
           cl.make_cool(eps=0.006, alpha=1.0, mode=cl.CL_D1, n_min=0, n_max=3, tol_rel=1e-3),
           cl.make_cool(eps=0.01, alpha=1.0, mode=cl.CL_D2_MEANABS, forced_sweeps=3)]

    def make(c):
        lat = _lat(L=c["L"], beta=c["beta"], theta=c["theta"], prec=c["prec"], seed=c["seed"])
        if c["k_ref"] > 0:
            lat.set_adaptive_step(c["k_ref"])
        return lat

    alone = []
    for c, e, cp in zip(chains, eps, cps):
        with make(c) as lat:
            reps = []
            for _ in range(5):
                lat.step(e, 1)
                reps.append(lat.cool(cp))
            alone.append((lat.links(), reps[-1], lat.observables(), lat.langevin_time()))
    lats = [make(c) for c in chains]
    try:
        with cl.Batch(lats, eps, cps, fused=True) as b:
            assert b.fused
            b.run(3)
            b.run(2)
            b.synchronize()
            for lat, (U, rep, obs, t) in zip(lats, alone):
                assert lat.step_count == 5
                assert np.array_equal(lat.links(), U)
                assert lat.last_cool_report() == rep
                assert lat.observables() == obs
                assert lat.langevin_time() == t
            # back to per-chain graphs, then fused again, mid-run
            b.set_fused(False)
            b.run(1)
            b.set_fused(True)
            b.run(1)
            assert all(lat.step_count == 7 for lat in lats)
    finally:
        for lat in lats:
            lat.close()


def test_fused_batch_refuses_mixed_precision():
    lats = [_lat(prec=cl.CL_FP64), _lat(prec=cl.CL_FP32_STORAGE, seed=4)]
    try:
        with cl.Batch(lats, 0.01) as b:
            with pytest.raises(cl.CLError) as ei:
                b.set_fused(True)
            assert ei.value.status == cl.CL_ERR_INVALID
            assert not b.fused
            b.run(1)  # still a working per-chain batch
    finally:
        for lat in lats:
            lat.close()


def test_batch_default_mode_follows_the_members():
    """A batch starts fused when its members allow it (one precision, FP64 or
    FP32 storage); adding a member of another precision switches it to
    per-chain graphs, and every chain still ends where it would alone."""
    cp = cl.make_cool(**ADAPT)
    lats = [_lat(prec=cl.CL_FP32_STORAGE, seed=41), _lat(prec=cl.CL_FP32_STORAGE, seed=42, L=(4, 4, 6, 4))]
    extra = _lat(prec=cl.CL_FP64, seed=43)
    refs = [_lat(prec=cl.CL_FP32_STORAGE, seed=41), _lat(prec=cl.CL_FP32_STORAGE, seed=42, L=(4, 4, 6, 4)),
            _lat(prec=cl.CL_FP64, seed=43)]
    try:
        with cl.Batch(lats, 0.01, [cp, cp]) as b:
            assert b.fused
            b.run(2)
            b.add(extra, 0.01, cp)
            assert not b.fused
            b.run(2)
        for ref, n in zip(refs, (4, 4, 2)):
            for _ in range(n):
                ref.step(0.01, 1)
                ref.cool(cp)
        for lat, ref in zip(lats + [extra], refs):
            assert np.array_equal(lat.links(), ref.links())
    finally:
        for lat in lats + [extra] + refs:
            lat.close()
