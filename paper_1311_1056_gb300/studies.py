"""Studies of Sec. 3-5 run on the library's kernels.

* cooling_decay: the distance d = UN - 1 of a gauge-transformed unitary
  configuration under gauge cooling alone, one sweep at a time, for the
  choices D_0, D_1, D_2 of the adaptive strength alpha_ad = alpha / D
  (Sec. 4), on SU(2) Polyakov chains of N links (the model of Sec. 3-4) and on
  an SU(3) lattice.
* precision_table: the FP32-storage form against the FP64 form on identical
  noise (same start, seed and step counter): max |U32 - U64| over the links
  and the error of every observable after a number of steps.
* theta_scan: CL with adaptive cooling (alpha_ad = 0.1 / D_2) and the
  adaptive step size on small SU(3) lattices at several beta and
  theta_L^2 = 0, +-1, +-4 (Sec. 5), as one batch of chains; returns the
  series of the plaquette, Q_L and the unitarity norm.

* longrun: independent chains (one Philox seed each) of CL with adaptive
  cooling advanced together as one batch, the observables of every chain
  recorded every few steps; and chain_means / compare_means, the statistics
  that compare two such ensembles (long trajectories decorrelate
  chaotically, so two arithmetic forms can only agree in distribution).

Every number comes from the CUDA kernels through the C-ABI (cl.py).
"""
import numpy as np

from . import cl

MODES = {"D0": cl.CL_D0, "D1": cl.CL_D1, "D2": cl.CL_D2_MEANABS}


def chain_cooling(n_links, mode, alpha=1.0, eps=0.01, sweeps=2000, sigma=0.1, seed=3, n_chains=1):
    """d after every sweep (shape (sweeps, n_chains)) for SU(2) chains of
    n_links links, cooled from U_k = Om_k Om_{k+1}^{-1} (no Langevin update)."""
    cp = cl.make_cool(eps, alpha, MODES[mode], forced_sweeps=1)
    with cl.PolyakovChains(n_chains, n_links, 1.0, np.arange(seed, seed + n_chains), gauge_sigma=sigma) as pc:
        rec = pc.run(sweeps, 0.0, cp, obs_every=1)
    return rec[:, :, 2] - 1.0


def lattice_cooling(L, mode, alpha=1.0, eps=0.01, sweeps=500, sigma=0.1, seed=3, prec=cl.CL_FP64):
    """d after every sweep for an SU(3) lattice: cold start transformed by a
    random SL(3,C) gauge transformation (spread sigma), cooled one sweep per call."""
    cp = cl.make_cool(eps, alpha, MODES[mode], forced_sweeps=1)
    out = np.zeros(sweeps)
    with cl.Lattice(L, beta=6.0, prec=prec, seed=seed, start=cl.CL_START_COLD, gauge_sigma=sigma) as lat:
        for k in range(sweeps):
            rep = lat.cool(cp)
            out[k] = rep["un_after"] - 1.0
    return out


def summarize(d, thresholds=(1e-3, 1e-5), marks=(10, 100, 1000)):
    """Sweeps to reach each threshold (None if never), d at the marks and the
    log-log slope of d over the last decade of sweeps."""
    d = np.asarray(d, dtype=np.float64)
    n = len(d)
    out = {"first_sweep_below": {}, "d_at": {}}
    for t in thresholds:
        idx = np.nonzero(d <= t)[0]
        out["first_sweep_below"]["%g" % t] = int(idx[0]) + 1 if idx.size else None
    for m in marks:
        if m <= n:
            out["d_at"][str(m)] = float(d[m - 1])
    lo = max(1, n // 10)
    x = np.log(np.arange(lo, n) + 1.0)
    y = np.log(np.maximum(np.abs(d[lo:]), 1e-300))
    out["loglog_slope_last_decade"] = float(np.polyfit(x, y, 1)[0]) if n - lo > 2 else None
    out["d_final"] = float(d[-1])
    return out


def theta_scan(L=(6, 6, 6, 6), betas=(5.9, 6.0, 6.1), theta2=(0.0, 1.0, -1.0, 4.0, -4.0), n_steps=4000,
               eps=0.005, every=20, k_ref=12.0, seed=100, prec=cl.CL_FP64, cool=None):
    """theta_L = sqrt(theta_L^2): real for theta_L^2 > 0, imaginary for < 0.
    One batch of len(betas) * len(theta2) chains; every `every` steps the
    plaquette and Q_L of each chain are recorded.  Returns a list of dicts
    (beta, theta2, plaquette and Q series)."""
    cp = cool if cool is not None else cl.make_cool(eps, 0.1, cl.CL_D2_MEANABS, n_min=0, n_max=10,
                                                    tol_rel=0.01, d_floor=1e-6)
    specs = [(b, t2) for b in betas for t2 in theta2]
    lats = []
    for i, (b, t2) in enumerate(specs):
        th = np.sqrt(t2) if t2 >= 0 else 1j * np.sqrt(-t2)
        lat = cl.Lattice(L, beta=b, theta=th, prec=prec, seed=seed + i, start=cl.CL_START_COLD,
                         own_stream=True)
        lat.set_adaptive_step(k_ref)
        lats.append(lat)
    series = [[] for _ in specs]
    try:
        with cl.Batch(lats, eps, [cp] * len(lats)) as b:
            for _ in range(n_steps // every):
                b.run(every)
                b.synchronize()
                for i, lat in enumerate(lats):
                    series[i].append(cl.cl_observables(lat.h, check=False))
        times = [lat.langevin_time()[0] for lat in lats]
    finally:
        for lat in lats:
            lat.close()
    out = []
    for (b, t2), ser, t in zip(specs, series, times):
        out.append({"beta": b, "theta2": t2, "langevin_time": t,
                    "plaq": np.array([o["plaq_re"] + 1j * o["plaq_im"] for o in ser]),
                    "q": np.array([o["q_re"] + 1j * o["q_im"] for o in ser]),
                    "un": np.array([o["un"] for o in ser])})
    return out


OBS_KEYS = ("plaq_re", "plaq_im", "un", "q_re", "q_im", "sw_re", "sw_im", "s_re", "s_im", "max_det_dev")


def precision_table(L=(32, 32, 32, 32), beta=6.2, theta=1.0, eps=0.005, sweeps=10, checkpoints=(1, 10, 100),
                    seed=1, prec=None):
    """A reduced-precision form (FP32 storage by default, or DF64) vs FP64 on
    the same workload as the throughput bench (Haar start, fixed count of D_1
    sweeps).  Returns {n_steps: {"links": max abs difference, observable:
    (fp64 value, abs difference, relative difference)}}."""
    prec = cl.CL_FP32_STORAGE if prec is None else prec
    cp = cl.make_cool(eps, 1.0, cl.CL_D1, forced_sweeps=sweeps)
    out = {}
    with cl.Lattice(L, beta=beta, theta=theta, prec=cl.CL_FP64, seed=seed, start=cl.CL_START_HOT) as a, \
            cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=seed, start=cl.CL_START_HOT) as b:
        done = 0
        for n in sorted(checkpoints):
            for lat in (a, b):
                for _ in range(n - done):
                    lat.step(eps, 1)
                    lat.cool(cp, want_report=False)
            done = n
            oa, ob = a.observables(), b.observables()
            row = {"links": float(np.abs(a.links() - b.links()).max())}
            for k in OBS_KEYS:
                d = abs(ob[k] - oa[k])
                row[k] = (oa[k], d, d / abs(oa[k]) if oa[k] != 0 else None)
            out[n] = row
    return out


SERIES_KEYS = ("plaq_re", "plaq_im", "un", "q_re", "q_im")


def longrun_cool(eps=0.005):
    """The adaptive rule of the long runs: alpha_ad = 0.1 / D_2 (D_2 = <|f_ax|>),
    0..10 sweeps, stop below 1 % relative progress or within 1e-6 of SU(3)."""
    return cl.make_cool(eps, 0.1, cl.CL_D2_MEANABS, n_min=0, n_max=10, tol_rel=0.01, d_floor=1e-6)


def longrun(L, beta, theta, prec, seeds, n_steps, every=10, eps=0.005, cool=None, k_ref=0.0):
    """Chains from the cold start, one per seed, advanced together (one batch
    graph launch per step); every `every` steps the observables of each chain.
    Returns an array (n_chains, n_steps // every, len(SERIES_KEYS))."""
    cp = cool if cool is not None else longrun_cool(eps)
    lats = []
    for sd in seeds:
        lat = cl.Lattice(L, beta=beta, theta=theta, prec=prec, seed=int(sd), start=cl.CL_START_COLD,
                         own_stream=True)
        if k_ref > 0.0:
            lat.set_adaptive_step(k_ref)
        lats.append(lat)
    out = np.zeros((len(lats), n_steps // every, len(SERIES_KEYS)))
    try:
        with cl.Batch(lats, eps, [cp] * len(lats)) as b:
            for r in range(n_steps // every):
                b.run(every)
                b.synchronize()
                for i, lat in enumerate(lats):
                    o = cl.cl_observables(lat.h, check=False)
                    out[i, r] = [o[k] for k in SERIES_KEYS]
    finally:
        for lat in lats:
            lat.close()
    return out


def chain_means(series, drop=0.2):
    """Per-chain means after dropping the first `drop` of each series
    (thermalisation), then the ensemble mean and its standard error from the
    chain-to-chain scatter (the chains are independent).  Chains with a
    non-finite record are left out and counted."""
    series = np.asarray(series)
    n0 = int(series.shape[1] * drop)
    ok = np.all(np.isfinite(series), axis=(1, 2))
    m = series[ok, n0:, :].mean(axis=1)
    k = m.shape[0]
    mean = m.mean(axis=0)
    err = m.std(axis=0, ddof=1) / np.sqrt(k) if k > 1 else np.full(m.shape[1], np.inf)
    return {"mean": mean, "err": err, "chains": k, "dropped": int((~ok).sum())}


def compare_means(a, b, rel_floor=1e-12):
    """z = |mean_a - mean_b| / sqrt(err_a^2 + err_b^2 + floor^2) per
    observable, floor = rel_floor * max(1, |mean|): the rounding level of the
    coarser form, below which two means count as equal (UN = 1 on SU(3) is
    exact in one form and 1 + O(rounding) in another)."""
    d = np.abs(a["mean"] - b["mean"])
    floor = rel_floor * np.maximum(1.0, np.abs(a["mean"]))
    return d / np.sqrt(a["err"] ** 2 + b["err"] ** 2 + floor ** 2)
