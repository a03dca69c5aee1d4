"""Pins of the final fit's outlier rejection (Sec. 2.2: "final fit including outlier rejection";
the reading: a listed hit whose predicted chi2 exceeds a cut is not used, the layer is still
crossed).  Wrong hits planted in known assignments must be rejected, true hits kept, and the fit
must recover unit pulls; without a cut the fit is unchanged."""
import numpy as np

import oracle
from paper_2312_11728_gb300 import pipeline, synth as S


def _pulls(r, truth, ok):
    P, Cm, T = r["p"][ok], r["c"][ok], truth[ok]
    d = P - T
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    return {"k": d[:, 3] / np.sqrt(Cm[:, 9]), "phi": d[:, 4] / np.sqrt(Cm[:, 14]),
            "theta": d[:, 5] / np.sqrt(Cm[:, 20])}


def test_outlier_rejection_removes_planted_hits():
    g = S.geometry_barrel()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 3000, 41, 0, eta_max=1.0, noise_per_layer=300,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    batch = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(batch)
    layers, hits, p0, c0, truth_last, nh, sel = S.fit_workload(ev)
    bad, swaps = pipeline.plant_wrong_hits(batch, fi, 0.3, 7)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    clean = o.fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0, outlier_chi2=0.0)
    same = o.fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0, outlier_chi2=1e12)
    assert np.array_equal(clean["p"], same["p"]) and np.array_equal(clean["c"], same["c"])
    plain = o.fit_batch(fi.layers, bad, X, V, fi.p0, fi.c0, outlier_chi2=0.0)
    cut = o.fit_batch(fi.layers, bad, X, V, fi.p0, fi.c0, outlier_chi2=30.0)
    ok = (plain["status"] == 0) & (cut["status"] == 0) & (clean["status"] == 0)
    swapped = np.zeros(fi.layers.shape[0], bool)
    swapped[[i for i, _ in swaps]] = True
    # each swapped track loses (about) one update, the others none (chi2(3) > 30: p = 1e-6)
    lost = clean["nupd"] - cut["nupd"]
    assert np.mean(lost[ok & swapped] == 1) > 0.95
    assert np.mean(lost[ok & ~swapped] == 0) > 0.999
    # the rejected fit has unit pulls again; the plain fit of the swapped tracks does not
    for name, pl in _pulls(cut, truth_last, ok).items():
        assert abs(pl.std() - 1.0) < 0.06, (name, pl.std())
    pk = _pulls(plain, truth_last, ok & swapped)["phi"]
    assert pk.std() > 1.5
