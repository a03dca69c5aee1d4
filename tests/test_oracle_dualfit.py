"""Pins of the oracle's exact fit derivative (oracle/dualfit.py: the fit on forward-mode dual
numbers) against things other than itself: its values are the C oracle's fit (the same steps in
FP64), its derivatives converge with the C oracle's central differences as their step leaves the
rounding-noise regime, and at the true alignment with noise-free hits and no material (every
residual zero) the gradient of the sum of squares vanishes."""
import numpy as np
import pytest

import oracle
from oracle import dualfit as DF, gradient as OG
from paper_2312_11728_gb300 import pipeline, synth as S


def _hit_layer(batch):
    hl = np.zeros(batch.hit_xyz.shape[0], np.int64)
    for s in range(len(batch.hit_off) - 1):
        hl[batch.hit_off[s]:batch.hit_off[s + 1]] = s % batch.n_layers
    return hl


@pytest.fixture(scope="module")
def phase2_small():
    g = S.geometry_phase2()
    ev = S.simulate_event(g, 40, 3, 0, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=0)
    b = S.concat_events([ev], g.n_layers)
    return g, b, pipeline.fit_inputs(b)


def test_values_equal_the_c_oracle(phase2_small):
    """Per track: the same status and the same total chi2 as orc_fit_batch (barrel and disks)."""
    g, b, fi = phase2_small
    X, V = b.hit_xyz.astype(np.float64), b.hit_cov.astype(np.float64)
    r = oracle.Oracle(g, S.default_params()).fit_batch(fi.layers, fi.hits, X, V, fi.p0.astype(np.float64),
                                                       fi.c0.astype(np.float64))
    chi2, status, *_ = DF.gradient(g, fi.layers, fi.hits, X, V, fi.p0, fi.c0)
    assert np.array_equal(status, r["status"])
    ok = status == 0
    assert ok.mean() > 0.9
    assert np.allclose(chi2[ok], r["chi2"][ok], rtol=1e-11, atol=1e-12)


def test_derivatives_converge_with_central_differences(phase2_small):
    """Central differences of the C oracle approach the dual-number derivative as the step grows
    out of the chi2's rounding noise, until truncation takes over; at the best steps they agree
    to a few 1e-6 of the largest derivative of each kind."""
    g, b, fi = phase2_small
    hl = _hit_layer(b)
    chi2, status, dp0, dal, dxs = DF.gradient(g, fi.layers, fi.hits, b.hit_xyz, b.hit_cov, fi.p0, fi.c0)
    errs = []
    for h_ang in (1e-6, 1e-5):
        r = OG.fd_gradient(g, S.default_params(), fi.layers, fi.hits, b.hit_xyz, b.hit_cov, hl, fi.p0, fi.c0,
                           h_p0=(1e-4, 1e-4, 1e-4, 1e-5, h_ang, h_ang))
        ok = (status == 0) & (r[1] == 0)
        errs.append([np.abs(r[2][ok][:, k] - dp0[ok][:, k]).max() / np.abs(dp0[ok][:, k]).max() for k in (4, 5)])
    assert errs[1][0] < errs[0][0] and errs[1][1] < errs[0][1], errs
    assert max(errs[1]) < 5e-6, errs
    for k in range(4):
        assert np.abs(r[2][ok][:, k] - dp0[ok][:, k]).max() < 1e-4 * np.abs(dp0[ok][:, k]).max(), k
    used = np.unique(fi.layers[fi.layers >= 0])
    assert np.abs(r[3][used] - dal[used]).max() < 1e-5 * np.abs(dal[used]).max()
    assert np.abs(r[4][used] - dxs[used]).max() < 1e-5 * np.abs(dxs[used]).max()


def test_gradient_vanishes_at_the_true_alignment():
    """Noise-free hits placed at the generator's FP64 crossing points, no material, fits started
    at the true vertex state: every residual is zero up to the generator's crossing precision, so
    the chi2 and every derivative of it (alignment, thickness, starting state) vanish against the
    same tracks fitted to hits smeared by their 30 um errors."""
    g = S.geometry_phase2()
    ev = S.simulate_event(g, 25, 8, 0, pt_sampler=S.sample_pt_phase2, eta_max=2.5, noise_total=0,
                          material=False, smear=False)
    b = S.concat_events([ev], g.n_layers)
    layers, hits, p0, c0, _, nh, sel = S.fit_workload(ev, 8, sig_pos=0.0, sig_z=0.0, rel_k=0.0, sig_ang=0.0)
    c0 = np.zeros_like(c0)
    for i, s in enumerate((0.01, 0.01, 0.01, 1e-4, 1e-4, 1e-4)):
        c0[:, i * (i + 1) // 2 + i] = s
    X = b.hit_xyz.astype(np.float64)
    for t, tr in enumerate(sel):   # exact crossing points of the truth (FP64)
        for j in range(ev.track_hits.shape[1]):
            h = ev.track_hits[tr, j]
            if h >= 0:
                X[h] = ev.track_truth[tr, j, :3]
    V = b.hit_cov.astype(np.float64)
    chi2, st, dp0, dal, dxs = DF.gradient(g, layers, hits, X, V, p0, c0, material_on=False)
    ok = st == 0
    assert ok.mean() > 0.9
    assert chi2[ok].max() < 1e-12
    rng = np.random.default_rng(3)
    Xs = X + rng.standard_normal(X.shape) * np.sqrt(V[:, [0, 2, 5]])
    chi2s, sts, dp0s, dals, dxss = DF.gradient(g, layers, hits, Xs, V, p0, c0, material_on=False)
    oks = ok & (sts == 0)
    assert np.median(chi2s[oks]) > 1.0
    assert np.abs(dal).max() < 1e-5 * np.abs(dals).max()
    assert np.abs(dxs).max() == 0.0 and np.abs(dxss).max() == 0.0   # no material in these fits
    assert np.abs(dp0[oks]).max() < 1e-5 * np.abs(dp0s[oks]).max()
