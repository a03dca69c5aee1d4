"""Backward fit (Sec. 2.2, mkgb_fit_backward) against the oracle's backward fit, element by element
on the same inputs: the GPU forward fit's FP32 output is the start state of both, so the two
backward fits see identical inputs.  Tolerances as for the forward fit (oracle/parity.py)."""
import numpy as np
import pytest

import oracle
from oracle import parity as PR
from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mkgb.load_library()


def _workload(which):
    if which == "small_barrel":
        g, ev = S.workload_small_barrel()
        return g, S.concat_events([ev], g.n_layers)
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, 1501, 0, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=4000)
           for e in range(3)]
    return g, S.concat_events(evs, g.n_layers)


def _forward_then_backward(g, batch, params, fi=None, scale=100.0):
    ctx = pipeline.make_context(g, params)
    fi = fi or pipeline.fit_inputs(batch)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    n = fi.layers.shape[0]
    f = dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
             status=np.zeros(n, np.int32))
    ctx.fit(fi.layers, fi.hits, fi.p0, fi.c0, f["p"], f["c"], f["chi2"], f["status"])
    b = dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
             status=np.zeros(n, np.int32))
    ctx.fit_backward(fi.layers, fi.hits, f["p"], f["c"], b["p"], b["c"], b["chi2"], b["status"], cov_scale=scale)
    b["counters"] = ctx.counters(1)
    return ctx, fi, f, b


@pytest.mark.parametrize("which", ["small_barrel", "phase2_small"])
def test_backward_fit_matches_oracle(lib, which):
    g, batch = _workload(which)
    params = S.default_params()
    _, fi, f, b = _forward_then_backward(g, batch, params)
    orc = oracle.Oracle(g, params)
    r = orc.bkfit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
                        f["p"].astype(np.float64), f["c"].astype(np.float64), 100.0)
    ok_fwd = f["status"] == 0
    rep = PR.compare_fit(b, r, mask=ok_fwd)
    assert np.array_equal(b["status"][ok_fwd], r["status"][ok_fwd]), rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n"] > 0.95 * fi.layers.shape[0]
    # work counters: crossed backward steps and updates, as the oracle counts them on the same
    # inputs (all tracks, the forward fit's failures included, when every status agrees)
    if np.array_equal(b["status"], r["status"]):
        assert b["counters"][0] == r["counters"][0] and b["counters"][2] == r["counters"][2]


def test_backward_fit_fp64_path(lib):
    """precision = FP64: every backward fit in FP64, far inside the tolerances."""
    g, batch = _workload("phase2_small")
    params = dict(S.default_params(), precision=2)
    _, fi, f, b = _forward_then_backward(g, batch, params)
    r = oracle.Oracle(g, params).bkfit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64),
                                             batch.hit_cov.astype(np.float64), f["p"].astype(np.float64),
                                             f["c"].astype(np.float64), 100.0)
    rep = PR.compare_fit(b, r, mask=f["status"] == 0)
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    # the outputs are FP32 words: rounding the global-frame covariance to FP32 alone leaves up to
    # ~0.05 of the tolerance in the surface-normal row of the surface-frame comparison
    assert rep["worst_param"] < 0.05 and rep["worst_cov"] < 0.1, rep


def test_backward_fit_edge_cases(lib):
    """No tracks; a track with one listed layer (only the update on it); a track without hits
    (propagation only); cov_scale = 1; invalid arguments."""
    g, batch = _workload("small_barrel")
    params = S.default_params()
    fi = pipeline.fit_inputs(batch)
    ctx = pipeline.make_context(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    z = lambda *s, t=np.float32: np.zeros(s, t)
    ctx.fit_backward(z(0, 5, t=np.int32), z(0, 5, t=np.int32), z(0, 6), z(0, 21), z(0, 6), z(0, 21), z(0),
                     z(0, t=np.int32))
    n = 8
    layers, hits = fi.layers[:n].copy(), fi.hits[:n].copy()
    layers[0, 1:] = -1                  # one listed layer
    hits[1, :] = -1                     # no hits at all
    f = dict(p=z(n, 6), c=z(n, 21), chi2=z(n), status=z(n, t=np.int32))
    ctx.fit(layers, hits, fi.p0[:n], fi.c0[:n], f["p"], f["c"], f["chi2"], f["status"])
    orc = oracle.Oracle(g, params)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    for scale in (100.0, 1.0):
        b = dict(p=z(n, 6), c=z(n, 21), chi2=z(n), status=z(n, t=np.int32))
        ctx.fit_backward(layers, hits, f["p"], f["c"], b["p"], b["c"], b["chi2"], b["status"], cov_scale=scale)
        r = orc.bkfit_batch(layers, hits, X, V, f["p"].astype(np.float64), f["c"].astype(np.float64), scale)
        rep = PR.compare_fit(b, r)
        assert rep["status_bad"] == 0 and rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
        assert b["chi2"][1] == 0.0
    with pytest.raises(mkgb.MkgbError):
        ctx.fit_backward(layers, hits, f["p"], f["c"], z(n, 6), z(n, 21), z(n), z(n, t=np.int32), cov_scale=0.0)
    bad = hits.copy()
    bad[2, 0] = int(batch.hit_xyz.shape[0]) + 5
    with pytest.raises(mkgb.MkgbError):
        ctx.fit_backward(layers, bad, f["p"], f["c"], z(n, 6), z(n, 21), z(n), z(n, t=np.int32))


def test_backward_fit_full_size_sampled(lib):
    """1,000,000 tracks over 34 layers (10% curling at 0.5-0.7 GeV) on the device: forward fit
    then backward fit in FP32 (FP64 refit above kappa_fp64), a sample of 3000 against the
    oracle's backward fit from the same start states."""
    import torch
    g, evs = S.workload_loopers(n_events=50, n_tracks=20000, seed=7)
    batch = S.concat_events(evs, g.n_layers)
    fi = pipeline.fit_inputs(batch)
    n = fi.layers.shape[0]
    assert n > 900_000
    ctx = pipeline.make_context(g, S.default_params())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.load_hits(batch.n_events, batch.hit_off, dev(batch.hit_xyz), dev(batch.hit_cov))
    L, H = dev(fi.layers), dev(fi.hits)
    out = lambda: dict(p=torch.zeros((n, 6), device="cuda"), c=torch.zeros((n, 21), device="cuda"),
                       chi2=torch.zeros(n, device="cuda"), status=torch.zeros(n, dtype=torch.int32, device="cuda"))
    f, b = out(), out()
    ctx.fit(L, H, dev(fi.p0), dev(fi.c0), f["p"], f["c"], f["chi2"], f["status"])
    ctx.fit_backward(L, H, f["p"], f["c"], b["p"], b["c"], b["chi2"], b["status"])
    torch.cuda.synchronize()
    fh = {k: v.cpu().numpy() for k, v in f.items()}
    bh = {k: v.cpu().numpy() for k, v in b.items()}
    assert (bh["status"][fh["status"] == 0] == 0).mean() > 0.99
    rng = np.random.default_rng(13)
    s = np.sort(rng.choice(n, 3000, replace=False))
    r = oracle.Oracle(g, S.default_params()).bkfit_batch(
        fi.layers[s], fi.hits[s], batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
        fh["p"][s].astype(np.float64), fh["c"][s].astype(np.float64), 100.0)
    rep = PR.compare_fit({k: v[s] for k, v in bh.items()}, r, mask=fh["status"][s] == 0)
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep


def test_fits_with_outlier_rejection_match_oracle(lib):
    """Known assignments with wrong hits planted in 30% of the tracks, fitted forwards and then
    backwards with the outlier cut at 30: the same hits rejected and the same results as the
    oracle's fits, on the tracks without a chi2 within 1e-3 of the cut."""
    g, batch = _workload("phase2_small")
    params = dict(S.default_params(), fit_outlier_chi2=30.0)
    fi0 = pipeline.fit_inputs(batch)
    bad, swaps = pipeline.plant_wrong_hits(batch, fi0, 0.3, 9)
    assert len(swaps) > 0.2 * fi0.layers.shape[0]
    fi = pipeline.FitInputs(fi0.layers, bad, fi0.p0, fi0.c0, fi0.event)
    ctx, _, f, b = _forward_then_backward(g, batch, params, fi=fi)
    orc = oracle.Oracle(g, params)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    rf = orc.fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0)
    rep = PR.compare_fit(f, rf, mask=rf["near_cut"] == 0)
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n"] > 0.95 * fi.layers.shape[0]
    rb = orc.bkfit_batch(fi.layers, fi.hits, X, V, f["p"].astype(np.float64), f["c"].astype(np.float64), 100.0)
    m = (f["status"] == 0) & (rf["near_cut"] == 0) & (rb["near_cut"] == 0)
    rep = PR.compare_fit(b, rb, mask=m)
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    # the planted hits are gone: the forward fit used one update fewer on the swapped tracks
    ref = orc.fit_batch(fi0.layers, fi0.hits, X, V, fi0.p0, fi0.c0, outlier_chi2=0.0)
    sw = np.zeros(fi.layers.shape[0], bool)
    sw[[i for i, _ in swaps]] = True
    ok = (rf["status"] == 0) & (ref["status"] == 0)
    assert np.mean((ref["nupd"] - rf["nupd"])[ok & sw] == 1) > 0.9
