"""Pins of the oracle's backward fit (Sec. 2.2: each found track re-traversed inwards, refitting
its parameters): the reversed trajectory, the inward crossing, the backward step, and the
backward fit on exact and on smeared hits.  Readings: the backward fit starts on the last
listed layer from the forward fit's state with its covariance scaled by 100, reverses the
direction of motion (k -> -k, phi -> phi + pi, theta -> pi - theta), crosses the inner layers
along the reversed helix and adds the mean energy loss back in each layer's material."""
import numpy as np
import pytest

import oracle
from paper_2312_11728_gb300 import synth as S

G = S.geometry_phase2()
CB = 0.00299792458 * float(G.bz)


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle(G, dict(material=0))


def sym(c):
    M = np.zeros((6, 6))
    M[np.tril_indices(6)] = c
    return M + np.tril(M, -1).T


def test_reverse_traces_the_same_points_backwards(orc):
    """Closed form: the reversed state at path s sits where the original was at -s, moving the
    opposite way; reversing twice is the identity."""
    rng = np.random.default_rng(1)
    for _ in range(200):
        p = np.array([rng.uniform(-50, 50), rng.uniform(-50, 50), rng.uniform(-100, 100),
                      rng.choice([-1, 1]) / rng.uniform(0.5, 20), rng.uniform(-np.pi, np.pi), rng.uniform(0.2, 2.9)])
        A = rng.standard_normal((6, 6))
        c = (A @ A.T)[np.tril_indices(6)]
        pr, cr = orc.reverse(p, c)
        p2, c2 = orc.reverse(pr, cr)
        assert np.allclose(p2, p, atol=1e-12) and np.allclose(c2, c, atol=1e-12)
        for s in rng.uniform(0.1, 40, 3):
            a, b = orc.helix(pr, s), orc.helix(p, -s)
            assert np.allclose(a[:3], b[:3], atol=1e-9)
            assert abs(np.angle(np.exp(1j * (a[4] - b[4] - np.pi)))) < 1e-9
            assert abs(a[5] - (np.pi - b[5])) < 1e-12
        # covariance of the reversed parameters: the linear map diag(1,1,1,-1,1,-1)
        D = np.diag([1, 1, 1, -1, 1, -1.0])
        assert np.allclose(sym(cr), D @ sym(c) @ D, atol=1e-12)


def test_inward_crossing_matches_circle_intersection(orc):
    """States outside a barrel layer moving inward: the crossing equals the generator's
    circle-circle intersection (the first positive root along the motion), lies on the cylinder,
    and the radius stays above R before it."""
    rng = np.random.default_rng(2)
    barrels = [i for i in range(G.n_layers) if G.kind[i] == S.BARREL]
    n_checked = n_missed = 0
    for _ in range(600):
        lay = int(rng.choice(barrels[:-1]))
        R = G.pos[lay]
        r0 = rng.uniform(R + 0.5, 110.0)
        a = rng.uniform(-np.pi, np.pi)
        # direction with an inward radial component
        phi = a + np.pi + rng.uniform(-1.2, 1.2)
        k = rng.choice([-1, 1]) / np.exp(rng.uniform(np.log(0.5), np.log(50)))
        p = np.array([r0 * np.cos(a), r0 * np.sin(a), rng.uniform(-20, 20), k, np.angle(np.exp(1j * phi)),
                      rng.uniform(1.2, 1.9)])
        ok, s, _ = orc.path_inward(lay, p)
        w = -CB * k
        s_ref = S._cylinder_crossing(p[:1], p[1:2], p[4:5], np.array([w]), R)[0]
        if not np.isfinite(s_ref):
            assert not ok
            n_missed += 1
            continue
        q = orc.helix(p, s_ref)
        if not (G.lo[lay] <= q[2] <= G.hi[lay]):
            assert not ok
            continue
        assert ok
        assert abs(s - s_ref) < 1e-8 * max(1.0, s_ref)
        q = orc.helix(p, s)
        assert abs(np.hypot(q[0], q[1]) - R) < 1e-10 * R
        grid = np.linspace(0, s, 100)[1:-1]
        assert min(np.hypot(*orc.helix(p, t)[:2]) for t in grid) > R
        n_checked += 1
    assert n_checked > 200 and n_missed > 5


def test_backward_step_undoes_the_forward_step(orc):
    """Material off: inner surface -> outer surface (forward) -> inner surface (backward) is the
    identity on the state and on a surface-constrained covariance (J_bwd J_fwd = 1 there)."""
    rng = np.random.default_rng(3)
    n = 0
    for _ in range(300):
        k = rng.choice([-1, 1]) / np.exp(rng.uniform(np.log(0.7), np.log(30)))
        p = np.array([0.0, 0.0, rng.uniform(-5, 5), k, rng.uniform(-np.pi, np.pi), rng.uniform(1.1, 2.0)])
        A = rng.standard_normal((6, 6)) * np.array([0.01, 0.01, 0.01, 0.05 * abs(k), 0.003, 0.003])
        c = (A @ A.T)[np.tril_indices(6)]
        lin, lout = sorted(rng.choice(10, 2, replace=False))
        r1, p1, c1, _ = orc.propagate(lin, p, c, material=0)       # onto the inner surface
        if r1 != 1:
            continue
        r2, p2, c2, _ = orc.propagate(lout, p1, c1, material=0)
        if r2 != 1:
            continue
        r3, p3, c3, _ = orc.propagate_backward(lin, p2, c2, material=0)
        assert r3 == 1
        d = p3 - p1
        d[4] = np.angle(np.exp(1j * d[4]))
        assert np.abs(d).max() < 1e-9
        M1, M3 = sym(c1), sym(c3)
        sc = np.sqrt(np.outer(np.diag(M1), np.diag(M1)))
        assert np.all(np.abs(M3 - M1) <= 1e-7 * sc + 1e-18)
        n += 1
    assert n > 100


def test_backward_step_adds_the_energy_back(orc):
    """Material on: the backward step through a layer raises |p| (|k| falls) and adds the same
    Highland variance to the angles as the forward step through that layer."""
    o = oracle.Oracle(G, dict(material=1))
    p = np.array([0.0, 0.0, 0.0, 1.0 / 0.8, 0.3, 1.4])
    c = (np.eye(6) * 1e-6)[np.tril_indices(6)]
    r, p5, c5, _ = o.propagate(5, p, c, material=0)
    assert r == 1
    r, pb, cb, _ = o.propagate_backward(2, p5, c5, material=1)
    r0, pb0, cb0, _ = o.propagate_backward(2, p5, c5, material=0)
    assert r == 1 and r0 == 1
    assert abs(pb[3]) < abs(pb0[3])
    # the variance added to theta equals the forward material step's at the same crossing
    pr, cr = o.reverse(pb0, cb0)
    ok, pm, cm = o.material(2, pr, cr, direction=-1.0)
    assert ok and np.isclose(sym(cb)[5, 5] - sym(cb0)[5, 5], sym(cm)[5, 5] - sym(cr)[5, 5], rtol=1e-9)


def _fit_then_backfit(o, ev, scale=100.0, from_truth=False):
    layers, hits, p0, c0, truth_last, nh, sel = S.fit_workload(ev)
    if from_truth:   # start the forward fit exactly on the simulated helix (at the origin)
        k = ev.track_q[sel] / ev.track_pt[sel]
        th = 2 * np.arctan(np.exp(-ev.track_eta[sel]))
        p0 = np.stack([0 * k, 0 * k, 0 * k, k, ev.track_phi[sel], th], -1)
    xyz, cov = ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64)
    f = o.fit_batch(layers, hits, xyz, cov, p0, c0)
    b = o.bkfit_batch(layers, hits, xyz, cov, f["p"], f["c"], scale)
    return f, b, sel


def test_noise_free_backward_fit_recovers_the_first_hit_state():
    """Exact helix hits, no material: the backward-fitted state at the innermost hit equals the
    simulated truth there (to the float32 storage of the hits), with vanishing chi2."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g, dict(material=0))
    ev = S.simulate_event(g, 300, 5, 0, eta_max=1.0, material=False, smear=False)
    f, b, sel = _fit_then_backfit(o, ev, from_truth=True)
    assert np.all(f["status"] == 0) and np.all(b["status"] == 0)
    truth_first = ev.track_truth[sel, 0]
    d = b["p"] - truth_first
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    assert np.abs(d[:, :3]).max() < 2e-5
    assert np.abs(d[:, 3:]).max() < 2e-5
    assert b["chi2"].max() / b["nupd"].min() < 1e-3


def test_backward_fit_pulls_at_the_first_hit_are_unit_normal():
    """Smeared hits with material: pulls of the backward-fitted state against the truth of the
    segment that enters the innermost layer (the backward step through a layer adds its
    material, so the state describes the track before that layer's scattering in the flight
    direction: for the first layer, the helix from the origin, computed with the event
    generator's own crossing and motion).  The reused forward information, scaled by 1/100,
    narrows the pulls by ~1%."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 4000, 11, 0, eta_max=1.0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    f, b, sel = _fit_then_backfit(o, ev)
    ok = (f["status"] == 0) & (b["status"] == 0)
    assert ok.mean() > 0.99
    k0 = ev.track_q[sel] / ev.track_pt[sel]
    th0 = 2 * np.arctan(np.exp(-ev.track_eta[sel]))
    ph0 = ev.track_phi[sel]
    w = -CB * k0
    lay0 = S.fit_workload(ev)[0][:, 0]
    assert np.all(lay0 == 0)
    z0 = np.zeros_like(k0)
    s0 = S._cylinder_crossing(z0, z0, ph0, w, g.pos[0])
    xn, yn, zn, psi = S._move(z0, z0, z0, ph0, th0, w, s0)
    truth_in = np.stack([xn, yn, zn, k0, np.angle(np.exp(1j * psi)), th0], -1)
    assert np.allclose(truth_in[:, :3], ev.track_truth[sel, 0, :3], atol=1e-9)
    P, Cm, T = b["p"][ok], b["c"][ok], truth_in[ok]
    d = P - T
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    phi = np.arctan2(P[:, 1], P[:, 0])
    t = np.stack([-np.sin(phi), np.cos(phi)], -1)
    var_t = t[:, 0] ** 2 * Cm[:, 0] + 2 * t[:, 0] * t[:, 1] * Cm[:, 1] + t[:, 1] ** 2 * Cm[:, 2]
    pulls = {"rphi": (d[:, :2] * t).sum(1) / np.sqrt(var_t),
             "z": d[:, 2] / np.sqrt(Cm[:, 5]), "k": d[:, 3] / np.sqrt(Cm[:, 9]),
             "phi": d[:, 4] / np.sqrt(Cm[:, 14]), "theta": d[:, 5] / np.sqrt(Cm[:, 20])}
    for name, pl in pulls.items():
        assert abs(pl.mean()) < 0.06, name
        assert abs(pl.std() - 1.0) < 0.06, (name, pl.std())
    # the inner-layer state knows the track better than the forward fit's first hit prior did
    assert np.median(Cm[:, 9]) < np.median(f["c"][ok, 9]) * 10


def _backward_search_inputs(g, ev, o, n_skip=3):
    """Tracks with their first n_skip layers removed, forward- then backward-fitted: the start
    states of a backward search on their innermost remaining layer."""
    from paper_2312_11728_gb300 import pipeline
    batch = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(batch)
    keep = (fi.layers >= 0).sum(1) >= n_skip + 3
    fo = pipeline.outer_fit_inputs(fi, n_skip)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    f = o.fit_batch(fo.layers, fo.hits, X, V, fo.p0, fo.c0)
    b = o.bkfit_batch(fo.layers, fo.hits, X, V, f["p"], f["c"], 100.0)
    ok = keep & (f["status"] == 0) & (b["status"] == 0)
    return batch, fi, fo, b, ok


def test_backward_search_recovers_the_inner_hits():
    """Barrel tracks with 200 noise hits per layer: started from the backward fit of their hits
    beyond the first three layers, the backward search finds the true hits on those three
    layers for nearly every track (the plan reversed: steps 7, 8, 9 are layers 2, 1, 0)."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 800, 21, 0, eta_max=1.0, noise_per_layer=200,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    batch, fi, fo, b, ok = _backward_search_inputs(g, ev, o)
    assert ok.mean() > 0.95
    idx = np.nonzero(ok)[0]
    r = o.build_backward_event(batch.hit_off[:g.n_layers + 1], batch.hit_xyz.astype(np.float64),
                               batch.hit_cov.astype(np.float64), b["p"][idx], b["c"][idx], fo.layers[idx, 0])
    assert np.all(r["start"] == g.n_layers - fo.layers[idx, 0])
    # reversed barrel plan: step k is layer 9 - k; the removed layers 2, 1, 0 are steps 7, 8, 9
    found = r["hits"][:, 7:10]
    truth = fi.hits[idx, 2::-1]
    rate = (found == truth).all(1).mean()
    assert rate > 0.95, rate
    assert np.all(r["nfound"] <= 3) and np.mean(r["nfound"] == 3) > 0.95


def test_backward_search_binned_equals_brute_force():
    """The eta-phi bins are an index only: the backward search with the binned lookup and with
    a scan of every hit of the layer gives the same results."""
    g = S.geometry_phase2()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 300, 22, 0, eta_max=3.0, noise_total=3000, pt_sampler=S.sample_pt_phase2)
    batch, fi, fo, b, ok = _backward_search_inputs(g, ev, o)
    idx = np.nonzero(ok)[0]
    args = (batch.hit_off[:g.n_layers + 1], batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
            b["p"][idx], b["c"][idx], fo.layers[idx, 0])
    r1 = o.build_backward_event(*args, binned=True)
    r2 = o.build_backward_event(*args, binned=False)
    for k in ("hits", "nfound", "nholes", "start"):
        assert np.array_equal(r1[k], r2[k]), k
    assert np.array_equal(r1["params"], r2["params"]) and np.array_equal(r1["score"], r2["score"])
