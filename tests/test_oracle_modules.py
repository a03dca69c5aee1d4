"""Pins of the oracle's module planes (Sec. 3.1: module position and normal, the Phase-2 tilted
modules) and of the overlap-hit pickup (Sec. 2.2: a single additional detector-overlap hit).

The plane step is pinned by what geometry fixes: its crossing lies on the helix and on the plane
and is the crossing nearest to the state (brute-force scan), a plane z = z_d reproduces the disk
step's independent closed form, the Jacobian matches central finite differences and obeys the
chain rule through an intermediate plane.  The search and the fit on simulated modular events
are pinned by the simulation's truth (which hits, which overlap hits) and by unit pulls."""
import numpy as np
import pytest

import oracle
from oracle import parity as PR
from paper_2312_11728_gb300 import pipeline, synth as S


@pytest.fixture(scope="module")
def geo():
    return S.geometry_phase2_modular()


def _states(rng, n, r=36.0):
    """States on a cylinder of radius r, moving outward, pT 0.5-20 GeV, |eta| < 2."""
    phi_pos = rng.uniform(-np.pi, np.pi, n)
    eta = rng.uniform(-2, 2, n)
    th = 2 * np.arctan(np.exp(-eta))
    pt = np.exp(rng.uniform(np.log(0.5), np.log(20.0), n))
    k = rng.choice([-1.0, 1.0], n) / pt
    phi = phi_pos + rng.uniform(-0.4, 0.4, n)
    z = r / np.tan(th)
    return np.stack([r * np.cos(phi_pos), r * np.sin(phi_pos), z, k, phi, th], -1)


def _planes(rng, p):
    """A tilted plane a few mm from each state: normal in the r-z plane, tilted towards the
    track's polar direction (as the modules facing the origin are) within +-0.3 rad."""
    rh = np.array([np.cos(np.arctan2(p[1], p[0])), np.sin(np.arctan2(p[1], p[0])), 0.0])
    beta = 0.5 * np.pi - p[5] + rng.uniform(-0.3, 0.3)
    n = np.cos(beta) * rh + np.array([0.0, 0.0, np.sin(beta)])
    n /= np.linalg.norm(n)
    c = p[:3] + rng.uniform(-0.5, 0.5) * n + rng.uniform(-1, 1) * np.cross(n, [0, 0, 1.0])
    return c, n


def test_plane_crossing_is_nearest_root(geo):
    orc = oracle.Oracle(geo)
    rng = np.random.default_rng(3)
    P = _states(rng, 60)
    for p in P:
        c, n = _planes(rng, p)
        ok, s, _ = orc.path_plane(p, c, n)
        assert ok
        q = orc.helix(p, s)
        assert abs(np.dot(q[:3] - c, n)) < 1e-10
        # brute force: every sign change of g(s) = n.(x(s) - c) on a fine grid of [-10, 10]
        grid = np.linspace(-10, 10, 4001)
        g = np.array([np.dot(orc.helix(p, t)[:3] - c, n) for t in grid])
        roots = grid[:-1][np.sign(g[:-1]) != np.sign(g[1:])]
        assert roots.size >= 1
        assert abs(abs(s) - np.min(np.abs(roots))) < 6e-3


def test_plane_z_equals_disk_step(geo):
    """The plane z = z_d with normal z-hat is the disk: same path length (s = (z_d - z) tan theta)
    and the same Jacobian as the disk layer's step."""
    orc = oracle.Oracle(geo)
    rng = np.random.default_rng(5)
    disk = int(np.nonzero((geo.kind == S.DISK) & (geo.pos > 0))[0][0])
    zd = float(geo.pos[disk])
    for _ in range(30):
        p = np.array([rng.uniform(5, 20), rng.uniform(-5, 5), zd - rng.uniform(0.2, 4.0),
                      rng.choice([-1, 1]) / rng.uniform(1.0, 20.0), rng.uniform(-np.pi, np.pi),
                      rng.uniform(0.2, 0.6)])
        ok, s, _ = orc.path_plane(p, [0, 0, zd], [0, 0, 1.0])
        ok2, s2, _ = orc.path(disk, p)
        assert ok
        assert abs(s - (zd - p[2]) * np.tan(p[5])) < 1e-9 * (1 + abs(s))
        if ok2:
            assert abs(s - s2) < 1e-9 * (1 + abs(s))
            np.testing.assert_allclose(orc.jacobian_plane(p, s, [0, 0, 1.0]), orc.jacobian(disk, p, s2),
                                       rtol=1e-9, atol=1e-12)


def _plane_map(orc, p, c, n):
    ok, s, _ = orc.path_plane(p, c, n)
    assert ok
    return orc.helix(p, s)


def test_plane_jacobian_finite_differences(geo):
    orc = oracle.Oracle(geo)
    rng = np.random.default_rng(7)
    P = _states(rng, 25)
    h = np.array([1e-5, 1e-5, 1e-5, 1e-7, 1e-7, 1e-7])
    for p in P:
        c, n = _planes(rng, p)
        ok, s, _ = orc.path_plane(p, c, n)
        J = orc.jacobian_plane(p, s, n)
        Jn = np.zeros((6, 6))
        for j in range(6):
            e = np.zeros(6)
            e[j] = h[j]
            Jn[:, j] = (_plane_map(orc, p + e, c, n) - _plane_map(orc, p - e, c, n)) / (2 * h[j])
        np.testing.assert_allclose(J, Jn, rtol=1e-5, atol=2e-6)


def test_plane_chain_rule(geo):
    """Two steps through an intermediate plane give the direct step's parameters, and the product
    of their Jacobians equals the direct Jacobian (all maps between surfaces)."""
    orc = oracle.Oracle(geo)
    rng = np.random.default_rng(11)
    for p in _states(rng, 20):
        c1, n1 = _planes(rng, p)
        ok, s1, _ = orc.path_plane(p, c1, n1)
        q1 = orc.helix(p, s1)
        c2 = q1[:3] + 0.4 * n1
        n2 = n1 + np.array([0.05, -0.03, 0.08])
        n2 /= np.linalg.norm(n2)
        ok2, s2, _ = orc.path_plane(q1, c2, n2)
        okd, sd, _ = orc.path_plane(p, c2, n2)
        assert ok and ok2 and okd
        q2 = orc.helix(q1, s2)
        qd = orc.helix(p, sd)
        np.testing.assert_allclose(q2, qd, rtol=1e-10, atol=1e-10)
        J12 = orc.jacobian_plane(q1, s2, n2) @ orc.jacobian_plane(p, s1, n1)
        # the first map's Jacobian is taken on its plane: project out the direction along which
        # the first plane's state cannot move (n1 . position) by comparing on the plane states
        Jd = orc.jacobian_plane(p, sd, n2)
        np.testing.assert_allclose(J12, Jd, rtol=1e-7, atol=1e-9)


def test_plane_step_transports_covariance(geo):
    """propagate_plane = crossing, helix and J C J^T; the covariance has no variance along the
    plane's normal (the state is on the plane)."""
    orc = oracle.Oracle(geo)
    rng = np.random.default_rng(13)
    for p in _states(rng, 10):
        c, n = _planes(rng, p)
        A = rng.standard_normal((6, 6)) * np.array([1e-2, 1e-2, 1e-2, 1e-3, 1e-3, 1e-3])
        C6 = A @ A.T
        c21 = C6[np.tril_indices(6)]
        ok, q, cq, s = orc.propagate_plane(p, c21, c, n)
        assert ok
        J = orc.jacobian_plane(p, s, n)
        M = np.zeros((6, 6))
        M[np.tril_indices(6)] = cq
        M = M + np.tril(M, -1).T
        np.testing.assert_allclose(M, J @ C6 @ J.T, rtol=1e-10, atol=1e-16)
        assert abs(n @ M[:3, :3] @ n) < 1e-12 * np.trace(M[:3, :3])


def _modular_batch(geo, n_events=2, n_tracks=400, noise=1500, seed=21):
    evs = [S.simulate_event(geo, n_tracks, seed, e, pt_sampler=S.sample_pt_phase2, eta_max=2.5, noise_total=noise)
           for e in range(n_events)]
    return S.concat_events(evs, geo.n_layers)


def _oracle_with_modules(geo, batch, params=None):
    orc = oracle.Oracle(geo, params or S.default_params())
    orc.set_modules(geo.modules.c, geo.modules.n, batch.hit_mod)
    return orc


@pytest.mark.parametrize("disks", [False, True])
def test_module_search_finds_true_hits_and_overlaps(geo, disks):
    """On modular events the search takes the true hit on most modular layer crossings and picks
    up the true overlap hit where the track crossed two modules; every overlap hit lies on the
    same layer as, and on another module than, the step's hit.  disks: the endcaps' 4th-6th disks
    built from planar modules too."""
    if disks:
        geo = S.geometry_phase2_modular_disks()
    batch = _modular_batch(geo)
    orc = _oracle_with_modules(geo, batch)
    o = PR.oracle_build(orc, batch)
    good = good_n = ovl_ok = ovl_n = 0
    L = batch.n_layers
    for k, si in enumerate(o["seed_index"]):
        if not np.isfinite(o["score"][k]):
            continue
        e = int(batch.seed_event[si])
        ev = batch.events[e]
        base = int(batch.hit_off[e * L])
        t = int(batch.seed_track[si])
        plan = geo.plans[o["region"][k]]
        for step, lay in enumerate(plan):
            h, ov = o["hits"][k, step], o["ovl"][k, step]
            if ov >= 0:
                assert h >= 0 and batch.hit_mod[ov] >= 0 and batch.hit_mod[ov] != batch.hit_mod[h]
                assert geo.modules.layer[batch.hit_mod[ov]] == lay == geo.modules.layer[batch.hit_mod[h]]
            if lay not in geo.modules.grid:
                assert ov < 0
                continue
            j = np.nonzero(ev.track_layers[t] == lay)[0]
            if j.size == 0:
                continue
            good_n += 1
            good += int(h == ev.track_hits[t, j[0]] + base or h == ev.track_ovl[t, j[0]] + base)
            if ev.track_ovl[t, j[0]] >= 0:
                ovl_n += 1
                pair = {ev.track_hits[t, j[0]] + base, ev.track_ovl[t, j[0]] + base}
                ovl_ok += int({h, ov} == pair)
    assert good_n > 500 and good / good_n > 0.95, (good, good_n)
    assert ovl_n > 50 and ovl_ok / ovl_n > 0.85, (ovl_ok, ovl_n)


def test_overlap_bonus_raises_score_only(geo):
    """score_overlap changes the score by exactly score_overlap per picked-up overlap hit where
    the hit lists agree (the bonus is uniform over a candidate's module-hit children)."""
    batch = _modular_batch(geo, n_events=1, n_tracks=300, seed=23)
    o0 = PR.oracle_build(_oracle_with_modules(geo, batch, S.default_params(score_overlap=0.0)), batch)
    o1 = PR.oracle_build(_oracle_with_modules(geo, batch, S.default_params(score_overlap=1.5)), batch)
    same = np.all(o0["hits"] == o1["hits"], 1) & np.all(o0["ovl"] == o1["ovl"], 1) & np.isfinite(o0["score"])
    assert same.mean() > 0.9
    nov = (o1["ovl"] >= 0).sum(1)
    assert nov[same].sum() > 20
    np.testing.assert_allclose(o1["score"][same] - o0["score"][same], 1.5 * nov[same], atol=1e-9)
    assert np.all(o0["chi2"][same] == o1["chi2"][same])


def test_seed_on_module_planes_recovers_truth():
    """Seeding cylinders built from modules, noise-free hits, no material: the seed fit takes each
    hit on its module's plane and ends on the third hit with the helix's own parameters (three
    exact points of a helix fix it); the same seeds with the hits taken on the cylinders miss it."""
    g = S.geometry_phase2_modular(layers=(0, 1, 2))
    ev = S.simulate_event(g, 200, 27, 0, pt_sampler=S.sample_pt_phase2, eta_max=1.0, noise_total=0,
                          material=False, smear=False)
    b = S.concat_events([ev], g.n_layers)
    params = dict(S.default_params(), material=0)
    sl = oracle.hit_layers(b.hit_off, b.seed_hits)
    X, V = b.hit_xyz.astype(np.float64), b.hit_cov.astype(np.float64)
    mod_seed = (b.hit_mod[b.seed_hits] >= 0).all(1)
    assert mod_seed.mean() > 0.8
    orc = _oracle_with_modules(g, b, params)
    r = orc.seed_batch(b.seed_hits, sl, X, V)
    ok = (r["status"] == 0) & mod_seed
    assert ok.sum() > 0.8 * mod_seed.sum()
    # truth: the hit itself for the position; q/pT and theta are constants of the helix without
    # material; the direction at the hit from the truth at the cylinder crossing: the chord between
    # two points of a circle runs along the mean of the tangent angles at its ends
    x3 = b.hit_xyz[b.seed_hits[ok, 2]].astype(np.float64)
    t3 = ev.track_truth[b.seed_track[ok], 2]
    alpha = np.arctan2(x3[:, 1] - t3[:, 1], x3[:, 0] - t3[:, 0])
    alpha = np.where(np.cos(alpha - t3[:, 4]) < 0, alpha + np.pi, alpha)
    phi3 = 2 * alpha - t3[:, 4]
    p = r["p"][ok]
    dpos = np.abs(p[:, :3] - x3).max(1)
    assert dpos.max() < 1e-4                                   # hits stored in float32
    assert np.abs(p[:, 3] / t3[:, 3] - 1).max() < 1e-3
    assert np.abs(p[:, 5] - t3[:, 5]).max() < 1e-5
    # the chord's angle carries the float32 rounding of the hit (~1e-6 cm) over the chord length
    chord = np.hypot(x3[:, 0] - t3[:, 0], x3[:, 1] - t3[:, 1])
    assert np.all(np.abs(np.angle(np.exp(1j * (p[:, 4] - phi3)))) < 1e-5 + 1e-5 / chord)
    orc.set_modules(None, None, None)
    r0 = orc.seed_batch(b.seed_hits, sl, X, V)
    ok0 = r0["status"][ok] == 0
    d0 = np.abs(r0["p"][ok][ok0, :3] - x3[ok0]).max(1)
    assert np.median(d0) > 100 * max(np.median(dpos), 1e-6)


def test_no_modules_is_plain_search(geo):
    """With the module table cleared, hits are taken on the reference cylinder and no overlap hit
    is ever picked up."""
    batch = _modular_batch(geo, n_events=1, n_tracks=200, seed=29)
    orc = _oracle_with_modules(geo, batch)
    orc.set_modules(None, None, None)
    o = PR.oracle_build(orc, batch)
    assert np.all(o["ovl"] == -1)


def test_modular_fit_pulls(geo):
    """Fit over the true assignment of modular events (module hits used on their planes): the
    pulls of the fitted parameters at the last hit against the simulation's truth have unit
    width; a fit that used module hits on the reference cylinder instead would not."""
    batch = _modular_batch(geo, n_events=2, n_tracks=600, noise=0, seed=31)
    fi = pipeline.fit_inputs(batch)
    orc = _oracle_with_modules(geo, batch, S.default_params())
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    r = orc.fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0)
    truth = []
    for e, ev in enumerate(batch.events):
        nh = (ev.track_layers >= 0).sum(1)
        sel = np.nonzero(nh >= 1)[0]
        truth.append(ev.track_truth[sel, nh[sel] - 1])
    truth = np.concatenate(truth)
    ok = (r["status"] == 0) & ((fi.layers >= 0).sum(1) >= 8)
    d = r["p"][ok][:, 3:] - truth[ok][:, 3:]
    d[:, 1] = np.angle(np.exp(1j * d[:, 1]))
    pulls = d / np.sqrt(r["c"][ok][:, [9, 14, 20]])
    # curvature, phi and theta at the last hit (on an outer cylinder or a disk)
    for i in range(3):
        assert abs(np.std(pulls[:, i]) - 1.0) < 0.12, (i, np.std(pulls[:, i]))
        assert abs(np.mean(pulls[:, i])) < 0.12
    orc.set_modules(None, None, None)
    r0 = orc.fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0)
    ok0 = (r0["status"] == 0) & ((fi.layers >= 0).sum(1) >= 8)
    assert np.median(r0["chi2"][ok0]) > 3 * np.median(r["chi2"][ok])


def test_modular_backward_fit_pulls_at_the_first_hit():
    """The backward fit (Sec. 2.2) through modular layers, module hits used on their planes:
    forward fit, then backward fit from the last hit; the pulls of the state on the innermost
    (plain) cylinder against the truth of the segment entering it (the helix from the origin, by
    the generator's own crossing and motion) have unit width."""
    g = S.add_modules(S.geometry_barrel(), [3, 4, 5])
    ev = S.simulate_event(g, 3000, 12, 0, eta_max=1.0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    batch = S.concat_events([ev], g.n_layers)
    orc = _oracle_with_modules(geo=g, batch=batch)
    layers, hits, p0, c0, _, nh, sel = S.fit_workload(ev)
    X, V = ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64)
    f = orc.fit_batch(layers, hits, X, V, p0, c0)
    b = orc.bkfit_batch(layers, hits, X, V, f["p"], f["c"], 100.0)
    ok = (f["status"] == 0) & (b["status"] == 0) & (layers[:, 0] == 0) & (nh >= 8)
    assert ok.mean() > 0.9
    assert (batch.hit_mod[hits[ok]] >= 0).any(1).mean() > 0.8   # the tracks cross module layers
    k0 = ev.track_q[sel] / ev.track_pt[sel]
    th0 = 2 * np.arctan(np.exp(-ev.track_eta[sel]))
    ph0 = ev.track_phi[sel]
    w = -S.C_LIGHT * g.bz * k0
    z0 = np.zeros_like(k0)
    s0 = S._cylinder_crossing(z0, z0, ph0, w, g.pos[0])
    xn, yn, zn, psi = S._move(z0, z0, z0, ph0, th0, w, s0)
    truth_in = np.stack([xn, yn, zn, k0, np.angle(np.exp(1j * psi)), th0], -1)
    P, Cm, T = b["p"][ok], b["c"][ok], truth_in[ok]
    d = P - T
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    for i, ci in ((3, 9), (4, 14), (5, 20), (2, 5)):
        pl = d[:, i] / np.sqrt(Cm[:, ci])
        assert abs(pl.mean()) < 0.08, i
        assert abs(pl.std() - 1.0) < 0.08, (i, pl.std())


def test_modular_backward_search_recovers_the_inner_hits():
    """Barrel tracks through modular cylinders 3-5 (100 noise hits per layer): with their first
    five layers removed, forward- and backward-fitted (module hits on their planes), the backward
    search (Sec. 2.2) from the state on cylinder 5 finds the true hits on layers 4, 3 (module
    planes) and 2, 1, 0 for nearly every track, and the true overlap hits where the track crossed
    two modules of a layer."""
    from paper_2312_11728_gb300 import pipeline
    g = S.add_modules(S.geometry_barrel(), [3, 4, 5])
    ev = S.simulate_event(g, 800, 22, 0, eta_max=1.0, noise_per_layer=100,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    batch = S.concat_events([ev], g.n_layers)
    o = _oracle_with_modules(geo=g, batch=batch)
    fi = pipeline.fit_inputs(batch)
    n_skip = 5
    keep = ((fi.layers >= 0).sum(1) >= n_skip + 3) & np.all(fi.layers[:, :n_skip] == np.arange(n_skip), 1)
    fo = pipeline.outer_fit_inputs(fi, n_skip)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    f = o.fit_batch(fo.layers, fo.hits, X, V, fo.p0, fo.c0)
    b = o.bkfit_batch(fo.layers, fo.hits, X, V, f["p"], f["c"], 100.0)
    ok = keep & (f["status"] == 0) & (b["status"] == 0)
    assert ok.mean() > 0.8
    idx = np.nonzero(ok)[0]
    r = o.build_backward_event(batch.hit_off[:g.n_layers + 1], X, V, b["p"][idx], b["c"][idx], fo.layers[idx, 0])
    # reversed barrel plan: step k is layer 9 - k; the removed layers 4..0 are steps 5..9.  On a
    # layer the track crossed twice, the search takes the better-fitting of the two true hits and
    # picks up the other one (one event: global hit ids = event-local ids)
    found, fovl = r["hits"][:, 5:10], r["ovl"][:, 5:10]
    truth, tovl = fi.hits[idx, 4::-1], ev.track_ovl[idx][:, 4::-1]
    one = (tovl < 0) & (found == truth) & (fovl < 0)
    two = (tovl >= 0) & (((found == truth) & (fovl == tovl)) | ((found == tovl) & (fovl == truth)))
    assert (one | two).all(1).mean() > 0.9, (one | two).all(1).mean()
    assert (tovl >= 0).sum() > 50 and two.sum() > 0.85 * (tovl >= 0).sum()
