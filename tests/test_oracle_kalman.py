"""Pins of the oracle's chi2, Kalman update, seeding and fit: the information-filter
identity, the Joseph form, noise-free truth recovery, and the statistics (unit pulls,
chi2(3) per 3D hit) of fits to the independent event simulator."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2312_11728_gb300 import synth as S


def sym(c21):
    M = np.zeros((6, 6))
    M[np.tril_indices(6)] = c21
    return M + M.T - np.diag(np.diag(M))


def rand_spd(rng, n, scale):
    A = rng.standard_normal((n, n))
    M = A @ A.T + n * np.eye(n)
    d = np.asarray(scale)
    return M * np.outer(d, d) / n


@pytest.fixture(scope="module")
def orc():
    return oracle.Oracle(S.geometry_barrel())


def test_update_equals_information_filter(orc):
    """C+ = (C^-1 + H^T V^-1 H)^-1 and p+ = C+ (C^-1 p + H^T V^-1 m); chi2 is the minimum of the
    joint objective (p+ - p)^T C^-1 (p+ - p) + (m - H p+)^T V^-1 (m - H p+)."""
    rng = np.random.default_rng(1)
    H = np.hstack([np.eye(3), np.zeros((3, 3))])
    for _ in range(200):
        C = rand_spd(rng, 6, [0.01, 0.01, 0.02, 0.05, 0.003, 0.003])
        V = rand_spd(rng, 3, [0.003, 0.003, 0.01])
        p = rng.standard_normal(6) * 0.3
        p[5] = 1.0
        m = p[:3] + rng.standard_normal(3) * 0.01
        c21 = C[np.tril_indices(6)]
        v6 = V[np.tril_indices(3)]
        for joseph in (False, True):
            ok, po, co, x2 = orc.update(p, c21, m, v6, joseph=joseph)
            assert ok
            Ci = np.linalg.inv(C)
            Vi = np.linalg.inv(V)
            Cp = np.linalg.inv(Ci + H.T @ Vi @ H)
            pp = Cp @ (Ci @ p + H.T @ Vi @ m)
            pp[4] = np.angle(np.exp(1j * pp[4]))
            assert np.allclose(sym(co), Cp, rtol=1e-8, atol=1e-12 * np.abs(Cp).max())
            assert np.allclose(po, pp, atol=1e-10)
            J = (pp - p) @ Ci @ (pp - p) + (m - H @ pp) @ Vi @ (m - H @ pp)
            assert abs(x2 - J) < 1e-8 * max(1.0, J)
            ok2, x2b = orc.chi2(p, c21, m, v6)
            assert ok2 and abs(x2b - x2) < 1e-12 * max(1.0, x2)


def test_joseph_equals_standard_in_fp64(orc):
    rng = np.random.default_rng(2)
    for _ in range(200):
        C = rand_spd(rng, 6, [0.1, 0.1, 0.1, 0.5, 0.05, 0.05])
        V = rand_spd(rng, 3, [0.003, 0.003, 0.01])
        p = np.array([1.0, 2.0, 3.0, 0.5, 0.2, 1.1])
        m = p[:3] + 0.01
        _, p1, c1, _ = orc.update(p, C[np.tril_indices(6)], m, V[np.tril_indices(3)], joseph=False)
        _, p2, c2, _ = orc.update(p, C[np.tril_indices(6)], m, V[np.tril_indices(3)], joseph=True)
        M1, M2 = sym(c1), sym(c2)
        d = np.sqrt(np.outer(np.diag(M1), np.diag(M1)))
        assert np.all(np.abs(M1 - M2) <= 1e-10 * d + 1e-15)
        assert np.all(np.linalg.eigvalsh(M1) > 0)


def test_noise_free_fit_recovers_truth():
    g = S.geometry_barrel()
    o = oracle.Oracle(g, dict(material=0))
    ev = S.simulate_event(g, 300, 5, 0, eta_max=1.0, material=False, smear=False)
    layers, hits, p0, c0, truth_last, nh, sel = S.fit_workload(ev)
    # start exactly at the truth: every predicted residual is zero up to float32 storage of the hits
    k = ev.track_q[sel] / ev.track_pt[sel]
    th = 2 * np.arctan(np.exp(-ev.track_eta[sel]))
    p0 = np.stack([0 * k, 0 * k, 0 * k, k, ev.track_phi[sel], th], -1)
    r = o.fit_batch(layers, hits, ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64), p0, c0)
    assert np.all(r["status"] == 0)
    d = r["p"] - truth_last
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    assert np.abs(d[:, :3]).max() < 2e-5          # float32 hit storage: |x| <= 100 cm -> ~4e-6 rounding
    assert np.abs(d[:, 3:]).max() < 1e-6
    assert r["chi2"].max() / r["nupd"].min() < 1e-3   # residuals at the 1e-6 cm level vs 30 um errors


def test_seed_recovers_truth_on_noise_free_hits():
    """The circle through three exact helix points is the helix: k, phi and theta at hit 1 exact."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g, dict(material=0))
    ev = S.simulate_event(g, 200, 6, 0, eta_max=1.0, material=False, smear=False)
    xyz = ev.hit_xyz.astype(np.float64)
    sl = oracle.hit_layers(ev.layer_off, ev.seed_hits)
    n_ok = 0
    for i, tr in enumerate(ev.seed_track):
        h = xyz[ev.seed_hits[i]].ravel()
        v = ev.hit_cov[ev.seed_hits[i]].astype(np.float64).ravel()
        ok, p, c, pinit = o.seed(h, v, sl[i])
        assert ok
        t1 = ev.track_truth[tr, 0]
        t3 = ev.track_truth[tr, 2]
        assert abs(pinit[3] / t1[3] - 1) < 2e-4            # hits stored in float32
        assert abs(np.angle(np.exp(1j * (pinit[4] - t1[4])))) < 2e-5
        assert abs(pinit[5] - t1[5]) < 2e-5
        assert np.allclose(p[:3], t3[:3], atol=1e-4)
        assert abs(p[3] / t3[3] - 1) < 1e-3
        assert abs(np.angle(np.exp(1j * (p[4] - t3[4])))) < 1e-4
        n_ok += 1
    assert n_ok == len(ev.seed_track)


def test_seed_of_a_straight_track_and_of_a_very_stiff_one():
    """Three hits on a straight line (q/pT = 0): the prior takes the line (no circle through three
    collinear points) and the fit ends on hit 3 with q/pT 0 and the line's angles.  A 500 TeV track,
    whose three points bend by ~1e-8 of the chord squared (the range where a coarser straight-line
    threshold would take the line instead), gets the circle's q/pT as its prior and keeps it."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g, dict(material=0))
    r = np.asarray(g.pos[:3], np.float64)
    v = np.tile(np.array([1e-6, 0.0, 1e-6, 0.0, 0.0, 1e-5]), 3)
    for phi0, cot in ((0.3, 0.2), (-2.5, -0.7), (1.9, 0.0)):
        h = np.stack([r * np.cos(phi0), r * np.sin(phi0), 1.5 + r * cot], 1).ravel()
        ok, p, c, pinit = o.seed(h, v, [0, 1, 2])
        assert ok
        assert pinit[3] == 0.0
        assert abs(p[3]) < 1e-9
        assert abs(np.angle(np.exp(1j * (p[4] - phi0)))) < 1e-9
        assert abs(p[5] - np.arctan2(1.0, cot)) < 1e-9
        assert np.allclose(p[:3], h[6:9], atol=1e-9)
    # a stiff helix: q/pT = 2e-6 /GeV, starting at the origin towards phi0, crossing the cylinders
    cB = 0.299792458e-2 * g.bz
    k, phi0, cot = 2e-6, 0.7, 0.3
    om = -cB * k                     # signed curvature in 1/cm (the oracle's convention)
    pts = []
    for R in r:
        # on a circle through the origin the chord to the point at radius R is R itself and runs
        # at half the turning angle, arcsin(R om / 2), from the start direction
        half = np.arcsin(R * om / 2.0)
        pts.append((R * np.cos(phi0 + half), R * np.sin(phi0 + half), 2.0 * half / om * cot))
    h = np.asarray(pts).ravel()
    ax, ay, bx, by = h[3] - h[0], h[4] - h[1], h[6] - h[0], h[7] - h[1]
    assert 1e-12 < abs(ax * by - ay * bx) / (bx * bx + by * by) < 1e-7
    ok, p, c, pinit = o.seed(h, v, [0, 1, 2])
    assert ok and abs(pinit[3] / k - 1) < 1e-6 and abs(p[3] / k - 1) < 1e-3


@pytest.fixture(scope="module")
def smeared_fit():
    g = S.geometry_barrel()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 6000, 11, 0, eta_max=1.0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    layers, hits, p0, c0, truth_last, nh, sel = S.fit_workload(ev)
    r = o.fit_batch(layers, hits, ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64), p0, c0)
    return r, truth_last, layers, hits, p0, c0, ev, o


def test_fit_pulls_are_unit_normal(smeared_fit):
    r, truth, *_ = smeared_fit
    ok = r["status"] == 0
    P, Cm, T = r["p"][ok], r["c"][ok], truth[ok]
    d = P - T
    d[:, 4] = np.angle(np.exp(1j * d[:, 4]))
    phi = np.arctan2(P[:, 1], P[:, 0])
    t = np.stack([-np.sin(phi), np.cos(phi)], -1)
    var_t = t[:, 0] ** 2 * Cm[:, 0] + 2 * t[:, 0] * t[:, 1] * Cm[:, 1] + t[:, 1] ** 2 * Cm[:, 2]
    pulls = {"rphi": (d[:, :2] * t).sum(1) / np.sqrt(var_t),
             "z": d[:, 2] / np.sqrt(Cm[:, 5]), "k": d[:, 3] / np.sqrt(Cm[:, 9]),
             "phi": d[:, 4] / np.sqrt(Cm[:, 14]), "theta": d[:, 5] / np.sqrt(Cm[:, 20])}
    for name, pl in pulls.items():
        assert abs(pl.mean()) < 0.05, name
        assert abs(pl.std() - 1.0) < 0.04, (name, pl.std())


def test_predicted_chi2_is_chi2_with_3_dof(smeared_fit):
    r, truth, layers, hits, p0, c0, ev, o = smeared_fit
    # per-hit predicted chi2: refit track by track on a subsample, recording each step
    xyz = ev.hit_xyz.astype(np.float64)
    cov = ev.hit_cov.astype(np.float64)
    vals = []
    for i in range(800):
        p, c = p0[i], c0[i]
        for j in range(layers.shape[1]):
            if layers[i, j] < 0:
                break
            rc, pp, cc, _ = o.propagate(layers[i, j], p, c)
            assert rc == 1
            ok, p, c, x2 = o.update(pp, cc, xyz[hits[i, j]], cov[hits[i, j]])
            vals.append(x2)
    vals = np.array(vals)
    n = vals.size
    assert abs(vals.mean() - 3.0) < 3 * np.sqrt(6.0 / n)
    assert stats.kstest(vals, stats.chi2(3).cdf).pvalue > 0.01
    # and the total over all tracks
    ok = r["status"] == 0
    mean = r["chi2"][ok].sum() / r["nupd"][ok].sum()
    assert abs(mean - 3.0) < 3 * np.sqrt(6.0 / r["nupd"][ok].sum()) + 0.02


def test_covariances_are_psd_with_the_surface_normal_as_null_direction(smeared_fit):
    """A state on a layer surface has no spread along the surface normal (the crossing is
    constrained to the surface), so C is positive semi-definite of rank 5; C_pos + V is SPD."""
    r, *_ = smeared_fit
    for p, c in zip(r["p"][:2000], r["c"][:2000]):
        M = sym(c)
        w = np.linalg.eigvalsh(M)
        assert w[0] > -1e-12 * w[-1]
        assert w[1] > 1e-9 * w[-1] or w[1] > 1e-14
        n = np.array([p[0], p[1], 0.0]) / np.hypot(p[0], p[1])
        assert n @ M[:3, :3] @ n < 1e-6 * np.trace(M[:3, :3])
        assert np.all(np.linalg.eigvalsh(M[:3, :3] + np.diag([9e-6, 9e-6, 1e-4])) > 0)


def test_update_is_accurate_when_the_innovation_covariance_is_ill_conditioned(orc):
    """A prior spread of 10 cm along one surface direction against a 30 um hit gives cond(S) ~ 1e7.
    The oracle's update must match a 50-digit evaluation of the same posterior."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(21)
    for _ in range(5):
        u = rng.standard_normal(3); u[2] = 0.3 * u[2]; u /= np.linalg.norm(u)
        sig = np.array([100.0, 0.05, 1e-2, 1e-3, 3e-3, 1e-3])
        A = rng.standard_normal((6, 6)) * 0.3 + np.eye(6)
        C = A @ np.diag(sig ** 2) @ A.T
        C[:3, :3] += 150.0 * np.outer(u, u)
        V = np.diag([9e-6, 9e-6, 1e-4])
        p = np.array([60.0, 80.0, 100.0, -1.5, -2.5, 1.0])
        m = p[:3] + 0.003
        ok, po, co, x2 = orc.update(p, C[np.tril_indices(6)], m, V[np.tril_indices(3)], joseph=True)
        assert ok
        Cm, Vm = mp.matrix(C.tolist()), mp.matrix(V.tolist())
        H = mp.matrix(np.hstack([np.eye(3), np.zeros((3, 3))]).tolist())
        S = H * Cm * H.T + Vm
        K = Cm * H.T * mp.inverse(S)
        Cx = Cm - K * S * K.T
        ref = np.array([[float(Cx[i, j]) for j in range(6)] for i in range(6)])
        got = sym(co)
        scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
        assert np.all(np.abs(got - ref) <= 1e-7 * scale + 1e-20)
        kk = np.linalg.cond(S.tolist() and np.array([[float(S[i, j]) for j in range(3)] for i in range(3)]))
        assert kk > 1e6
