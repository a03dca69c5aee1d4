"""Pins of the oracle's combinatorial search (Sec. 2.2 forward search): the eta-phi bins
never change results (binned == brute force), the beam with N >= number of paths finds
the exact best path of an exhaustive enumeration, and isolated tracks recover their hits."""
import numpy as np
import pytest

import oracle
from paper_2312_11728_gb300 import synth as S


def _event_arrays(ev):
    return ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64)


def test_binned_equals_brute_force_barrel():
    g, ev = S.workload_small_barrel()
    o = oracle.Oracle(g)
    x, c = _event_arrays(ev)
    sl = oracle.hit_layers(ev.layer_off, ev.seed_hits)
    a = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl, binned=True)
    b = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl, binned=False)
    for k in ("params", "cov", "score", "chi2", "nfound", "nholes", "hits", "tie_step"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["counters"][:3], b["counters"][:3])
    assert b["counters"][3] > 10 * a["counters"][3]   # the bins do prune


def test_binned_equals_brute_force_phase2_endcaps():
    g = S.geometry_phase2()
    ev = S.simulate_event(g, 600, 3, 0, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=3000)
    o = oracle.Oracle(g)
    x, c = _event_arrays(ev)
    sl = oracle.hit_layers(ev.layer_off, ev.seed_hits)
    a = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl, binned=True)
    b = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl, binned=False)
    for k in ("params", "score", "hits", "nfound"):
        assert np.array_equal(a[k], b[k]), k
    assert {0, 1, 2} <= set(np.unique(a["region"]).tolist())
    assert (a["region"] < 0).mean() < 0.01


def test_isolated_tracks_recover_all_their_hits():
    """No noise: with a hit bonus large enough that any accepted hit beats a hole, every
    true hit is found; with the default score (B=4, P=8) a hit with chi2 above ~12 may lose
    to a hole, but nothing foreign is ever picked up."""
    g = S.geometry_barrel()
    ev = S.simulate_event(g, 40, 8, 0, eta_max=1.0, noise_per_layer=0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    x, c = _event_arrays(ev)
    sl = oracle.hit_layers(ev.layer_off, ev.seed_hits)
    for bonus, complete in ((100.0, True), (4.0, False)):
        o = oracle.Oracle(g, dict(score_hit=bonus))
        r = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl)
        n_true = n_got = 0
        for i, tr in enumerate(ev.seed_track):
            true = set(ev.track_hits[tr][ev.track_hits[tr] >= 0][3:].tolist())
            got = set(r["hits"][i][r["hits"][i] >= 0].tolist())
            assert got <= true
            if complete:
                assert got == true and r["nholes"][i] == 0
            n_true += len(true)
            n_got += len(got)
        assert n_got / n_true > 0.95


def test_build_efficiency_and_purity_config_small_barrel():
    g, ev = S.workload_small_barrel()
    o = oracle.Oracle(g)
    x, c = _event_arrays(ev)
    sl = oracle.hit_layers(ev.layer_off, ev.seed_hits)
    r = o.build_event(ev.layer_off, x, c, ev.seed_hits, sl)
    good = tot = true_n = 0
    for i, tr in enumerate(ev.seed_track):
        h = r["hits"][i][r["hits"][i] >= 0]
        tot += h.size
        good += int((ev.hit_track[h] == tr).sum())
        true_n += int((ev.track_layers[tr] >= 0).sum()) - 3
    assert good / tot > 0.995
    assert good / true_n > 0.98
    assert (r["tie_step"] >= 0).mean() < 0.02


# ---------------------------------------------------------------- exhaustive enumeration

def _tiny_event(seed, n_tracks=3, n_clones=2, offset=(0.004, 0.012)):
    """Barrel event whose layers hold each true hit plus displaced copies of it, so that
    windows contain several compatible hits and the search has to branch."""
    g = S.geometry_barrel(n_layers=6)
    ev = S.simulate_event(g, n_tracks, seed, 0, eta_max=0.8, noise_per_layer=0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 0.8, 5.0))
    rng = np.random.default_rng(seed + 100)
    xyz, cov, lay_off = [], [], [0]
    remap = {}
    for L in range(g.n_layers):
        a, b = ev.layer_off[L], ev.layer_off[L + 1]
        for h in range(a, b):
            remap[h] = len(xyz)
            xyz.append(ev.hit_xyz[h].astype(np.float64))
            cov.append(ev.hit_cov[h].astype(np.float64))
            if L >= 3:
                for _ in range(n_clones):
                    d = rng.uniform(*offset) * rng.choice([-1, 1], 3) * np.array([1, 1, 2])
                    xyz.append(ev.hit_xyz[h].astype(np.float64) + d)
                    cov.append(ev.hit_cov[h].astype(np.float64))
        lay_off.append(len(xyz))
    seeds = np.array([[remap[h] for h in s] for s in ev.seed_hits], np.int32)
    return g, np.array(xyz), np.array(cov), np.array(lay_off, np.int64), seeds


def _enumerate(o, g, xyz, cov, lay_off, seed3, layers3, P):
    h = xyz[seed3].ravel()
    v = cov[seed3].ravel()
    ok, p, c, _ = o.seed(h, v, layers3)
    assert ok
    plan = g.plans[0]
    start = plan.index(int(layers3[2])) + 1
    paths = [(0.0, 0, False, p, c, [])]
    widest = 1
    for t in range(start, len(plan)):
        L = plan[t]
        new = []
        for sc, nh, stopped, p, c, hist in paths:
            if stopped:
                new.append((sc, nh, True, p, c, hist + [oracle.STOP]))
                continue
            rc, pp, cc, _ = o.propagate(L, p, c)
            if rc < 0:
                continue
            if rc == 0:
                new.append((sc, nh, False, p, c, hist + [oracle.SKIP]))
                continue
            w = o.window(L, pp, cc)
            for hid in range(lay_off[L], lay_off[L + 1]):
                m = xyz[hid]
                eta = np.arcsinh(m[2] / np.hypot(m[0], m[1]))
                phi = np.arctan2(m[1], m[0])
                dphi = abs(np.angle(np.exp(1j * (phi - w[1]))))
                if abs(eta - w[0]) <= w[2] and dphi <= w[3]:
                    okc, x2 = o.chi2(pp, cc, m, cov[hid])
                    if okc and x2 < P["chi2_cut"]:
                        oku, pu, cu, _ = o.update(pp, cc, m, cov[hid])
                        if oku:
                            new.append((sc + P["score_hit"] - x2, nh, False, pu, cu, hist + [hid]))
            if nh < P["max_holes"]:
                new.append((sc - P["score_hole"], nh + 1, False, pp, cc, hist + [oracle.MISS]))
            else:
                new.append((sc, nh, True, pp, cc, hist + [oracle.STOP]))
        paths = new
        widest = max(widest, len(paths))
    paths.sort(key=lambda q: -q[0])
    return paths, widest, start


@pytest.mark.parametrize("seed", [1, 2, 3, 4, 5, 6])
def test_beam_with_enough_candidates_finds_the_exhaustive_best(seed):
    g, xyz, cov, lay_off, seeds = _tiny_event(seed)
    P = S.default_params(max_cands=64, chi2_cut=60.0, max_holes=1, deta_min=0.01, dphi_min=0.01)
    o = oracle.Oracle(g, P)
    sl = oracle.hit_layers(lay_off, seeds)
    r = o.build_event(lay_off, xyz, cov, seeds, sl, binned=True)
    checked = 0
    for i in range(seeds.shape[0]):
        paths, widest, start = _enumerate(o, g, xyz, cov, lay_off, seeds[i], sl[i], o.params)
        if widest > 64:
            continue
        best = paths[0]
        if len(paths) > 1:
            assert paths[0][0] - paths[1][0] > 1e-9       # no exact tie in these events
        assert abs(r["score"][i] - best[0]) < 1e-9
        assert list(r["hits"][i][start:len(g.plans[0])]) == best[5]
        checked += 1
        assert widest >= 4        # the search really branched
    assert checked >= 2


def test_beam_with_one_candidate_is_greedy():
    """N = 1 keeps only the best child at every layer: compare with a greedy walk."""
    g, xyz, cov, lay_off, seeds = _tiny_event(9)
    P = S.default_params(max_cands=1, chi2_cut=60.0, max_holes=1, deta_min=0.01, dphi_min=0.01)
    o = oracle.Oracle(g, P)
    sl = oracle.hit_layers(lay_off, seeds)
    r = o.build_event(lay_off, xyz, cov, seeds, sl, binned=False)
    for i in range(seeds.shape[0]):
        ok, p, c, _ = o.seed(xyz[seeds[i]].ravel(), cov[seeds[i]].ravel(), sl[i])
        plan = g.plans[0]
        start = plan.index(int(sl[i][2])) + 1
        sc, nh, hist = 0.0, 0, []
        stopped = False
        for t in range(start, len(plan)):
            L = plan[t]
            if stopped:
                hist.append(oracle.STOP)
                continue
            rc, pp, cc, _ = o.propagate(L, p, c)
            if rc == 0:
                hist.append(oracle.SKIP)
                continue
            w = o.window(L, pp, cc)
            best = None
            for hid in range(lay_off[L], lay_off[L + 1]):
                m = xyz[hid]
                eta = np.arcsinh(m[2] / np.hypot(m[0], m[1]))
                dphi = abs(np.angle(np.exp(1j * (np.arctan2(m[1], m[0]) - w[1]))))
                if abs(eta - w[0]) <= w[2] and dphi <= w[3]:
                    _, x2 = o.chi2(pp, cc, m, cov[hid])
                    if x2 < P["chi2_cut"] and (best is None or x2 < best[0]):
                        best = (x2, hid)
            miss_score = sc - P["score_hole"] if nh < P["max_holes"] else sc
            if best is not None and sc + P["score_hit"] - best[0] >= miss_score:
                _, p, c, _ = o.update(pp, cc, xyz[best[1]], cov[best[1]])
                sc += P["score_hit"] - best[0]
                hist.append(best[1])
            elif nh < P["max_holes"]:
                p, c, sc, nh = pp, cc, sc - P["score_hole"], nh + 1
                hist.append(oracle.MISS)
            else:
                p, c, stopped = pp, cc, True
                hist.append(oracle.STOP)
        assert abs(r["score"][i] - sc) < 1e-9
        assert list(r["hits"][i][start:len(plan)]) == hist


def test_window_widths_match_monte_carlo_spread_of_eta_phi():
    """With n_sigma = 1 and no clamping, the half-widths are the standard deviations of eta and
    phi of a point distributed as N(predicted position, C_pos + V_layer)."""
    g = S.geometry_phase2()
    o = oracle.Oracle(g, dict(win_nsigma=1.0, deta_min=0.0, dphi_min=0.0, deta_max=10.0, dphi_max=10.0))
    rng = np.random.default_rng(12)
    for lay, p in ((4, [30.0, 35.0, 20.0, 0.5, 0.9, 1.0]), (15, [40.0, -20.0, 180.0, -1.0, -0.4, 0.3])):
        p = np.array(p)
        if g.kind[lay] == S.BARREL:
            p[:2] *= g.pos[lay] / np.hypot(p[0], p[1])
        else:
            p[2] = g.pos[lay]
        A = rng.standard_normal((6, 6)) * np.array([0.02, 0.03, 0.05, 0.01, 0.001, 0.001])
        C6 = A @ A.T
        c21 = C6[np.tril_indices(6)]
        w = o.window(lay, p, c21)
        phi_p = np.arctan2(p[1], p[0])
        cph, sph = np.cos(phi_p), np.sin(phi_p)
        R = np.array([[cph, -sph, 0], [sph, cph, 0], [0, 0, 1]])
        V = R @ np.diag(g.sig[lay] ** 2) @ R.T
        X = rng.multivariate_normal(p[:3], C6[:3, :3] + V, 400000)
        eta = np.arcsinh(X[:, 2] / np.hypot(X[:, 0], X[:, 1]))
        phi = np.arctan2(X[:, 1], X[:, 0])
        assert abs(w[0] - np.arcsinh(p[2] / np.hypot(p[0], p[1]))) < 1e-12
        assert abs(w[2] / eta.std() - 1.0) < 0.01
        assert abs(w[3] / np.angle(np.exp(1j * (phi - phi_p))).std() - 1.0) < 0.01
