"""Module planes and overlap hits on the GPU (Sec. 3.1 module position and normal: the Phase-2
tilted barrel; Sec. 2.2: a single additional detector-overlap hit) against the oracle, on the same
inputs: the Phase-2-like tracker with cylinders 3-5 built from flat and tilted modules, and the
same with the 4th-6th disk of each endcap built from planar modules.

Search: hit lists and overlap hits bit-exact up to the first near-tie step the oracle flags;
parameters, covariance and chi2 within the forward search's tolerances (oracle/parity.py).  Fit
over the true assignment: the fit's tolerances."""
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


@pytest.fixture(scope="module", params=["barrel_modules", "barrel_and_disk_modules"])
def work(request):
    g = S.geometry_phase2_modular() if request.param == "barrel_modules" else S.geometry_phase2_modular_disks()
    evs = [S.simulate_event(g, 1501, 41, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=4000)
           for e in range(3)]
    return g, S.concat_events(evs, g.n_layers)


def _ctx(g, batch, params):
    ctx = pipeline.make_context(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov, hit_module=batch.hit_mod)
    return ctx


def _oracle(g, batch, params):
    orc = oracle.Oracle(g, params)
    orc.set_modules(g.modules.c, g.modules.n, batch.hit_mod)
    return orc


def _check_ovl(out, o):
    """Overlap hits equal up to each seed's first near-tie step (the whole row without a tie)."""
    idx, mp = o["seed_index"], o["max_plan"]
    bad = []
    for k, si in enumerate(idx):
        t = o["tie_step"][k]
        n = mp if t < 0 else t
        if not np.array_equal(out["ovl"][si, :n], o["ovl"][k, :n]):
            bad.append(int(si))
    return bad


@pytest.mark.parametrize("precision", [0, 2])
def test_modular_search_matches_oracle(lib, work, precision):
    g, batch = work
    params = S.default_params(precision=precision)
    ctx = _ctx(g, batch, params)
    ctx.seed(batch.seed_hits)
    out = ctx.build(mkgb.alloc_tracks(batch.seed_hits.shape[0], g.max_plan, ovl=True))
    o = PR.oracle_build(_oracle(g, batch, params), batch)
    rep = PR.compare_build(out, o)
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["failed_mismatch"] == 0 and rep["count_bad"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n_tie"] < 0.05 * rep["n"], rep
    assert _check_ovl(out, o) == []
    # the modular layers are searched and overlap hits picked up
    n_ovl = int((out["ovl"] >= 0).sum())
    assert n_ovl > 0.05 * batch.seed_hits.shape[0], n_ovl
    if precision == 0:
        assert rep["worst_param"] < 0.5 and rep["worst_chi2"] < 0.5, rep


def test_modular_fit_matches_oracle(lib, work):
    g, batch = work
    params = S.default_params()
    ctx = _ctx(g, batch, params)
    fi = pipeline.fit_inputs(batch)
    n = fi.layers.shape[0]
    f = dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
             status=np.zeros(n, np.int32))
    ctx.fit(fi.layers, fi.hits, fi.p0, fi.c0, f["p"], f["c"], f["chi2"], f["status"])
    r = _oracle(g, batch, params).fit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64),
                                            batch.hit_cov.astype(np.float64), fi.p0, fi.c0)
    rep = PR.compare_fit(f, r)
    assert rep["status_bad"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n"] > 0.95 * n
    # the fit's work counters: crossed layers and updates as the oracle counts them
    cg = ctx.counters(1)
    assert cg[0] == r["counters"][0] and cg[2] == r["counters"][2]


def test_modular_fit_outlier_and_fp64(lib, work):
    """FP64 fit of modular tracks, and the outlier rule on module hits (a planted wrong hit on a
    module is rejected on its plane)."""
    g, batch = work
    fi0 = pipeline.fit_inputs(batch)
    bad, swaps = pipeline.plant_wrong_hits(batch, fi0, 0.3, 5)
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    for params, fi in ((S.default_params(precision=2), fi0),
                       (S.default_params(fit_outlier_chi2=30.0),
                        pipeline.FitInputs(fi0.layers, bad, fi0.p0, fi0.c0, fi0.event))):
        ctx = _ctx(g, batch, params)
        n = fi.layers.shape[0]
        f = dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
                 status=np.zeros(n, np.int32))
        ctx.fit(fi.layers, fi.hits, fi.p0, fi.c0, f["p"], f["c"], f["chi2"], f["status"])
        r = _oracle(g, batch, params).fit_batch(fi.layers, fi.hits, X, V, fi.p0, fi.c0)
        rep = PR.compare_fit(f, r, mask=r["near_cut"] == 0)
        assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
        assert rep["n"] > 0.9 * n


def test_modular_edge_cases(lib, work):
    g, batch = work
    params = S.default_params()
    ctx = pipeline.make_context(g, params)
    # module ids that do not fit the layers
    hm = batch.hit_mod.copy()
    i = int(np.nonzero(hm >= 0)[0][0])
    for v in (-1, int(g.modules.c.shape[0]), int(np.nonzero(g.modules.layer != g.modules.layer[hm[i]])[0][0])):
        hm2 = hm.copy()
        hm2[i] = v
        with pytest.raises(mkgb.MkgbError):
            ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov, hit_module=hm2)
    j = int(np.nonzero(hm < 0)[0][0])
    hm2 = hm.copy()
    hm2[j] = int(hm[i])
    with pytest.raises(mkgb.MkgbError):
        ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov, hit_module=hm2)
    # module tables that do not describe planes of this geometry
    from types import SimpleNamespace
    mods = g.modules
    for bad_mod in (SimpleNamespace(layer=mods.layer, c=mods.c, n=mods.n * 1.1),
                    SimpleNamespace(layer=np.full_like(mods.layer, g.n_layers), c=mods.c, n=mods.n),
                    SimpleNamespace(layer=mods.layer, c=np.where(np.arange(mods.c.shape[0])[:, None] == 3, np.nan, mods.c),
                                    n=mods.n)):
        with pytest.raises(mkgb.MkgbError):
            ctx.load_modules(bad_mod)
    ctx.load_modules(mods)
    # without modules loaded, module ids are refused
    plain = pipeline.make_context(S.geometry_phase2(), params)
    with pytest.raises(mkgb.MkgbError):
        plain.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov, hit_module=hm)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov, hit_module=hm)
    # a seed given a module hit of another track: its hits are taken on their planes as the
    # oracle takes them, and the result is the oracle's
    sh = batch.seed_hits[:6].copy()
    sh[0, 2] = i
    ctx.seed(sh)
    out = ctx.build(mkgb.alloc_tracks(6, g.max_plan, ovl=True))
    b6 = S.Batch(batch.n_events, batch.n_layers, batch.hit_xyz, batch.hit_cov, batch.hit_off, batch.hit_track,
                 sh, batch.seed_event[:6], batch.seed_track[:6], batch.events, batch.hit_mod)
    rep6 = PR.compare_build(out, PR.oracle_build(_oracle(g, batch, params), b6))
    assert len(rep6["hit_mismatch"]) == 0 and rep6["failed_mismatch"] == 0 and rep6["param_bad"] == 0, rep6
    # no overlap array requested: the search runs the same
    ctx.seed(batch.seed_hits[:200])
    a = ctx.build(mkgb.alloc_tracks(200, g.max_plan, ovl=True))
    b = ctx.build(mkgb.alloc_tracks(200, g.max_plan))
    assert np.array_equal(a["hits"], b["hits"]) and np.array_equal(a["score"], b["score"])
    # hits loaded without module ids: every hit on its layer's cylinder, no overlaps
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    ctx.seed(batch.seed_hits[:200])
    c = ctx.build(mkgb.alloc_tracks(200, g.max_plan, ovl=True))
    assert np.all(c["ovl"] == -1)


def test_modular_backward_fit_matches_oracle(lib, work):
    """The backward fit (Sec. 2.2) through the modular layers from the GPU forward fit's states:
    module hits used on their planes (the start state on its last hit's plane)."""
    g, batch = work
    params = S.default_params()
    ctx = _ctx(g, batch, params)
    fi = pipeline.fit_inputs(batch)
    n = fi.layers.shape[0]
    mk = lambda: dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
                      status=np.zeros(n, np.int32))
    f, b = mk(), mk()
    ctx.fit(fi.layers, fi.hits, fi.p0, fi.c0, f["p"], f["c"], f["chi2"], f["status"])
    ctx.fit_backward(fi.layers, fi.hits, f["p"], f["c"], b["p"], b["c"], b["chi2"], b["status"])
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    r = _oracle(g, batch, params).bkfit_batch(fi.layers, fi.hits, X, V, f["p"].astype(np.float64),
                                              f["c"].astype(np.float64), 100.0)
    ok = f["status"] == 0
    rep = PR.compare_fit(b, r, mask=ok)
    assert np.array_equal(b["status"][ok], r["status"][ok]), rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n"] > 0.95 * n


def test_modular_backward_search_matches_oracle(lib, work):
    """The backward search (Sec. 2.2) through modular layers: tracks without their first five
    layers (so that the search crosses modular layers 4 and 3 and the plain 2, 1, 0) are fitted
    forwards and backwards on the GPU, then both searches run inwards from that state; hit lists
    and overlap hits bit-exact outside near ties."""
    g, batch = work
    params = S.default_params()
    ctx = _ctx(g, batch, params)
    fi = pipeline.fit_inputs(batch)
    n_skip = 5
    keep = ((fi.layers >= 0).sum(1) >= n_skip + 3) & (fi.layers[:, 0] == 0)
    fo = pipeline.outer_fit_inputs(fi, n_skip)
    sel = np.nonzero(keep)[0]
    L, H = np.ascontiguousarray(fo.layers[sel]), np.ascontiguousarray(fo.hits[sel])
    n = len(sel)
    mk = lambda: dict(p=np.zeros((n, 6), np.float32), c=np.zeros((n, 21), np.float32), chi2=np.zeros(n, np.float32),
                      status=np.zeros(n, np.int32))
    f, b = mk(), mk()
    ctx.fit(L, H, fo.p0[sel], fo.c0[sel], f["p"], f["c"], f["chi2"], f["status"])
    ctx.fit_backward(L, H, f["p"], f["c"], b["p"], b["c"], b["chi2"], b["status"])
    ok = (f["status"] == 0) & (b["status"] == 0)
    sel, L = sel[ok], L[ok]
    ev = np.ascontiguousarray(fi.event[sel].astype(np.int32))
    first = np.ascontiguousarray(L[:, 0])
    p, c = np.ascontiguousarray(b["p"][ok]), np.ascontiguousarray(b["c"][ok])
    out = ctx.build_backward(ev, first, p, c, mkgb.alloc_tracks(len(sel), g.max_plan, ovl=True))
    o = PR.oracle_build_backward(_oracle(g, batch, params), batch, ev, p, c, first)
    rep = PR.compare_build(out, o)
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["failed_mismatch"] == 0 and rep["count_bad"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n_tie"] < 0.05 * len(sel), rep
    assert _check_ovl(out, o) == []
    assert (out["ovl"] >= 0).sum() > 0.02 * len(sel)
    # the removed inner hits, on module planes included, are found again
    found = []
    for k, i in enumerate(sel):
        lay = list(g.plans[o["region"][k]][::-1])
        steps = [lay.index(l) for l in fi.layers[i, :n_skip]]
        found.append(np.mean(out["hits"][k, steps] == fi.hits[i, :n_skip]))
    assert np.mean(found) > 0.9, np.mean(found)


def test_modular_search_full_size_sampled(lib):
    """16 modular events x 20,000 tracks + 50,000 noise hits on the device, the launch
    configuration of the benchmark; a sample of 300 seeds against the oracle."""
    import torch
    g = S.geometry_phase2_modular_disks()
    evs = [S.simulate_event(g, 20000, 0, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=50000)
           for e in range(16)]
    batch = S.concat_events(evs, g.n_layers)
    params = S.default_params()
    ctx = pipeline.make_context(g, params)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ctx.load_hits(batch.n_events, batch.hit_off, dev(batch.hit_xyz), dev(batch.hit_cov), hit_module=dev(batch.hit_mod))
    S_ = batch.seed_hits.shape[0]
    ctx.seed(dev(batch.seed_hits))
    out = mkgb.alloc_tracks(S_, g.max_plan, device="cuda", ovl=True)
    ctx.build(out)
    torch.cuda.synchronize()
    out = {k: v.cpu().numpy() for k, v in out.items()}
    rng = np.random.default_rng(17)
    idx = np.sort(rng.choice(S_, 300, replace=False))
    o = PR.oracle_build(_oracle(g, batch, params), batch, seed_index=idx)
    rep = PR.compare_build(out, o)
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert _check_ovl(out, o) == []
    assert (out["ovl"] >= 0).sum() > 0.05 * S_


def _hit_layer(batch):
    hl = np.zeros(batch.hit_xyz.shape[0], np.int64)
    for s in range(len(batch.hit_off) - 1):
        hl[batch.hit_off[s]:batch.hit_off[s + 1]] = s % batch.n_layers
    return hl


def test_modular_fit_gradient_matches_oracle_differences(lib):
    """The derivative of the fit's total chi2 (mkgb_fit_grad, reverse sweep and forward mode) with
    module hits used on their planes, at an alignment and material off nominal, against the
    oracle's FP64 central differences with the same modules (oracle/gradient.py); tolerances as
    the layers-only derivative tests (tests/test_gpu_grad.py)."""
    from oracle import gradient as OG
    g = S.add_modules(S.geometry_barrel(), [3, 4, 5])
    ev = S.simulate_event(g, 400, 5, 0, eta_max=1.0,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    batch = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(batch)
    L = g.n_layers
    rng = np.random.default_rng(3)
    align = np.zeros((L, 6))
    align[:, :3] = 20e-4 * rng.standard_normal((L, 3))
    align[:, 3:] = 5e-5 * rng.standard_normal((L, 3))
    xscale = 1.0 + 0.1 * rng.standard_normal(L)
    chi2, status, dp0, dal, dxs = OG.fd_gradient(g, S.default_params(), fi.layers, fi.hits, batch.hit_xyz,
                                                 batch.hit_cov, _hit_layer(batch), fi.p0, fi.c0, align, xscale,
                                                 hit_mod=batch.hit_mod)
    ok = status == 0
    assert ok.mean() > 0.95
    assert (batch.hit_mod[fi.hits[ok]] >= 0).any(1).mean() > 0.8   # the tracks use module hits
    used = np.unique(fi.layers[fi.layers >= 0])
    ctx = _ctx(g, batch, S.default_params())
    for mode in (0, 1):
        out = dict(chi2=np.zeros(len(ok), np.float32), dp0=np.zeros((len(ok), 6), np.float32),
                   dal=np.zeros((L, 6), np.float32), dxs=np.zeros(L, np.float32), status=np.zeros(len(ok), np.int32))
        ctx.fit_grad(fi.layers, fi.hits, fi.p0, fi.c0, align.astype(np.float32), xscale.astype(np.float32),
                     out["chi2"], out["dp0"], out["dal"], out["dxs"], out["status"], mode=mode)
        assert np.array_equal(out["status"], status), mode
        assert PR.chi2_close(out["chi2"][ok], chi2[ok])[0].all(), mode
        for got, ref, name in ((out["dal"][used], dal[used], "align"), (out["dxs"][used], dxs[used], "xscale")):
            lhs, rhs = np.abs(got - ref), 1e-2 * np.abs(ref) + 1e-3 * np.abs(ref).max()
            assert np.all(lhs <= rhs), (name, mode, float((lhs / rhs).max()))
        for k in range(6):
            r = np.abs(out["dp0"][ok, k] - dp0[ok, k]) / np.maximum(np.abs(dp0[ok, k]), 1e-3 * np.abs(dp0[ok, k]).max())
            assert np.median(r) < 1e-3 and np.percentile(r, 98) < 1e-2, (k, mode, np.median(r), np.percentile(r, 98))


def test_modular_one_call_pass_equals_separate_calls(lib, work):
    """mkgb_run_modular (load hits with module ids, seed, search, fit in one call; the fit on a
    second stream) gives bit-identical outputs to the separate calls."""
    import torch
    g, batch = work
    params = S.default_params()
    fi = pipeline.fit_inputs(batch)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    n, nt = batch.seed_hits.shape[0], fi.layers.shape[0]
    X, V, HM, SH = dev(batch.hit_xyz), dev(batch.hit_cov), dev(batch.hit_mod), dev(batch.seed_hits)
    L, H, P0, C0 = dev(fi.layers), dev(fi.hits), dev(fi.p0), dev(fi.c0)
    res = []
    for one_call in (True, False):
        ctx = pipeline.make_context(g, params)
        out = mkgb.alloc_tracks(n, g.max_plan, device="cuda", ovl=True)
        fo = [torch.zeros((nt, 6), device="cuda"), torch.zeros((nt, 21), device="cuda"), torch.zeros(nt, device="cuda"),
              torch.zeros(nt, dtype=torch.int32, device="cuda")]
        if one_call:
            ctx.run(batch.n_events, batch.hit_off, X, V, SH, out, L, H, P0, C0, *fo, hit_module=HM)
        else:
            ctx.load_hits(batch.n_events, batch.hit_off, X, V, hit_module=HM)
            ctx.fit(L, H, P0, C0, *fo)
            ctx.seed(SH)
            ctx.build(out)
        torch.cuda.synchronize()
        res.append(({k: v.cpu().numpy() for k, v in out.items()}, [f.cpu().numpy() for f in fo]))
    (a, fa), (b, fb) = res
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    for x, y in zip(fa, fb):
        assert np.array_equal(x, y)
    assert (a["ovl"] >= 0).sum() > 0


def test_seeds_on_modular_layers_match_oracle(lib):
    """Seeding layers built from modules (cylinders 0-2 of flat and tilted modules): every seed hit
    is taken on its module's plane in the seed fit (Sec. 3.1), on the GPU as in the oracle; seed
    states and the search from them against the oracle."""
    g = S.geometry_phase2_modular(layers=(0, 1, 2))
    evs = [S.simulate_event(g, 800, 43, e, pt_sampler=S.sample_pt_phase2, eta_max=2.5, noise_total=2000)
           for e in range(2)]
    batch = S.concat_events(evs, g.n_layers)
    params = S.default_params()
    assert (batch.hit_mod[batch.seed_hits] >= 0).any(1).mean() > 0.5   # most seeds carry module hits
    ctx = _ctx(g, batch, params)
    n = batch.seed_hits.shape[0]
    state, cov, info = np.zeros((n, 6), np.float32), np.zeros((n, 21), np.float32), np.zeros((n, 3), np.int32)
    ctx.seed(batch.seed_hits, state, cov, info)
    orc = _oracle(g, batch, params)
    lo = batch.hit_off
    sl = np.concatenate([oracle.hit_layers(lo[e * g.n_layers:(e + 1) * g.n_layers + 1],
                                           batch.seed_hits[batch.seed_event == e]) for e in range(batch.n_events)])
    r = orc.seed_batch(batch.seed_hits, sl, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64))
    assert np.array_equal(info[:, 2], r["status"]) and np.array_equal(info[:, 0], r["region"])
    ok = r["status"] == 0
    assert ok.mean() > 0.95
    pok, prat = PR.param_close(state[ok], r["p"][ok])
    cok, crat = PR.cov_close_surface(cov[ok], r["c"][ok], r["p"][ok], r["surf"])
    assert pok.all() and cok.all(), (prat.max(), crat.max())
    out = ctx.build(mkgb.alloc_tracks(n, g.max_plan, ovl=True))
    rep = PR.compare_build(out, PR.oracle_build(orc, batch))
    assert len(rep["hit_mismatch"]) == 0 and rep["failed_mismatch"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
