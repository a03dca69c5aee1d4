"""CUDA path vs the FP64 oracle, element by element on the same seeded inputs, through the C ABI.

Tolerances: parameters 1e-4 relative (floors 1 cm / 1 rad and 0.01 c/GeV for q/pT), covariance
1e-3 * sqrt(C_ii C_jj), chi2 1e-3 * max(1, chi2); selected hit indices bit-exact up to the first
near-tie step the oracle flags (see oracle/parity.py)."""
import numpy as np
import pytest

import oracle
from oracle import parity as PR
from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu


def _report(name, rep):
    """Writes a comparison report to $MKGB_REPORT_DIR (if set) for offline diagnosis."""
    import json
    import os
    d = os.environ.get("MKGB_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, f"{name}.json"), "w") as f:
            json.dump(rep, f, default=lambda o: o.tolist() if hasattr(o, "tolist") else str(o), indent=1)
    return rep


@pytest.fixture(scope="session")
def lib():
    B.build()
    return mkgb.load_library()


def _ctx(geom, params):
    return pipeline.make_context(geom, params)


def _sym_rand_cov(rng, n, scales):
    A = rng.standard_normal((n, 6, 6)) * np.asarray(scales)[None, :, None]
    M = A @ A.transpose(0, 2, 1) / 6.0
    return M[:, np.tril_indices(6)[0], np.tril_indices(6)[1]]


# ------------------------------------------------------------------ single steps

def test_step_propagation_matches_oracle(lib):
    g = S.geometry_phase2()
    params = S.default_params()
    ctx = _ctx(g, params)
    orc = oracle.Oracle(g, params)
    rng = np.random.default_rng(1)
    n = 4000
    r = rng.uniform(0, 30, n)
    a = rng.uniform(-np.pi, np.pi, n)
    pt = np.exp(rng.uniform(np.log(0.5), np.log(50), n))
    th = rng.uniform(0.1, np.pi - 0.1, n)
    p = np.stack([r * np.cos(a), r * np.sin(a), rng.uniform(-40, 40, n), rng.choice([-1, 1], n) / pt,
                  rng.uniform(-np.pi, np.pi, n), th], -1).astype(np.float32)
    c = _sym_rand_cov(rng, n, [0.01, 0.01, 0.02, 0.05, 0.002, 0.002]).astype(np.float32)
    layers = rng.integers(3, g.n_layers, n).astype(np.int32)
    po, co, cr = np.zeros((n, 6), np.float32), np.zeros((n, 21), np.float32), np.zeros(n, np.int32)
    ctx.propagate(layers, p, c, po, co, cr)
    n_cmp = 0
    for i in range(n):
        pi, ci = p[i].astype(np.float64), c[i].astype(np.float64)
        ok, s, margin = orc.path(int(layers[i]), pi)
        rc, pp, cc, _ = orc.propagate(int(layers[i]), pi, ci)
        if margin < 1e-4:
            continue
        assert cr[i] == rc, (i, cr[i], rc)
        if rc == 1:
            pok, _ = PR.param_close(po[i], pp)
            cok, _ = PR.cov_close_surface(co[i][None], cc[None], pp[None], orc.surfaces())
            assert pok.all(), (i, po[i], pp)
            assert cok.all(), (i, co[i], cc)
            n_cmp += 1
    assert n_cmp > 800


def test_step_update_matches_oracle(lib):
    g = S.geometry_barrel()
    params = S.default_params()
    ctx = _ctx(g, params)
    orc = oracle.Oracle(g, params)
    rng = np.random.default_rng(2)
    n = 3000
    p = np.stack([rng.uniform(-100, 100, n), rng.uniform(-100, 100, n), rng.uniform(-250, 250, n),
                  rng.uniform(-2, 2, n), rng.uniform(-np.pi, np.pi, n), rng.uniform(0.2, 2.9, n)], -1)
    c = _sym_rand_cov(rng, n, [0.005, 0.005, 0.01, 0.02, 0.001, 0.001])
    V = _sym_rand_cov(rng, n, [0.003, 0.003, 0.01, 0, 0, 0])[:, :6]
    m = p[:, :3] + rng.standard_normal((n, 3)) * 0.004
    p, c, V, m = p.astype(np.float32), c.astype(np.float32), V.astype(np.float32), m.astype(np.float32)
    po, co, x2, ok = np.zeros((n, 6), np.float32), np.zeros((n, 21), np.float32), np.zeros(n, np.float32), np.zeros(n, np.int32)
    ctx.update(p, c, m, V, po, co, x2, ok)
    for i in range(n):
        okr, pp, cc, xr = orc.update(p[i].astype(np.float64), c[i].astype(np.float64),
                                     m[i].astype(np.float64), V[i].astype(np.float64))
        assert ok[i] == int(okr)
        if okr:
            assert PR.chi2_close(x2[i], xr)[0], (i, x2[i], xr)
            assert PR.param_close(po[i], pp)[0].all(), (i, po[i], pp)
            assert PR.cov_close(co[i], cc)[0].all(), (i, co[i], cc)


# ------------------------------------------------------------------ seeds, fit, build

@pytest.fixture(scope="module")
def small_barrel():
    g, ev = S.workload_small_barrel()
    batch = S.concat_events([ev], g.n_layers)
    params = S.default_params()
    return g, batch, params


@pytest.fixture(scope="module")
def phase2_small():
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, 1501, 0, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=4000)
           for e in range(3)]
    batch = S.concat_events(evs, g.n_layers)
    return g, batch, S.default_params()


@pytest.mark.parametrize("which", ["small_barrel", "phase2_small"])
def test_seed_states_match_oracle(lib, which, request):
    g, batch, params = request.getfixturevalue(which)
    ctx = _ctx(g, params)
    res = pipeline.run_host(ctx, batch, g.max_plan)
    orc = oracle.Oracle(g, params)
    lo = batch.hit_off
    sl = np.concatenate([oracle.hit_layers(lo[e * g.n_layers:(e + 1) * g.n_layers + 1],
                                           batch.seed_hits[batch.seed_event == e]) for e in range(batch.n_events)])
    r = orc.seed_batch(batch.seed_hits, sl, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64))
    info = res["seed_info"]
    _report(f"seed_{which}", dict(region_mismatch=np.nonzero(info[:, 0] != r["region"])[0],
                                 status_mismatch=np.nonzero(info[:, 2] != r["status"])[0],
                                 worst_param=float(PR.param_close(res["seed_state"][r["status"] == 0],
                                                                  r["p"][r["status"] == 0])[1].max()),
                                 worst_cov=float(PR.cov_close_surface(res["seed_cov"][r["status"] == 0],
                                                                      r["c"][r["status"] == 0], r["p"][r["status"] == 0],
                                                                      r["surf"])[1].max())))
    assert np.array_equal(info[:, 0], r["region"])
    assert np.array_equal(info[:, 1], r["start"])
    assert np.array_equal(info[:, 2], r["status"])
    ok = r["status"] == 0
    pok, prat = PR.param_close(res["seed_state"][ok], r["p"][ok])
    cok, crat = PR.cov_close_surface(res["seed_cov"][ok], r["c"][ok], r["p"][ok], r["surf"])
    assert pok.all(), prat.max()
    assert cok.all(), crat.max()


@pytest.mark.parametrize("pt", [(60.0, 500.0), (0.5, 0.6)])
def test_seeds_all_or_none_refitted_in_fp64_match_oracle(lib, pt):
    """Stiff tracks only (pT 60-500 GeV: >90% of the seeds fit |q/pT| < 0.03 and go through the
    FP64 refit list; the rest are short forward seeds whose q/pT the three hits fix only loosely)
    and soft tracks only (0.5-0.6 GeV: the list stays empty): seed states against the oracle, as
    for the mixed workloads."""
    g = S.geometry_phase2()
    ev = S.simulate_event(g, 1500, 5, 0, pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, *pt), eta_max=3.0,
                          noise_total=1000)
    batch = S.concat_events([ev], g.n_layers)
    params = S.default_params()
    ctx = _ctx(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    n = batch.seed_hits.shape[0]
    state, cov, info = np.zeros((n, 6), np.float32), np.zeros((n, 21), np.float32), np.zeros((n, 3), np.int32)
    ctx.seed(batch.seed_hits, state, cov, info)
    r = oracle.Oracle(g, params).seed_batch(batch.seed_hits, oracle.hit_layers(batch.hit_off, batch.seed_hits),
                                            batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64))
    ok = r["status"] == 0
    refit = np.abs(r["p"][ok, 3]) < 0.03
    assert refit.mean() > 0.9 if pt[0] > 1 else not refit.any()
    assert np.array_equal(info[:, 2], r["status"])
    with np.errstate(divide="ignore"):   # failed seeds carry theta 0
        eta = -np.log(np.tan(0.5 * r["p"][:, 5]))
    far = ~(ok & (np.abs(np.abs(eta) - g.barrel_eta_max) < 1e-5))
    assert np.array_equal(info[far, 0], r["region"][far])
    pok, prat = PR.param_close(state[ok], r["p"][ok])
    cok, crat = PR.cov_close_surface(cov[ok], r["c"][ok], r["p"][ok], r["surf"])
    assert pok.all(), prat.max()
    assert cok.all(), crat.max()


@pytest.mark.parametrize("which", ["small_barrel", "phase2_small"])
def test_fit_over_known_assignment_matches_oracle(lib, which, request):
    g, batch, params = request.getfixturevalue(which)
    ctx = _ctx(g, params)
    fi = pipeline.fit_inputs(batch)
    res = pipeline.run_host(ctx, batch, g.max_plan, fi)
    orc = oracle.Oracle(g, params)
    r = orc.fit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
                      fi.p0.astype(np.float64), fi.c0.astype(np.float64))
    rep = _report(f"fit_{which}", PR.compare_fit(res["fit"], r))
    assert rep["status_bad"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["n"] > 0.95 * fi.layers.shape[0]
    c = res["fit"]["counters"]
    assert c[0] == r["counters"][0] and c[2] == r["counters"][2]


@pytest.mark.parametrize("which", ["small_barrel", "phase2_small"])
def test_build_matches_oracle(lib, which, request):
    g, batch, params = request.getfixturevalue(which)
    ctx = _ctx(g, params)
    res = pipeline.run_host(ctx, batch, g.max_plan)
    orc = oracle.Oracle(g, params)
    o = PR.oracle_build(orc, batch)
    rep = _report(f"build_{which}", PR.compare_build(res["build"], o))
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["failed_mismatch"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0 and rep["count_bad"] == 0, rep
    assert rep["n_tie"] < 0.03 * rep["n"], rep
    # work counters agree up to the near-tie seeds
    gc, oc = res["build_counters"], o["counters"]
    for k in range(3):
        assert abs(gc[k] - oc[k]) <= 0.02 * oc[k] + 10, (k, gc, oc)


def test_all_fp64_path_matches_oracle(lib, phase2_small):
    """The plain comparison path (precision MKGB_FP64: every Kalman step of the search and the fit
    in FP64) against the oracle with the same tolerances as the FP32 path."""
    g, batch, params = phase2_small
    p64 = dict(params, precision=2)
    ctx = _ctx(g, p64)
    fi = pipeline.fit_inputs(batch)
    res = pipeline.run_host(ctx, batch, g.max_plan, fi)
    orc = oracle.Oracle(g, p64)
    o = PR.oracle_build(orc, batch)
    rep = _report("build_fp64_phase2_small", PR.compare_build(res["build"], o))
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["failed_mismatch"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0 and rep["count_bad"] == 0, rep
    r = orc.fit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
                      fi.p0.astype(np.float64), fi.c0.astype(np.float64))
    rf = _report("fit_fp64_phase2_small", PR.compare_fit(res["fit"], r))
    assert rf["status_bad"] == 0 and rf["param_bad"] == 0 and rf["cov_bad"] == 0 and rf["chi2_bad"] == 0, rf
    # FP64 sits far inside the tolerances that FP32 uses
    assert rep["worst_param"] < 0.05 and rf["worst_param"] < 0.05, (rep["worst_param"], rf["worst_param"])


def test_device_and_host_paths_agree_and_are_deterministic(lib, phase2_small):
    import torch
    g, batch, params = phase2_small
    ctx = _ctx(g, params)
    fi = pipeline.fit_inputs(batch)
    host = pipeline.run_host(ctx, batch, g.max_plan, fi)
    db = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    outs = []
    for _ in range(2):
        pipeline.run_step(ctx, db)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy().copy() for k, v in db.out.items()})
    for k in outs[0]:
        assert np.array_equal(outs[0][k], outs[1][k]), k
        assert np.array_equal(outs[0][k], host["build"][k]), k
    assert np.array_equal(db.fit["p"].cpu().numpy(), host["fit"]["p"])


def test_search_fp64_redo_of_ill_conditioned_updates(lib, phase2_small):
    """With a low condition threshold many search updates are redone in FP64 (k_rescue): the
    results still match the oracle, and they differ from the run without the redo."""
    g, batch, params = phase2_small
    outs = {}
    for kappa in (1e3, 0.0):
        p = dict(params, kappa_fp64=kappa)
        res = pipeline.run_host(_ctx(g, p), batch, g.max_plan)
        outs[kappa] = res["build"]
        if kappa > 0:
            o = PR.oracle_build(oracle.Oracle(g, p), batch)
            rep = _report("build_redo_phase2_small", PR.compare_build(res["build"], o))
            assert len(rep["hit_mismatch"]) == 0 and rep["failed_mismatch"] == 0, rep
            assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    changed = np.any(outs[1e3]["cov"] != outs[0.0]["cov"], axis=1)
    assert changed.sum() > 10


def test_one_call_run_matches_separate_calls(lib, phase2_small):
    """mkgb_run (the fit on a second stream inside the call) gives the separate calls' results
    bit for bit, twice in a row."""
    import torch
    g, batch, params = phase2_small
    fi = pipeline.fit_inputs(batch)
    ref_ctx = _ctx(g, params)
    ref = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    pipeline.run_step(ref_ctx, ref)
    torch.cuda.synchronize()
    ctx = _ctx(g, params)
    db = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    for _ in range(2):
        pipeline.run_step_fused(ctx, db)
        torch.cuda.synchronize()
        for k in ref.out:
            assert torch.equal(ref.out[k], db.out[k]), k
        for k in ("p", "c", "chi2", "status"):
            assert torch.equal(ref.fit[k], db.fit[k]), k


def _host_run(ctx, batch, fi, max_plan, pinned):
    import torch
    from paper_2312_11728_gb300 import mkgb as M
    n, T = batch.seed_hits.shape[0], fi.layers.shape[0]
    if pinned:
        h = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        out = {k: torch.from_numpy(v).pin_memory() for k, v in M.alloc_tracks(n, max_plan).items()}
        fo = [torch.zeros((T, 6)).pin_memory(), torch.zeros((T, 21)).pin_memory(), torch.zeros(T).pin_memory(),
              torch.zeros(T, dtype=torch.int32).pin_memory()]
    else:
        h = lambda a: np.ascontiguousarray(a)
        out = M.alloc_tracks(n, max_plan)
        fo = [np.zeros((T, 6), np.float32), np.zeros((T, 21), np.float32), np.zeros(T, np.float32),
              np.zeros(T, np.int32)]
    ctx.run_host(batch.n_events, batch.hit_off, h(batch.hit_xyz), h(batch.hit_cov), h(batch.seed_hits), out,
                 h(fi.layers), h(fi.hits), h(fi.p0), h(fi.c0), *fo)
    cv = lambda a: a.numpy() if hasattr(a, "numpy") else a
    return {k: cv(v) for k, v in out.items()}, [cv(a) for a in fo]


@pytest.mark.parametrize("n_events", [1, 3, 11])
def test_host_array_run_matches_device_run(lib, n_events):
    """mkgb_run_host (host arrays; the hits copied in chunks of events and prepared per chunk, the
    copies overlapping the kernels) gives mkgb_run's results bit for bit, with page-locked and
    with pageable host arrays, twice in a row; 11 events make uneven chunks."""
    import torch
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, 300 + 97 * e, 5, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=1500)
           for e in range(n_events)]
    batch = S.concat_events(evs, g.n_layers)
    params = S.default_params()
    fi = pipeline.fit_inputs(batch)
    ref_ctx = _ctx(g, params)
    ref = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    pipeline.run_step_fused(ref_ctx, ref)
    torch.cuda.synchronize()
    ctx = _ctx(g, params)
    for pinned in (True, False, True):
        out, fo = _host_run(ctx, batch, fi, g.max_plan, pinned)
        for k in ref.out:
            assert np.array_equal(ref.out[k].cpu().numpy(), out[k]), (k, pinned)
        for k, a in zip(("p", "c", "chi2", "status"), fo):
            assert np.array_equal(ref.fit[k].cpu().numpy(), a), (k, pinned)
    with pytest.raises(mkgb.MkgbError):   # device tensors are refused
        ctx.run_host(batch.n_events, batch.hit_off, ref.xyz, ref.cov, ref.seeds, ref.out, ref.fit["layers"],
                     ref.fit["hits"], ref.fit["p0"], ref.fit["c0"], ref.fit["p"], ref.fit["c"], ref.fit["chi2"])


# ------------------------------------------------------------------ edge cases

def test_edge_cases_empty_single_and_ragged(lib):
    g = S.geometry_barrel()
    params = S.default_params()
    ctx = _ctx(g, params)
    ev = S.simulate_event(g, 5, 4, 0, eta_max=1.0, noise_per_layer=0)
    batch = S.concat_events([ev], g.n_layers)
    # zero seeds
    ctx.load_hits(1, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    ctx.seed(np.zeros((0, 3), np.int32))
    out = ctx.build(mkgb.alloc_tracks(0, g.max_plan))
    assert out["hits"].shape == (0, g.max_plan)
    # one seed, and an invalid one (index out of range -> status 1, score -inf)
    sh = np.concatenate([batch.seed_hits[:1], np.array([[0, 1, 10 ** 6]], np.int32)])
    info = np.zeros((2, 3), np.int32)
    ctx.seed(sh, np.zeros((2, 6), np.float32), np.zeros((2, 21), np.float32), info)
    out = ctx.build(mkgb.alloc_tracks(2, g.max_plan))
    assert info[0, 2] == 0 and info[1, 2] == 1
    assert np.isfinite(out["score"][0]) and out["score"][1] == -np.inf
    assert np.all(out["hits"][1] == mkgb.HIT_PRE)
    # empty layers: an event with hits on only the first three layers
    keep = batch.hit_off[3]
    off = np.concatenate([batch.hit_off[:4], np.full(g.n_layers - 3, keep)]).astype(np.int64)
    ctx.load_hits(1, off, batch.hit_xyz[:keep], batch.hit_cov[:keep])
    ctx.seed(batch.seed_hits)
    out = ctx.build(mkgb.alloc_tracks(batch.seed_hits.shape[0], g.max_plan))
    assert np.all(out["hits"][:, 3:] < 0)
    # bad arguments are errors, not faults
    with pytest.raises(mkgb.MkgbError):
        ctx.build(mkgb.alloc_tracks(batch.seed_hits.shape[0], 3))
    with pytest.raises(mkgb.MkgbError):
        ctx.set_params(dict(params, max_cands=9))
    with pytest.raises(mkgb.MkgbError):
        ctx.load_hits(1, np.array([0, 5, 3] + [3] * (g.n_layers - 2), np.int64), batch.hit_xyz, batch.hit_cov)


@pytest.mark.parametrize("n_cands", [1, 8])
def test_candidate_limits_match_oracle(lib, small_barrel, n_cands):
    g, batch, params = small_barrel
    params = dict(params, max_cands=n_cands)
    ctx = _ctx(g, params)
    res = pipeline.run_host(ctx, batch, g.max_plan)
    o = PR.oracle_build(oracle.Oracle(g, params), batch)
    rep = PR.compare_build(res["build"], o)
    assert len(rep["hit_mismatch"]) == 0 and rep["param_bad"] == 0 and rep["chi2_bad"] == 0, rep


# ------------------------------------------------------------------ full-size workload, sampled

@pytest.fixture(scope="module")
def phase2_full():
    g, evs = S.workload_phase2()
    return g, S.concat_events(evs, g.n_layers), S.default_params()


def test_full_size_phase2_sampled_against_oracle(lib, phase2_full):
    """64 events x 20,000 tracks, in the launch configuration the benchmark times; the oracle
    recomputes a random sample of seeds (searches are independent per seed)."""
    import torch
    g, batch, params = phase2_full
    ctx = _ctx(g, params)
    fi = pipeline.fit_inputs(batch)
    db = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    pipeline.run_step(ctx, db)
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in db.out.items()}
    rng = np.random.default_rng(7)
    sample = np.sort(rng.choice(batch.seed_hits.shape[0], 400, replace=False))
    orc = oracle.Oracle(g, params)
    o = PR.oracle_build(orc, batch, sample)
    rep = _report("build_full_size", PR.compare_build(gpu, o))
    assert len(rep["hit_mismatch"]) == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    tsample = np.sort(rng.choice(fi.layers.shape[0], 2000, replace=False))
    r = orc.fit_batch(fi.layers[tsample], fi.hits[tsample], batch.hit_xyz.astype(np.float64),
                      batch.hit_cov.astype(np.float64), fi.p0[tsample].astype(np.float64),
                      fi.c0[tsample].astype(np.float64))
    gf = {k: db.fit[k].cpu().numpy()[tsample] for k in ("p", "c", "chi2", "status")}
    rep = _report("fit_full_size", PR.compare_fit(gf, r))
    assert rep["status_bad"] == 0 and rep["param_bad"] == 0 and rep["chi2_bad"] == 0, rep
    assert rep["cov_bad"] == 0, rep


def test_full_size_seeds_against_oracle(lib, phase2_full):
    """Every one of the 1.28M seeds of the 64-event batch (FP32 trajectory and Jacobian, FP64
    covariance transport and update) against the oracle's FP64 seed fit: region, start step and
    status equal, parameters and covariance within the tolerances."""
    g, batch, params = phase2_full
    ctx = _ctx(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    n = batch.seed_hits.shape[0]
    state, cov, info = np.zeros((n, 6), np.float32), np.zeros((n, 21), np.float32), np.zeros((n, 3), np.int32)
    ctx.seed(batch.seed_hits, state, cov, info)
    L = g.n_layers
    sl = np.concatenate([oracle.hit_layers(batch.hit_off[e * L:(e + 1) * L + 1],
                                           batch.seed_hits[batch.seed_event == e]) for e in range(batch.n_events)])
    r = oracle.Oracle(g, params).seed_batch(batch.seed_hits, sl, batch.hit_xyz.astype(np.float64),
                                            batch.hit_cov.astype(np.float64))
    # the region follows from the seed's eta against the barrel's eta limit, decided in FP32 on the
    # GPU and in FP64 by the oracle: a seed whose eta lies within 1e-5 of the limit may take either
    # region (a near-tie, as for hit selection); it must take one of the two
    with np.errstate(divide="ignore"):   # failed seeds carry theta 0
        eta = -np.log(np.tan(0.5 * r["p"][:, 5]))
    near = (r["status"] == 0) & (np.abs(np.abs(eta) - g.barrel_eta_max) < 1e-5)
    side = np.where(eta > 0, 1, 2)
    assert np.all((info[near, 0] == 0) | (info[near, 0] == side[near]))
    far = ~near
    bad_region = np.nonzero(far & (info[:, 0] != r["region"]))[0]
    ok = far & (r["status"] == 0)
    pok, prat = PR.param_close(state[ok], r["p"][ok])
    cok, crat = PR.cov_close_surface(cov[ok], r["c"][ok], r["p"][ok], r["surf"])
    okidx = np.nonzero(ok)[0]
    bad = okidx[~(pok.all(1) & cok.all(1))]
    _report("seed_full_size", dict(seeds=int(n), near_ties=int(near.sum()), bad_region=bad_region[:20],
                                   n_bad=int(bad.size), bad=bad[:50], bad_param_ratio=prat.max(1)[~(pok.all(1) & cok.all(1))][:50],
                                   bad_cov_ratio=crat.max(1)[~(pok.all(1) & cok.all(1))][:50],
                                   worst_param=float(prat.max()), worst_cov=float(crat.max())))
    assert bad_region.size == 0, (bad_region[:10], eta[bad_region[:10]])
    assert np.array_equal(info[far, 1], r["start"][far]) and np.array_equal(info[far, 2], r["status"][far])
    assert near.sum() < 20
    assert pok.all(), (int((~pok.all(1)).sum()), float(prat.max()))
    assert cok.all(), (int((~cok.all(1)).sum()), float(crat.max()))


# ------------------------------------------------------------------ uneven events, loopers at scale

def test_uneven_256_events_at_size_sampled_against_oracle(lib):
    """The uneven-batch workload at its size, as the benchmark runs it: 256 events of Poisson(8,000)
    tracks clipped to [200, 25,000], ~2.05M seeds searched in one call with the search kernels'
    shapes autotuned on the batch; the oracle recomputes a random sample of seeds and fit tracks
    (searches are independent per seed)."""
    import os
    import torch
    g, evs = S.workload_uneven(processes=min(16, os.cpu_count() or 1))
    batch = S.concat_events(evs, g.n_layers)
    assert batch.n_events == 256 and batch.seed_hits.shape[0] > 2_000_000
    params = S.default_params()
    ctx = _ctx(g, params)
    fi = pipeline.fit_inputs(batch)
    db = pipeline.DeviceBatch(batch, fi, g.max_plan, "cuda")
    pipeline.run_step(ctx, db)
    torch.cuda.synchronize()
    ctx.autotune(reps=1)   # keeps the fastest shapes, as the benchmark's pass does
    pipeline.run_step_fused(ctx, db)
    torch.cuda.synchronize()
    gpu = {k: v.cpu().numpy() for k, v in db.out.items()}
    rng = np.random.default_rng(17)
    sample = np.sort(rng.choice(batch.seed_hits.shape[0], 400, replace=False))
    orc = oracle.Oracle(g, params)
    rep = _report("build_uneven_256", PR.compare_build(gpu, PR.oracle_build(orc, batch, sample)))
    assert len(rep["hit_mismatch"]) == 0 and rep["failed_mismatch"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
    tsample = np.sort(rng.choice(fi.layers.shape[0], 2000, replace=False))
    r = orc.fit_batch(fi.layers[tsample], fi.hits[tsample], batch.hit_xyz.astype(np.float64),
                      batch.hit_cov.astype(np.float64), fi.p0[tsample].astype(np.float64),
                      fi.c0[tsample].astype(np.float64))
    gf = {k: db.fit[k].cpu().numpy()[tsample] for k in ("p", "c", "chi2", "status")}
    rep = _report("fit_uneven_256", PR.compare_fit(gf, r))
    assert rep["status_bad"] == 0 and rep["param_bad"] == 0 and rep["chi2_bad"] == 0 and rep["cov_bad"] == 0, rep


def test_uneven_events_match_oracle(lib):
    """Events of very different sizes in one call (Poisson track counts as in the uneven-batch
    workload, plus a 20-track, a 1,500-track and a track-less event with noise only): every
    seed and every fit track against the oracle."""
    rng = np.random.default_rng(3)
    counts = list(np.clip(rng.poisson(400, 5), 200, 25000)) + [20, 1500, 0]
    g, evs = S.workload_uneven(counts=counts, seed=3, noise_per_track=2.5)
    batch = S.concat_events(evs, g.n_layers)
    params = S.default_params()
    ctx = _ctx(g, params)
    fi = pipeline.fit_inputs(batch)
    res = pipeline.run_host(ctx, batch, g.max_plan, fi)
    orc = oracle.Oracle(g, params)
    o = PR.oracle_build(orc, batch)
    rep = _report("build_uneven", PR.compare_build(res["build"], o))
    assert len(rep["hit_mismatch"]) == 0 and rep["failed_mismatch"] == 0, rep
    assert rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0 and rep["count_bad"] == 0, rep
    r = orc.fit_batch(fi.layers, fi.hits, batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64),
                      fi.p0.astype(np.float64), fi.c0.astype(np.float64))
    rf = PR.compare_fit(res["fit"], r)
    assert rf["status_bad"] == 0 and rf["param_bad"] == 0 and rf["cov_bad"] == 0 and rf["chi2_bad"] == 0, rf


@pytest.fixture(scope="module")
def loopers_1m():
    g, evs = S.workload_loopers(n_events=50, n_tracks=20000, seed=5)
    return g, S.concat_events(evs, g.n_layers)


def test_loopers_precision_sweep_1m_tracks(lib, loopers_1m):
    """1,000,000 tracks over 34 layers, 10% at 0.5-0.7 GeV: the FP32 fit (FP64 refit of the
    tracks with an ill-conditioned S) and the all-FP64 fit against the oracle on a sample;
    errors in units of the tolerances and pulls against the generator's truth are reported."""
    import torch
    g, batch = loopers_1m
    fi = pipeline.fit_inputs(batch)
    assert fi.layers.shape[0] > 900_000
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(fi.layers.shape[0], 3000, replace=False))
    orc = oracle.Oracle(g, S.default_params())
    X, V = batch.hit_xyz.astype(np.float64), batch.hit_cov.astype(np.float64)
    r = orc.fit_batch(fi.layers[sample], fi.hits[sample], X, V, fi.p0[sample].astype(np.float64),
                      fi.c0[sample].astype(np.float64))
    out = {}
    for name, prec in (("fp32", 0), ("fp64", 2)):
        ctx = _ctx(g, dict(S.default_params(), precision=prec))
        ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                      torch.from_numpy(batch.hit_cov).cuda())
        d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda()
             for k, v in dict(layers=fi.layers, hits=fi.hits, p0=fi.p0, c0=fi.c0).items()}
        n = fi.layers.shape[0]
        o = dict(p=torch.zeros((n, 6), device="cuda"), c=torch.zeros((n, 21), device="cuda"),
                 chi2=torch.zeros(n, device="cuda"), status=torch.zeros(n, dtype=torch.int32, device="cuda"))
        ctx.fit(d["layers"], d["hits"], d["p0"], d["c0"], o["p"], o["c"], o["chi2"], o["status"])
        torch.cuda.synchronize()
        h = {k: v.cpu().numpy()[sample] for k, v in o.items()}
        rep = _report(f"fit_loopers_1m_{name}", PR.compare_fit(h, r))
        assert rep["status_bad"] == 0 and rep["param_bad"] == 0 and rep["cov_bad"] == 0 and rep["chi2_bad"] == 0, rep
        out[name] = rep
    assert out["fp64"]["worst_param"] <= out["fp32"]["worst_param"] + 1e-6
