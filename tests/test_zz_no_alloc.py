"""mkgb_fit_static (the fit entry point whose scratch is a fixed device array, no allocation)
against mkgb_fit on the same device inputs: two calls in a row of different sizes must each
reproduce mkgb_fit bit for bit, including the tracks refit in FP64 through the scratch list."""
import numpy as np
import pytest

from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu

MAX_TRACKS = 1 << 16


def _device_fit_inputs(fi, lo, hi):
    import torch
    d = dict(layers=fi.layers[lo:hi], hits=fi.hits[lo:hi], p0=fi.p0[lo:hi], c0=fi.c0[lo:hi])
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in d.items()}


def _outputs(n):
    import torch
    return dict(p=torch.zeros((n, 6), dtype=torch.float32, device="cuda"),
                c=torch.zeros((n, 21), dtype=torch.float32, device="cuda"),
                chi2=torch.zeros(n, dtype=torch.float32, device="cuda"),
                status=torch.full((n,), -7, dtype=torch.int32, device="cuda"))


def _run(fn, x, o):
    fn(x["layers"], x["hits"], x["p0"], x["c0"], o["p"], o["c"], o["chi2"], o["status"])


def _host(o):
    import torch
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in o.items()}


@pytest.fixture(scope="module")
def setup():
    B.build()
    mkgb.load_library()
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, 2500, 0, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=3000)
           for e in range(2)]
    batch = S.concat_events(evs, g.n_layers)
    fi = pipeline.fit_inputs(batch)
    return g, batch, fi


@pytest.mark.parametrize("kappa", [1e3, 0.0])
def test_two_calls_in_a_row_match_mkgb_fit(setup, kappa):
    import torch
    g, batch, fi = setup
    params = dict(S.default_params(), kappa_fp64=kappa)   # 1e3 sends many tracks to the FP64 refit list
    ctx = pipeline.make_context(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                  torch.from_numpy(batch.hit_cov).cuda())
    n = fi.layers.shape[0]
    # first call on the whole batch, second on a smaller slice (a stale list tail would show)
    for lo, hi in ((0, n), (n // 3, n // 3 + n // 4)):
        x = _device_fit_inputs(fi, lo, hi)
        ref, got = _outputs(hi - lo), _outputs(hi - lo)
        _run(ctx.fit, x, ref)
        _run(ctx.fit_static, x, got)
        a, b = _host(ref), _host(got)
        for k in a:
            assert np.array_equal(a[k], b[k]), (lo, hi, k)
        assert (b["status"] == 0).mean() > 0.95


def test_refit_list_is_used(setup):
    """With a low threshold the static call's output differs from the no-refit output."""
    import torch
    g, batch, fi = setup
    outs = []
    for kappa in (1e3, 0.0):
        ctx = pipeline.make_context(g, dict(S.default_params(), kappa_fp64=kappa))
        ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                      torch.from_numpy(batch.hit_cov).cuda())
        x = _device_fit_inputs(fi, 0, fi.layers.shape[0])
        o = _outputs(fi.layers.shape[0])
        _run(ctx.fit_static, x, o)
        outs.append(_host(o))
    changed = np.any(outs[0]["c"] != outs[1]["c"], axis=1)
    assert changed.sum() > 10


def test_limits_and_empty(setup):
    import torch
    g, batch, fi = setup
    ctx = pipeline.make_context(g, S.default_params())
    ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                  torch.from_numpy(batch.hit_cov).cuda())
    # over the static limit: rejected before any device work, with the limit in the message
    n = MAX_TRACKS + 1
    x = dict(layers=torch.full((n, 1), -1, dtype=torch.int32, device="cuda"),
             hits=torch.full((n, 1), -1, dtype=torch.int32, device="cuda"),
             p0=torch.zeros((n, 6), dtype=torch.float32, device="cuda"),
             c0=torch.zeros((n, 21), dtype=torch.float32, device="cuda"))
    with pytest.raises(mkgb.MkgbError, match="65536"):
        _run(ctx.fit_static, x, _outputs(n))
    # host arrays are refused by the binding
    with pytest.raises(mkgb.MkgbError):
        ctx.fit_static(fi.layers[:2], fi.hits[:2], fi.p0[:2], fi.c0[:2], np.zeros((2, 6), np.float32),
                       np.zeros((2, 21), np.float32), np.zeros(2, np.float32))
    # zero tracks is a no-op
    x0 = _device_fit_inputs(fi, 0, 0)
    _run(ctx.fit_static, x0, _outputs(0))
    torch.cuda.synchronize()


def test_largest_batch_every_refit_slot(setup):
    """Exactly 65536 tracks (the largest accepted batch) with a threshold low enough that a large
    part of them goes through the refit list: the static call still equals mkgb_fit, and a second
    call leaves the device's free memory unchanged (no allocation in the call)."""
    import torch
    g, batch, fi = setup
    ctx = pipeline.make_context(g, dict(S.default_params(), kappa_fp64=1e3))
    ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                  torch.from_numpy(batch.hit_cov).cuda())
    reps = -(-MAX_TRACKS // fi.layers.shape[0])
    tile = lambda a: np.ascontiguousarray(np.concatenate([a] * reps)[:MAX_TRACKS])
    x = {k: torch.from_numpy(tile(v)).cuda() for k, v in
         dict(layers=fi.layers, hits=fi.hits, p0=fi.p0, c0=fi.c0).items()}
    ref, got = _outputs(MAX_TRACKS), _outputs(MAX_TRACKS)
    _run(ctx.fit, x, ref)
    _run(ctx.fit_static, x, got)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    _run(ctx.fit_static, x, got)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    a, b = _host(ref), _host(got)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert (b["status"] == 0).mean() > 0.95


def test_module_hits_match_mkgb_fit():
    """Module hits (taken on their module planes) go through the same static call."""
    import torch
    B.build()
    mkgb.load_library()
    g = S.geometry_phase2_modular_disks()
    ev = S.simulate_event(g, 1500, 4, 0, pt_sampler=S.sample_pt_phase2, eta_max=2.5, noise_total=2000)
    b = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(b)
    ctx = pipeline.make_context(g, S.default_params())
    ctx.load_hits(b.n_events, b.hit_off, torch.from_numpy(b.hit_xyz).cuda(), torch.from_numpy(b.hit_cov).cuda(),
                  hit_module=torch.from_numpy(b.hit_mod).cuda())
    x = _device_fit_inputs(fi, 0, fi.layers.shape[0])
    ref, got = _outputs(fi.layers.shape[0]), _outputs(fi.layers.shape[0])
    _run(ctx.fit, x, ref)
    for _ in range(2):
        _run(ctx.fit_static, x, got)
        a, c = _host(ref), _host(got)
        for k in a:
            assert np.array_equal(a[k], c[k]), k
    assert (c["status"] == 0).mean() > 0.95
