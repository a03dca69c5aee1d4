"""Derivative of the fit's total chi2 on the GPU (mkgb_fit_grad, FP32 dual numbers: the reverse
sweep over checkpointed steps and the forward mode) against the oracle's exact FP64 derivative
(forward-mode dual numbers over the oracle's fit, oracle/dualfit.py) with tight bounds, against
the oracle's FP64 central differences (oracle/gradient.py) on the full 400-track workload, against
each other and against the symmetries of a barrel-only detector.

The bounds below are those of the central-difference comparison:

Tolerances, derived from the arithmetic: the derivative of a track's chi2 carries FP32 rounding
(2^-24) amplified by the conditioning of its fit (condition numbers of S of 1e3-1e5 for typical
tracks, up to 2^24 for the worst), i.e. 1e-4 to 1e-2 relative; central differences of the FP64
oracle are good to ~1e-4 relative at their steps.  Sums over tracks (the per-layer derivatives)
average the per-track errors.  So: per-layer derivatives within 1e-2 relative plus 1e-3 of the
largest of their kind; per-track derivatives with a median error below 1e-3 and 98% of the tracks
within 1e-2 (relative, floored at 1e-3 of the largest of their kind)."""
import numpy as np
import pytest

from oracle import gradient as OG
from oracle import parity as PR
from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mkgb.load_library()


def _hit_layer(batch):
    hl = np.zeros(batch.hit_xyz.shape[0], np.int64)
    for s in range(len(batch.hit_off) - 1):
        hl[batch.hit_off[s]:batch.hit_off[s + 1]] = s % batch.n_layers
    return hl


def _gpu_grad(g, batch, fi, align=None, xscale=None, params=None, mode=0):
    params = params or S.default_params()
    ctx = pipeline.make_context(g, params)
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    n, L = fi.layers.shape[0], g.n_layers
    align = np.zeros((L, 6), np.float32) if align is None else np.asarray(align, np.float32)
    xscale = np.ones(L, np.float32) if xscale is None else np.asarray(xscale, np.float32)
    out = dict(chi2=np.zeros(n, np.float32), dp0=np.zeros((n, 6), np.float32), dal=np.zeros((L, 6), np.float32),
               dxs=np.zeros(L, np.float32), status=np.zeros(n, np.int32))
    ctx.fit_grad(fi.layers, fi.hits, fi.p0, fi.c0, align, xscale, out["chi2"], out["dp0"], out["dal"], out["dxs"],
                 out["status"], mode=mode)
    return out


def _check_layer_grads(got, ref, name):
    lhs = np.abs(got - ref)
    rhs = 1e-2 * np.abs(ref) + 1e-3 * np.abs(ref).max()
    assert np.all(lhs <= rhs), (name, float((lhs / rhs).max()))


def _check_track_grads(got, ref, name):
    for k in range(got.shape[1]):
        r = np.abs(got[:, k] - ref[:, k]) / np.maximum(np.abs(ref[:, k]), 1e-3 * np.abs(ref[:, k]).max())
        assert np.median(r) < 1e-3 and np.percentile(r, 98) < 1e-2, (name, k, np.median(r), np.percentile(r, 98))


@pytest.fixture(scope="module")
def aligned_small():
    g, evs, al, xs = S.workload_aligned_fit(n_tracks=400, seed=2)
    batch = S.concat_events(evs, g.n_layers)
    return g, batch, pipeline.fit_inputs(batch), al, xs


@pytest.mark.parametrize("at_truth", [False, True])
def test_fit_gradient_matches_oracle_differences(lib, aligned_small, at_truth):
    """400 tracks through a misaligned detector with off-nominal material; derivatives at the
    nominal alignment and material, and at the ones that undo the simulated misalignment (to
    first order: the opposite shifts and rotations) with the true material."""
    g, batch, fi, al, xs = aligned_small
    align, xscale = (-al, xs) if at_truth else (None, None)
    chi2, status, dp0, dal, dxs = OG.fd_gradient(g, S.default_params(), fi.layers, fi.hits, batch.hit_xyz,
                                                 batch.hit_cov, _hit_layer(batch), fi.p0, fi.c0, align, xscale)
    ok = status == 0
    assert ok.mean() > 0.98
    used = np.unique(fi.layers[fi.layers >= 0])
    for mode in (0, 1):   # reverse sweep, forward mode
        got = _gpu_grad(g, batch, fi, align, xscale, mode=mode)
        assert np.array_equal(got["status"], status), mode
        c_ok, _ = PR.chi2_close(got["chi2"][ok], chi2[ok])
        assert c_ok.all(), mode
        _check_layer_grads(got["dal"][used], dal[used], f"align mode {mode}")
        _check_layer_grads(got["dxs"][used], dxs[used], f"xscale mode {mode}")
        _check_track_grads(got["dp0"][ok], dp0[ok], f"p0 mode {mode}")
    if at_truth:
        # undoing the misalignment lowers the chi2
        assert got["chi2"][ok].sum() < _gpu_grad(g, batch, fi)["chi2"][ok].sum()


def test_fit_gradient_barrel_symmetries(lib):
    """A barrel-only fit is invariant under a common z translation and a common rotation about
    the z axis of all hits and starting states; the derivatives must cancel accordingly."""
    g = S.geometry_barrel()
    ev = S.simulate_event(g, 400, 1, 0, eta_max=0.8, noise_per_layer=0)
    batch = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(batch)
    got = _gpu_grad(g, batch, fi)
    ok = got["status"] == 0
    dp0, dal = got["dp0"][ok].astype(np.float64), got["dal"].astype(np.float64)
    tz = dal[:, 2].sum() + dp0[:, 2].sum()
    assert abs(tz) < 1e-3 * (np.abs(dal[:, 2]).sum() + np.abs(dp0[:, 2]).sum())
    x0, y0 = fi.p0[ok, 0].astype(np.float64), fi.p0[ok, 1].astype(np.float64)
    track = dp0[:, 4] + x0 * dp0[:, 1] - y0 * dp0[:, 0]
    rz = dal[:, 5].sum() + track.sum()
    assert abs(rz) < 1e-3 * (np.abs(dal[:, 5]).sum() + np.abs(track).sum())


def test_autograd_function(lib, aligned_small):
    """FitChi2 as a torch.autograd.Function: backward gives the entry point's derivatives, and a
    small step against the alignment gradient lowers the total chi2."""
    import torch
    from paper_2312_11728_gb300.fitgrad import FitChi2
    g, batch, fi, al, xs = aligned_small
    ctx = pipeline.make_context(g, S.default_params())
    ctx.load_hits(batch.n_events, batch.hit_off, torch.from_numpy(batch.hit_xyz).cuda(),
                  torch.from_numpy(batch.hit_cov).cuda())
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    layers, hits, c0 = dev(fi.layers), dev(fi.hits), dev(fi.c0)
    align = torch.zeros((g.n_layers, 6), device="cuda", requires_grad=True)
    xscale = torch.ones(g.n_layers, device="cuda", requires_grad=True)
    p0 = dev(fi.p0).requires_grad_(True)
    total, status = FitChi2.apply(align, xscale, p0, ctx, layers, hits, c0)
    total.backward()
    ref = _gpu_grad(g, batch, fi)
    assert np.allclose(align.grad.cpu().numpy(), ref["dal"], rtol=1e-5, atol=1e-3)
    assert np.allclose(xscale.grad.cpu().numpy(), ref["dxs"], rtol=1e-5, atol=1e-3)
    assert np.allclose(p0.grad.cpu().numpy(), ref["dp0"], rtol=1e-5, atol=1e-3)
    assert total.item() == pytest.approx(ref["chi2"][ref["status"] == 0].sum(), rel=1e-6)
    with torch.no_grad():
        # largest change 1e-6 (cm or rad: ~1 um at 1 m against 30 um hit errors)
        step = -1e-6 * align.grad / align.grad.abs().max()
        t2, _ = FitChi2.apply(align + step, xscale, p0, ctx, layers, hits, c0)
    assert t2.item() < total.item()


def test_fit_gradient_full_size_sampled(lib):
    """The differentiable-fit workload at full size: 100,000 tracks over 22 layers of a
    misaligned detector.  Per-track derivatives of a sample against the oracle's differences."""
    g, evs, al, xs = S.workload_aligned_fit(n_tracks=100_000, seed=4)
    batch = S.concat_events(evs, g.n_layers)
    fi = pipeline.fit_inputs(batch)
    assert fi.layers.shape[0] > 99_000
    got = _gpu_grad(g, batch, fi)
    assert (got["status"] == 0).mean() > 0.98
    assert np.all(np.isfinite(got["dal"])) and np.all(np.isfinite(got["dxs"]))
    rng = np.random.default_rng(5)
    s = np.sort(rng.choice(fi.layers.shape[0], 300, replace=False))
    chi2, status, dp0, _, _ = OG.fd_gradient(g, S.default_params(), fi.layers[s], fi.hits[s], batch.hit_xyz,
                                             batch.hit_cov, _hit_layer(batch), fi.p0[s], fi.c0[s])
    ok = (status == 0) & (got["status"][s] == 0)
    _check_track_grads(got["dp0"][s][ok], dp0[ok], "p0 sampled")


def test_reverse_sweep_matches_forward_mode(lib, aligned_small):
    """The two derivative modes evaluate the same FP32 derivatives in a different order: they
    agree to a few FP32 roundings times the fit's conditioning, far inside the oracle tolerances."""
    g, batch, fi, al, xs = aligned_small
    rev = _gpu_grad(g, batch, fi, -al, xs, mode=0)
    fwd = _gpu_grad(g, batch, fi, -al, xs, mode=1)
    assert np.array_equal(rev["status"], fwd["status"])
    # the reverse sweep's values come from its plain FP32 pass, the forward mode's from the value
    # part of its dual numbers: the same operations, contracted into multiply-adds differently
    assert np.allclose(rev["chi2"], fwd["chi2"], rtol=1e-4, atol=1e-4)
    for k in ("dal", "dxs"):
        r, f = rev[k].astype(np.float64), fwd[k].astype(np.float64)
        assert np.all(np.abs(r - f) <= 1e-3 * np.abs(f) + 1e-4 * np.abs(f).max()), k
    ok = rev["status"] == 0
    r, f = rev["dp0"][ok].astype(np.float64), fwd["dp0"][ok].astype(np.float64)
    rel = np.abs(r - f) / np.maximum(np.abs(f), 1e-3 * np.abs(f).max(axis=0))
    assert np.median(rel) < 1e-4 and np.percentile(rel, 99) < 1e-2, (np.median(rel), np.percentile(rel, 99))


def _subset(fi, n):
    from types import SimpleNamespace
    return SimpleNamespace(layers=np.ascontiguousarray(fi.layers[:n]), hits=np.ascontiguousarray(fi.hits[:n]),
                           p0=np.ascontiguousarray(fi.p0[:n]), c0=np.ascontiguousarray(fi.c0[:n]))


@pytest.mark.parametrize("at_truth", [False, True])
def test_fit_gradient_matches_exact_derivative(lib, aligned_small, at_truth):
    """80 of the tracks against the oracle's exact FP64 derivative (forward-mode dual numbers over
    the oracle's fit, oracle/dualfit.py), with no difference noise on the reference side: the
    remaining error is the GPU's FP32 rounding (6e-8) amplified by the conditioning of each
    track's fit (kappa(S) ~ 1e2 typical, up to ~1e5).  Bounds: per-layer derivatives within 5e-4
    of the largest of their kind (measured <= 1e-4); per track, relative to the derivative floored
    at 1e-3 of the largest of its kind, median < 1e-4 (measured <= 2.3e-5), 98th percentile < 3e-3
    (<= 1.0e-3), every track < 1e-2 (<= 3.1e-3)."""
    from oracle import dualfit as DF
    g, batch, fi, al, xs = aligned_small
    sub = _subset(fi, 80)
    align = (-al).astype(np.float32) if at_truth else np.zeros((g.n_layers, 6), np.float32)
    xscale = xs.astype(np.float32) if at_truth else np.ones(g.n_layers, np.float32)
    chi2, status, dp0, dal, dxs = DF.gradient(g, sub.layers, sub.hits, batch.hit_xyz, batch.hit_cov, sub.p0,
                                              sub.c0, align.astype(np.float64), xscale.astype(np.float64))
    ok = status == 0
    used = np.unique(sub.layers[sub.layers >= 0])
    for mode in (0, 1):
        got = _gpu_grad(g, batch, sub, align, xscale, mode=mode)
        assert np.array_equal(got["status"], status), mode
        lay = [np.abs(got["dal"][used] - dal[used]).max() / np.abs(dal[used]).max(),
               np.abs(got["dxs"][used] - dxs[used]).max() / np.abs(dxs[used]).max()]
        trk = []
        for k in range(6):
            r = np.abs(got["dp0"][ok, k] - dp0[ok, k]) / np.maximum(np.abs(dp0[ok, k]), 1e-3 * np.abs(dp0[ok, k]).max())
            trk.append((float(np.median(r)), float(np.percentile(r, 98)), float(r.max())))
        msg = f"mode {mode} layers {lay[0]:.1e} {lay[1]:.1e} tracks " + " ".join(f"{m:.1e}/{p:.1e}/{x:.1e}"
                                                                            for m, p, x in trk)
        assert max(lay) < 5e-4, msg
        assert all(m < 1e-4 and p < 3e-3 and x < 1e-2 for m, p, x in trk), msg
