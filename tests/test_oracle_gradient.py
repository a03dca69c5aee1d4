"""The oracle's reference gradient of the fit's total chi2 (oracle/gradient.py: FP64 central
differences) against properties the derivative must have, independent of any fit code:
symmetries of a barrel-only detector and convergence in the step size."""
import numpy as np
import pytest

from oracle import gradient as OG
from paper_2312_11728_gb300 import pipeline, synth as S


def _hit_layer(batch):
    hl = np.zeros(batch.hit_xyz.shape[0], np.int64)
    for s in range(len(batch.hit_off) - 1):
        hl[batch.hit_off[s]:batch.hit_off[s + 1]] = s % batch.n_layers
    return hl


@pytest.fixture(scope="module")
def barrel_fit():
    g = S.geometry_barrel()
    ev = S.simulate_event(g, 120, 0, 0, eta_max=0.8, noise_per_layer=0)
    batch = S.concat_events([ev], g.n_layers)
    fi = pipeline.fit_inputs(batch)
    res = OG.fd_gradient(g, S.default_params(), fi.layers, fi.hits, batch.hit_xyz, batch.hit_cov, _hit_layer(batch),
                         fi.p0, fi.c0)
    return g, batch, fi, res


def test_gradient_translation_along_z_vanishes(barrel_fit):
    """Moving every hit and every starting point along z leaves a barrel-only fit unchanged (the
    cylinders, their material and the hit errors are z-invariant away from the layer ends)."""
    g, batch, fi, (chi2, status, dp0, dal, dxs) = barrel_fit
    total = dal[:, 2].sum() + dp0[status == 0, 2].sum()
    scale = np.abs(dal[:, 2]).sum() + np.abs(dp0[status == 0, 2]).sum()
    assert abs(total) < 1e-5 * scale, (total, scale)


def test_gradient_rotation_about_z_vanishes(barrel_fit):
    """Rotating every hit and every starting state about the z axis leaves the fit unchanged
    (the barrel hit errors are isotropic in the transverse plane): the alignment rotations w_z
    and the starting (x, y, phi) derivatives must cancel."""
    g, batch, fi, (chi2, status, dp0, dal, dxs) = barrel_fit
    ok = status == 0
    x0, y0 = fi.p0[ok, 0].astype(np.float64), fi.p0[ok, 1].astype(np.float64)
    track = dp0[ok, 4] + x0 * dp0[ok, 1] - y0 * dp0[ok, 0]
    total = dal[:, 5].sum() + track.sum()
    scale = np.abs(dal[:, 5]).sum() + np.abs(track).sum()
    assert abs(total) < 1e-5 * scale, (total, scale)


def test_gradient_is_converged_in_the_step(barrel_fit):
    """Halving the difference steps changes the derivatives by far less than their size
    (central differences converge as h^2; the steps stay above the oracle's chi2 noise)."""
    g, batch, fi, (chi2, status, dp0, dal, dxs) = barrel_fit
    r2 = OG.fd_gradient(g, S.default_params(), fi.layers, fi.hits, batch.hit_xyz, batch.hit_cov, _hit_layer(batch),
                        fi.p0, fi.c0, h_scale=5e-4, h_shift=5e-5, h_rot=5e-7, h_p0=(5e-5, 5e-5, 5e-5, 5e-6, 5e-7, 5e-7))
    assert np.allclose(r2[4], dxs, rtol=1e-5, atol=1e-7 * np.abs(dxs).max())
    assert np.allclose(r2[3], dal, rtol=2e-4, atol=1e-6 * np.abs(dal).max())
    ok = r2[1] == 0
    assert np.allclose(r2[2][ok], dp0[ok], rtol=1e-3, atol=1e-4 * np.abs(dp0[ok]).max())


def test_aligned_hits_follow_the_rigid_motion():
    """The alignment moves a layer's hits rigidly: distances between hits of one layer are kept
    (to first order in the small rotation) and the layer centre moves by the shift."""
    g = S.geometry_phase2()
    ev = S.simulate_event(g, 200, 0, 0, pt_sampler=S.sample_pt_phase2, eta_min=0.0, eta_max=3.0, noise_total=0)
    batch = S.concat_events([ev], g.n_layers)
    hl = _hit_layer(batch)
    al = np.zeros((g.n_layers, 6))
    al[12] = [1e-3, -2e-3, 3e-3, 0.0, 0.0, 1e-4]
    X = OG.aligned_hits(g, batch.hit_xyz, hl, al)
    sel = hl == 12
    other = ~sel
    assert np.array_equal(X[other], batch.hit_xyz[other].astype(np.float64))
    c = np.array([0.0, 0.0, g.pos[12]])
    rel0 = batch.hit_xyz[sel].astype(np.float64) - c
    rel1 = X[sel] - c - al[12, :3]
    assert np.allclose(np.linalg.norm(rel1, axis=1), np.linalg.norm(rel0, axis=1), rtol=1e-7)
    # the move is the same as the generator's (synth.move_hits) applied to the event
    moved = S.move_hits(g, ev, al)
    assert np.allclose(S.concat_events([moved], g.n_layers).hit_xyz, X, atol=1e-5)
