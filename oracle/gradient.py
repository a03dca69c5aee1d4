"""Reference gradient of the fit's total chi2 (test infrastructure: FP64 central differences of
the oracle's fit over a known assignment, Sec. 4).

Parameters: per layer l an alignment (d_x, d_y, d_z, w_x, w_y, w_z) moving the layer's hits as
h' = h + d + w x (h - c_l), with c_l the origin for a cylinder and (0, 0, z_l) for a disk (the
surfaces stay nominal), and a thickness scale m_l multiplying the layer's x/X0; per track its 6
starting parameters p0.  The total chi2 is the sum over the tracks that fit (status 0) of their
summed predicted chi2.  Derivatives are plain symmetric differences (f(x + h) - f(x - h)) / 2h
in FP64, with h relative to the parameter's natural scale; they are the definition of the
derivative, exact up to O(h^2) truncation and O(eps / h) rounding.
"""
from __future__ import annotations

import copy

import numpy as np

from . import Oracle


def aligned_hits(geom, hit_xyz, hit_layer, align):
    """Hits moved by the per-layer alignment (FP64)."""
    X = np.asarray(hit_xyz, np.float64).copy()
    align = np.asarray(align, np.float64)
    for l in range(geom.n_layers):
        sel = hit_layer == l
        if not np.any(sel):
            continue
        d, w = align[l, :3], align[l, 3:]
        if not np.any(d) and not np.any(w):
            continue
        c = np.array([0.0, 0.0, float(geom.pos[l]) if geom.kind[l] == 1 else 0.0])
        rel = X[sel] - c
        X[sel] = X[sel] + d + np.cross(w, rel)
    return X


def _geom_scaled(geom, xscale):
    g2 = copy.deepcopy(geom)
    g2.x_over_x0 = np.asarray(geom.x_over_x0, np.float64) * np.asarray(xscale, np.float64)
    return g2


def total_chi2(geom, params, layers, hits, hit_xyz, hit_cov, hit_layer, p0, c0, align, xscale, per_track=False,
               hit_mod=None):
    orc = Oracle(_geom_scaled(geom, xscale), params)
    if hit_mod is not None:   # module hits used on their module planes (nominal, not aligned)
        orc.set_modules(geom.modules.c, geom.modules.n, hit_mod)
    X = aligned_hits(geom, hit_xyz, hit_layer, align)
    r = orc.fit_batch(layers, hits, X, np.asarray(hit_cov, np.float64), np.asarray(p0, np.float64),
                      np.asarray(c0, np.float64))
    chi2 = np.where(r["status"] == 0, r["chi2"], 0.0)
    return (chi2, r["status"]) if per_track else float(chi2.sum())


def fd_gradient(geom, params, layers, hits, hit_xyz, hit_cov, hit_layer, p0, c0, align=None, xscale=None,
                h_shift=1e-4, h_rot=1e-6, h_scale=1e-3, h_p0=(1e-4, 1e-4, 1e-4, 1e-5, 1e-6, 1e-6), hit_mod=None):
    """FP64 central differences: (chi2 per track, status, d/dp0 [n, 6], d/dalign [L, 6], d/dxscale [L]).

    Steps: the oracle's chi2 carries ~1e-8 absolute noise from its Newton stopping rule, so the
    steps are ~1 um for shifts and rotations at 1 m, 1e-3 for the thickness scales, 1 um and
    1e-5 c/GeV or 1e-6 rad for the starting parameters; the truncation error at these steps is
    below 1e-5 relative (central differences converge as h^2)."""
    L = geom.n_layers
    align = np.zeros((L, 6)) if align is None else np.asarray(align, np.float64)
    xscale = np.ones(L) if xscale is None else np.asarray(xscale, np.float64)
    p0 = np.asarray(p0, np.float64)
    args = (geom, params, layers, hits, hit_xyz, hit_cov, hit_layer)
    kw = dict(per_track=True, hit_mod=hit_mod)
    chi2, status = total_chi2(*args, p0, c0, align, xscale, **kw)
    ok = status == 0
    # per-track starting parameters: each track's chi2 depends on its own p0 only
    dp0 = np.zeros_like(p0)
    for k in range(6):
        dp = np.zeros_like(p0)
        dp[:, k] = h_p0[k]
        cp, sp = total_chi2(*args, p0 + dp, c0, align, xscale, **kw)
        cm, sm = total_chi2(*args, p0 - dp, c0, align, xscale, **kw)
        dp0[:, k] = np.where(ok & (sp == 0) & (sm == 0), (cp - cm) / (2 * dp[:, k]), 0.0)
    used = np.unique(np.asarray(layers)[np.asarray(layers) >= 0])
    dal = np.zeros((L, 6))
    dxs = np.zeros(L)
    keep = lambda c, s: np.where(ok & (s == 0), c, 0.0).sum()
    for l in used:
        for k in range(6):
            h = h_shift if k < 3 else h_rot
            a = align.copy()
            a[l, k] += h
            cp, sp = total_chi2(*args, p0, c0, a, xscale, **kw)
            a[l, k] -= 2 * h
            cm, sm = total_chi2(*args, p0, c0, a, xscale, **kw)
            dal[l, k] = (keep(cp, sp) - keep(cm, sm)) / (2 * h)
        x = xscale.copy()
        x[l] += h_scale
        cp, sp = total_chi2(*args, p0, c0, align, x, **kw)
        x[l] -= 2 * h_scale
        cm, sm = total_chi2(*args, p0, c0, align, x, **kw)
        dxs[l] = (keep(cp, sp) - keep(cm, sm)) / (2 * h_scale)
    return chi2, status, dp0, dal, dxs
