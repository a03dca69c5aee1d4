"""Comparison of the CUDA path's outputs with the oracle's (test infrastructure).

Tolerances (stated by the method's target): parameters |dp_i| <= 1e-4 * max(|p_i|, f_i) with
floors f = (1, 1, 1, 0.01, 1, 1) (phi compared modulo 2 pi); covariance
|dC_ij| <= 1e-3 * sqrt(C_ii C_jj); chi2 |d chi2| <= 1e-3 * max(1, chi2); selected hit indices
bit-exact up to the first near-tie step the oracle flags for that seed.
"""
from __future__ import annotations

import numpy as np

from . import Oracle, hit_layers

P_FLOOR = np.array([1.0, 1.0, 1.0, 0.01, 1.0, 1.0])
TRI = np.tril_indices(6)


def param_close(pg, po, rel=1e-4):
    d = np.abs(np.asarray(pg, np.float64) - po)
    d[..., 4] = np.abs(np.angle(np.exp(1j * (np.asarray(pg, np.float64)[..., 4] - po[..., 4]))))
    tol = rel * np.maximum(np.abs(po), P_FLOOR)
    return d <= tol, d / tol


def cov_close(cg, co, rel=1e-3, floor=1e-5):
    """|dC_ij| <= rel * sqrt(d_i d_j).  d_i = C_ii, the position variances floored at `floor` of
    the largest position variance.  A state on a layer surface has no variance along the surface
    normal in exact arithmetic (a disk state none in z; a barrel state at x ~ R, y ~ 0 almost
    none in x), so such an entry is a projection of the in-surface variance through a small
    angle plus rounding residue: FP32 arithmetic resolves it to ~1e-9 of the largest position
    variance (a fraction of FP32's 6e-8 epsilon), which the 1e-3 relative test cannot ask of an
    entry below 1e-5 of that largest variance."""
    cg = np.asarray(cg, np.float64)
    diag_idx = [i * (i + 1) // 2 + i for i in range(6)]
    dg = np.abs(co[..., diag_idx])
    pos_max = dg[..., :3].max(axis=-1, keepdims=True)
    dg = np.concatenate([np.maximum(dg[..., :3], floor * pos_max), dg[..., 3:]], axis=-1)
    scale = np.sqrt(dg[..., TRI[0]] * dg[..., TRI[1]])
    d = np.abs(cg - co)
    return d <= rel * scale + 1e-30, d / (rel * scale + 1e-30)


def surface_frames(po, surf, tol=1e-4):
    """Per state (oracle parameters po, n x 6) the rotation T = diag(R, I3), R's rows the surface
    normal n, e1 (the direction projected onto the surface) and e2 = n x e1, of the layer surface
    the state lies on (surf = (kind, position) per layer: a cylinder |r - R| or a disk |z - z_d|
    within tol cm); on = False where no layer surface is that close (a module plane)."""
    kind, pos = (np.asarray(a) for a in surf)
    x, y, z = po[:, 0], po[:, 1], po[:, 2]
    r = np.hypot(x, y)
    d = np.where(kind[None, :] == 0, np.abs(r[:, None] - pos[None, :]), np.abs(z[:, None] - pos[None, :]))
    lay = np.argmin(d, axis=1)
    on = d[np.arange(len(po)), lay] < tol
    barrel = kind[lay] == 0
    rs = np.where(r > 0, r, 1.0)
    nrm = np.where(barrel[:, None], np.stack([x / rs, y / rs, np.zeros_like(x)], 1),
                   np.array([0.0, 0.0, 1.0])[None, :])
    st = np.sin(po[:, 5])
    u = np.stack([st * np.cos(po[:, 4]), st * np.sin(po[:, 4]), np.cos(po[:, 5])], 1)
    e1 = u - (u * nrm).sum(1, keepdims=True) * nrm
    l1 = np.linalg.norm(e1, axis=1, keepdims=True)
    on &= l1[:, 0] > 1e-6
    e1 = e1 / np.where(l1 > 0, l1, 1.0)
    e2 = np.cross(nrm, e1)
    T = np.zeros((len(po), 6, 6))
    T[:, 0, :3], T[:, 1, :3], T[:, 2, :3] = nrm, e1, e2
    T[:, 3, 3] = T[:, 4, 4] = T[:, 5, 5] = 1.0
    return T, on


def _full(c21):
    M = np.zeros(c21.shape[:-1] + (6, 6))
    M[..., TRI[0], TRI[1]] = c21
    M[..., TRI[1], TRI[0]] = c21
    return M


def cov_close_surface(cg, co, po, surf, rel=1e-3, normal_floor=1e-4):
    """The covariance test in the frame of the surface each state lies on: coordinates (n, e1,
    e2, k, phi, theta), n the surface normal.  |dC_ij| <= rel * sqrt(d_i d_j) with d_i = C_ii of
    the oracle, unfloored for the five in-surface coordinates; only the normal variance, zero in
    exact arithmetic for a state on its surface, is floored at normal_floor of the largest
    in-surface position variance: FP32 storage of the global-frame matrix alone leaves a few
    1e-9 of that variance in the normal entries (the rotation mixes entries of that size), so
    the normal row is held to ~1e-7 of it.  States on no layer surface within 1e-4 cm (a module
    plane) take the global-frame test."""
    cg = np.asarray(cg, np.float64)
    co = np.asarray(co, np.float64)
    if len(co) == 0:
        return np.zeros((0, 21), bool), np.zeros((0, 21))
    T, on = surface_frames(np.asarray(po, np.float64), surf)
    Mg = T @ _full(cg) @ T.transpose(0, 2, 1)
    Mo = T @ _full(co) @ T.transpose(0, 2, 1)
    dg = np.abs(np.diagonal(Mo, axis1=1, axis2=2)).copy()
    dg[:, 0] = np.maximum(dg[:, 0], normal_floor * dg[:, 1:3].max(1))
    scale = np.sqrt(dg[:, TRI[0]] * dg[:, TRI[1]])
    d = np.abs(Mg[:, TRI[0], TRI[1]] - Mo[:, TRI[0], TRI[1]])
    ok, ratio = d <= rel * scale + 1e-30, d / (rel * scale + 1e-30)
    if (~on).any():
        ok_g, ratio_g = cov_close(cg[~on], co[~on], rel)
        ok[~on], ratio[~on] = ok_g, ratio_g
    return ok, ratio


def chi2_close(xg, xo, rel=1e-3):
    d = np.abs(np.asarray(xg, np.float64) - xo)
    tol = rel * np.maximum(1.0, np.abs(xo))
    return d <= tol, d / tol


def oracle_build(orc: Oracle, batch, seed_index=None, binned=True):
    """Oracle forward search for the given seeds of a batch (all seeds by default), event by event."""
    S = batch.seed_hits.shape[0]
    idx = np.arange(S) if seed_index is None else np.asarray(seed_index)
    L = batch.n_layers
    xyz = batch.hit_xyz.astype(np.float64)
    cov = batch.hit_cov.astype(np.float64)
    mp = max(len(p) for p in orc.geom.plans)
    res = None
    for e in np.unique(batch.seed_event[idx]):
        sel = idx[batch.seed_event[idx] == e]
        lo = batch.hit_off[e * L:(e + 1) * L + 1]
        sh = batch.seed_hits[sel]
        r = orc.build_event(lo, xyz, cov, sh, hit_layers(lo, sh), binned=binned)
        if res is None:
            res = {k: (np.zeros((len(idx),) + v.shape[1:], v.dtype) if k != "counters" else np.zeros(4, np.int64))
                   for k, v in r.items()}
            pos = {s: i for i, s in enumerate(idx)}
        rows = [pos[s] for s in sel]
        for k, v in r.items():
            if k == "counters":
                res[k] += v
            else:
                res[k][rows] = v
    res["seed_index"] = idx
    res["max_plan"] = mp
    res["surf"] = orc.surfaces()
    return res


def oracle_build_backward(orc: Oracle, batch, track_event, p_start, c_start, first_layer, index=None,
                          binned=True):
    """Oracle backward search (Sec. 2.2) of the given tracks (all by default), event by event; the
    result has the layout of oracle_build (seed_index = the track indices)."""
    T = len(first_layer)
    idx = np.arange(T) if index is None else np.asarray(index)
    L = batch.n_layers
    xyz = batch.hit_xyz.astype(np.float64)
    cov = batch.hit_cov.astype(np.float64)
    mp = max(len(p) for p in orc.geom.plans)
    res = None
    ev = np.asarray(track_event)
    for e in np.unique(ev[idx]):
        sel = idx[ev[idx] == e]
        lo = batch.hit_off[e * L:(e + 1) * L + 1]
        r = orc.build_backward_event(lo, xyz, cov, np.asarray(p_start, np.float64)[sel],
                                     np.asarray(c_start, np.float64)[sel], np.asarray(first_layer)[sel],
                                     binned=binned)
        if res is None:
            res = {k: (np.zeros((len(idx),) + v.shape[1:], v.dtype) if k != "counters" else np.zeros(4, np.int64))
                   for k, v in r.items()}
            pos = {s: i for i, s in enumerate(idx)}
        rows = [pos[s] for s in sel]
        for k, v in r.items():
            if k == "counters":
                res[k] += v
            else:
                res[k][rows] = v
    res["seed_index"] = idx
    res["max_plan"] = mp
    res["surf"] = orc.surfaces()
    return res


def compare_build(gpu: dict, orc: dict):
    """Per-seed comparison of build outputs.  gpu: numpy arrays over all seeds; orc: oracle_build
    result for orc['seed_index'].  Returns a report dict; callers assert on it."""
    idx = orc["seed_index"]
    mp = orc["max_plan"]
    gh = np.asarray(gpu["hits"])[idx, :mp]
    oh = orc["hits"][:, :mp]
    tie = orc["tie_step"]
    n = len(idx)
    hit_ok = np.ones(n, bool)
    full = np.zeros(n, bool)
    for i in range(n):
        if tie[i] < 0:
            hit_ok[i] = np.array_equal(gh[i], oh[i])
            full[i] = True
        else:
            hit_ok[i] = np.array_equal(gh[i, :tie[i]], oh[i, :tie[i]])
    ok_score = np.isfinite(orc["score"])
    cmp = full & ok_score
    pg = np.asarray(gpu["params"])[idx]
    cg = np.asarray(gpu["cov"])[idx]
    p_ok, p_ratio = param_close(pg[cmp], orc["params"][cmp])
    if "surf" in orc:
        c_ok, c_ratio = cov_close_surface(cg[cmp], orc["cov"][cmp], orc["params"][cmp], orc["surf"])
    else:
        c_ok, c_ratio = cov_close(cg[cmp], orc["cov"][cmp])
    x_ok, x_ratio = chi2_close(np.asarray(gpu["chi2"])[idx][cmp], orc["chi2"][cmp])
    same_int = (np.asarray(gpu["nfound"])[idx][cmp] == orc["nfound"][cmp]) & \
               (np.asarray(gpu["nholes"])[idx][cmp] == orc["nholes"][cmp])
    fail_gpu = ~np.isfinite(np.asarray(gpu["score"])[idx])
    return dict(n=n, n_tie=int((tie >= 0).sum()), hit_mismatch=np.nonzero(~hit_ok)[0],
                n_full=int(cmp.sum()), param_bad=int((~p_ok).any(1).sum()), cov_bad=int((~c_ok).any(1).sum()),
                chi2_bad=int((~x_ok).sum()), count_bad=int((~same_int).sum()),
                failed_mismatch=int((fail_gpu != ~ok_score).sum()),
                worst_param=float(p_ratio.max()) if p_ratio.size else 0.0,
                worst_cov=float(c_ratio.max()) if c_ratio.size else 0.0,
                worst_chi2=float(x_ratio.max()) if x_ratio.size else 0.0,
                bad_seeds=idx[cmp][(~p_ok).any(1) | (~c_ok).any(1) | ~x_ok][:20],
                worst_cov_elem=int(np.argmax(c_ratio.max(0))) if c_ratio.size else -1,
                worst_param_elem=int(np.argmax(p_ratio.max(0))) if p_ratio.size else -1,
                worst_param_seeds=(idx[cmp][np.argsort(-p_ratio.max(1))[:5]].tolist() if p_ratio.size else []),
                worst_param_ratios=(np.sort(p_ratio.max(1))[::-1][:5].tolist() if p_ratio.size else []))


def compare_fit(gpu: dict, orc: dict, mask=None):
    st_ok = np.asarray(gpu["status"]) == orc["status"]
    m = (orc["status"] == 0) & st_ok if mask is None else mask & (orc["status"] == 0) & st_ok
    p_ok, p_ratio = param_close(np.asarray(gpu["p"])[m], orc["p"][m])
    if "surf" in orc:
        c_ok, c_ratio = cov_close_surface(np.asarray(gpu["c"])[m], orc["c"][m], orc["p"][m], orc["surf"])
    else:
        c_ok, c_ratio = cov_close(np.asarray(gpu["c"])[m], orc["c"][m])
    x_ok, x_ratio = chi2_close(np.asarray(gpu["chi2"])[m], orc["chi2"][m])
    return dict(n=int(m.sum()), status_bad=int((~st_ok).sum()), param_bad=int((~p_ok).any(1).sum()),
                cov_bad=int((~c_ok).any(1).sum()), chi2_bad=int((~x_ok).sum()),
                worst_param=float(p_ratio.max()) if p_ratio.size else 0.0,
                worst_cov=float(c_ratio.max()) if c_ratio.size else 0.0,
                worst_chi2=float(x_ratio.max()) if x_ratio.size else 0.0,
                bad_tracks=np.nonzero(m)[0][(~p_ok).any(1) | (~c_ok).any(1) | ~x_ok][:20],
                worst_cov_elem=int(np.argmax(c_ratio.max(0))) if c_ratio.size else -1)
