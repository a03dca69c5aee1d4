"""Seeded synthetic tracker events: the shared input generator.

The paper's workloads (simulated ttbar events with pile-up in the CMS Phase-1 and
Phase-2 trackers, Sec. 2.3) are not available, so events are simulated here with
the shapes the method sees: tracks from the origin through barrel cylinders and
endcap disks in a uniform solenoid field, one Gaussian-smeared 3D hit per crossed
layer, multiple-scattering kicks and mean energy loss at each crossing, uniform
noise hits, and seeds made of the true hits on the first three crossed layers.

This module is test and benchmark input only.  It contains no step of the Kalman
filter: tracks are moved with the circle-centre description of a helix
(circle-circle intersection for cylinders), which is a different formulation
from the path-length form with Newton iteration that the filter uses, and all
random numbers are drawn here.  Both the CUDA path and the FP64 oracle consume
its arrays; it imports neither of them.

Units: cm, GeV, tesla, radians.  Packed 3x3 covariance order: xx, yx, yy, zx, zy, zz.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

BARREL = 0
DISK = 1

C_LIGHT = 0.00299792458      # curvature [1/cm] = C_LIGHT * B[T] / pT[GeV]
M_PION = 0.13957039          # GeV
M_ELECTRON = 0.51099895e-3   # GeV
# Silicon (PDG atomic and nuclear properties)
SI_K = 0.307075              # MeV cm^2 / mol
SI_Z_OVER_A = 0.49848
SI_RHO = 2.329               # g / cm^3
SI_X0 = 9.37                 # cm
SI_I = 173.0e-9              # GeV
INCIDENCE_CAP = 10.0


# --------------------------------------------------------------------------- geometry

@dataclass
class Geometry:
    """Layers (Sec. 3.1: an r-z bounding box that aggregates hits) and layer plans."""
    kind: np.ndarray          # int32 [L]: BARREL or DISK
    pos: np.ndarray           # float64 [L]: R (barrel) or z (disk)
    lo: np.ndarray            # barrel zmin / disk rmin
    hi: np.ndarray            # barrel zmax / disk rmax
    x_over_x0: np.ndarray     # thickness at normal incidence [X0]
    sig: np.ndarray           # float64 [L,3]: hit sigma along (r-hat, phi-hat, z-hat)
    n_eta: np.ndarray         # int32 [L] eta bins of the hit index
    n_phi: np.ndarray         # int32 [L] phi bins of the hit index
    eta_lo: np.ndarray        # float64 [L] eta range covered by the bins
    eta_hi: np.ndarray
    plans: list               # list of lists of layer indices, one per tracking region
    bz: float = 3.8
    barrel_eta_max: float = 1.0   # |eta_seed| below this -> region 0, else 1 (+z) / 2 (-z)
    modules: "Modules | None" = None   # flat modules of the modular layers (None: no module hits)

    @property
    def n_layers(self) -> int:
        return int(self.kind.shape[0])

    def plan_arrays(self):
        """Concatenated plans and their offsets (int32), the form the C interfaces take."""
        off = np.zeros(len(self.plans) + 1, np.int32)
        for i, pl in enumerate(self.plans):
            off[i + 1] = off[i] + len(pl)
        flat = np.concatenate([np.asarray(p, np.int32) for p in self.plans]).astype(np.int32)
        return flat, off

    @property
    def max_plan(self) -> int:
        return max(len(p) for p in self.plans)


@dataclass
class Modules:
    """Flat detector modules (Sec. 3.1: module position, normal and phi-direction vectors): the
    plane through c with unit normal n; u (the phi-direction) and v = n x u span it, the module
    covers |u.(x - c)| <= hw, |v.(x - c)| <= hl.  Per modular layer, modules form rings of
    n_phi staves (centres at phi = j 2pi/n_phi, radius alternating R +- dr so that neighbouring
    staves overlap in phi) at z centres z_k; rings beyond |z| > z_flat are tilted so that their
    normal points at the origin (the Phase-2 tilted barrel)."""
    c: np.ndarray        # float64 [M,3] (float32-representable)
    n: np.ndarray        # float64 [M,3]
    u: np.ndarray        # float64 [M,3]
    v: np.ndarray        # float64 [M,3]
    hw: np.ndarray       # float64 [M]
    hl: np.ndarray       # float64 [M]
    layer: np.ndarray    # int32 [M]
    grid: dict           # layer -> (first module, n_phi, z centres [K])


def _f32(v):
    """Values the C interface carries as float32, so that every consumer sees the same geometry."""
    return np.asarray(v, np.float32).astype(np.float64)


def _layer_table(rows, plans, bz=3.8, barrel_eta_max=1.0) -> Geometry:
    kind = np.array([r[0] for r in rows], np.int32)
    pos = _f32([r[1] for r in rows])
    lo = _f32([r[2] for r in rows])
    hi = _f32([r[3] for r in rows])
    xx0 = _f32([r[4] for r in rows])
    sig = _f32([r[5] for r in rows])
    n_eta = np.array([r[6] for r in rows], np.int32)
    n_phi = np.array([r[7] for r in rows], np.int32)
    eta_lo = np.empty(len(rows))
    eta_hi = np.empty(len(rows))
    for i in range(len(rows)):
        if kind[i] == BARREL:
            eta_lo[i] = np.arcsinh(lo[i] / pos[i])
            eta_hi[i] = np.arcsinh(hi[i] / pos[i])
        else:
            a = np.arcsinh(pos[i] / hi[i])
            b = np.arcsinh(pos[i] / lo[i])
            eta_lo[i], eta_hi[i] = min(a, b), max(a, b)
    return Geometry(kind, pos, lo, hi, xx0, sig, n_eta, n_phi, _f32(eta_lo), _f32(eta_hi),
                    [list(p) for p in plans], float(_f32(bz)), float(_f32(barrel_eta_max)))


SIG_BARREL = (30e-4, 30e-4, 100e-4)   # (r, r-phi, z): 30 um r-phi, 100 um z, 30 um along the normal
SIG_DISK = (100e-4, 30e-4, 30e-4)     # (r, r-phi, z): z is the disk normal


def barrel_radii(n=10, r0=4.0, r1=100.0):
    return [r0 + (r1 - r0) * i / (n - 1) for i in range(n)]


def disk_z(n=12, z0=125.0, z1=275.0):
    return [z0 + (z1 - z0) * j / (n - 1) for j in range(n)]


def _eta_bins(width, lo, hi):
    return max(8, int(np.ceil((hi - lo) / width)))


def add_modules(geom: Geometry, layers, dz=4.8, z_flat=30.0, width=9.0, dr=0.3, overlap=1.08,
                max_tilt_deg=80.0, sig_window=(0.5, 0.4, 0.5)) -> Geometry:
    """Makes the given barrel layers modular (Sec. 3.1 module vectors; the Phase-2 tilted barrel):
    each cylinder of radius R becomes rings of flat staves, and its hits lie on the module planes.
    The cylinder stays the layer's reference surface (window, material, binning); its window
    resolution becomes sig_window, the spread of module hits about the cylinder crossing."""
    cs, ns, us, vs, hws, hls, lay = [], [], [], [], [], [], []
    grid = {}
    sig = geom.sig.copy()
    for l in layers:
        assert geom.kind[l] == BARREL
        R, zmax = float(geom.pos[l]), float(geom.hi[l])
        nphi = int(np.ceil(2 * np.pi * R / width))
        nphi += nphi % 2
        K = int(np.floor(zmax / dz))
        zc = dz * np.arange(-K, K + 1)
        grid[l] = (len(cs), nphi, zc, "z")
        dphi = 2 * np.pi / nphi
        for k in zc:
            beta = np.arctan2(k, R) if abs(k) > z_flat else 0.0
            beta = float(np.clip(beta, -np.radians(max_tilt_deg), np.radians(max_tilt_deg)))
            for j in range(nphi):
                ph = j * dphi
                rj = R + (dr if j % 2 == 0 else -dr)
                rh = np.array([np.cos(ph), np.sin(ph), 0.0])
                u = np.array([-np.sin(ph), np.cos(ph), 0.0])
                n = np.cos(beta) * rh + np.array([0.0, 0.0, np.sin(beta)])
                v = np.cross(n, u)
                cs.append(rj * rh + np.array([0.0, 0.0, k]))
                ns.append(n); us.append(u); vs.append(v)
                hws.append(rj * np.tan(0.5 * dphi) * overlap)
                # a tilted ring faces the origin: its angular extent seen from there matches the
                # ring spacing (cos^2 beta dz / R) with 4% overlap
                hls.append(0.5 * dz * np.cos(beta) * 1.04 if beta != 0.0 else 0.5 * dz * 1.04)
                lay.append(l)
        sig[l] = sig_window
    return _with_modules(geom, cs, ns, us, vs, hws, hls, lay, grid, sig)


def _with_modules(geom, cs, ns, us, vs, hws, hls, lay, grid, sig):
    """geom with these modules added to those it has (module indices continue after them)."""
    f = lambda a: _f32(np.array(a))
    n = f(ns)
    n = n / np.linalg.norm(n, axis=1, keepdims=True)
    new = Modules(f(cs), n, np.array(us), np.array(vs), np.array(hws), np.array(hls), np.array(lay, np.int32), grid)
    old = geom.modules
    if old is not None:
        M = old.c.shape[0]
        new = Modules(np.concatenate([old.c, new.c]), np.concatenate([old.n, new.n]),
                      np.concatenate([old.u, new.u]), np.concatenate([old.v, new.v]),
                      np.concatenate([old.hw, new.hw]), np.concatenate([old.hl, new.hl]),
                      np.concatenate([old.layer, new.layer]),
                      {**old.grid, **{l: (e[0] + M,) + tuple(e[1:]) for l, e in grid.items()}})
    return Geometry(geom.kind, geom.pos, geom.lo, geom.hi, geom.x_over_x0, _f32(sig), geom.n_eta, geom.n_phi,
                    geom.eta_lo, geom.eta_hi, [list(p) for p in geom.plans], geom.bz, geom.barrel_eta_max, new)


def add_disk_modules(geom: Geometry, layers, n_rings=6, nphi=48, dz=0.2, overlap=1.08,
                     sig_window=(0.1, 0.1, 0.1)) -> Geometry:
    """Makes the given disks modular (Sec. 3.1 module vectors; the Phase-2 endcap's planar
    modules): each disk becomes n_rings rings of nphi flat modules facing along z, the rings
    equal in r, the modules alternating z_d +- dz so that neighbours overlap in phi (8%) and r
    (4%).  The disk stays the layer's reference surface; its window resolution becomes
    sig_window (a module hit lies on the track within dz of the disk crossing, so at nearly the
    crossing's eta and phi)."""
    cs, ns, us, vs, hws, hls, lay = [], [], [], [], [], [], []
    grid = {}
    sig = geom.sig.copy()
    for l in layers:
        assert geom.kind[l] == DISK
        zd, r0, r1 = float(geom.pos[l]), float(geom.lo[l]), float(geom.hi[l])
        dr = (r1 - r0) / n_rings
        rc = r0 + dr * (np.arange(n_rings) + 0.5)
        grid[l] = (len(cs), nphi, rc, "r")
        dphi = 2 * np.pi / nphi
        for k, rk in enumerate(rc):
            for j in range(nphi):
                ph = j * dphi
                rh = np.array([np.cos(ph), np.sin(ph), 0.0])
                u = np.array([-np.sin(ph), np.cos(ph), 0.0])
                n = np.array([0.0, 0.0, 1.0])
                cs.append(rk * rh + np.array([0.0, 0.0, zd + (dz if (j + k) % 2 == 0 else -dz)]))
                ns.append(n); us.append(u); vs.append(np.cross(n, u))
                hws.append(rk * np.tan(0.5 * dphi) * overlap)
                hls.append(0.5 * dr * 1.04)
                lay.append(l)
        sig[l] = sig_window
    return _with_modules(geom, cs, ns, us, vs, hws, hls, lay, grid, sig)


def geometry_phase2_modular_disks(**kw) -> Geometry:
    """geometry_phase2_modular with the 4th to 6th disk of each endcap (|z| = 166-193 cm) built
    from planar modules too."""
    g = geometry_phase2_modular(**kw)
    disks = [l for l in range(g.n_layers) if g.kind[l] == DISK]
    by_side = {s: sorted([l for l in disks if np.sign(g.pos[l]) == s], key=lambda l: abs(g.pos[l])) for s in (1, -1)}
    return add_disk_modules(g, by_side[1][3:6] + by_side[-1][3:6])


def geometry_phase2_modular(layers=(3, 4, 5), **kw) -> Geometry:
    """The Phase-2-like tracker with cylinders 3-5 (r = 36, 47, 57 cm) built from flat modules,
    flat for |z| <= 30 cm and tilted towards the origin beyond (Sec. 3.1: module position, normal
    and phi-direction; the Phase-2 tilted barrel).  The seeding cylinders 0-2 keep hits on their
    own surfaces."""
    return add_modules(geometry_phase2(**kw), layers)


def _module_crossings(mods: Modules, layer, x, y, z, psi, th, om):
    """Crossings of tracks at their cylinder crossing (x, y, z, direction psi, theta, curvature om)
    with the modules around that point: Newton in the transverse path sigma on
    n.(X(sigma) - c) = 0 along the circle-centre trajectory, kept if |sigma| < 10 cm and inside
    the module.  Returns per track up to two (module, sigma, point) in path order."""
    first, nphi, zc, coord = mods.grid[layer]
    dphi = 2 * np.pi / nphi
    j0 = np.round(np.mod(np.arctan2(y, x), 2 * np.pi) / dphi).astype(np.int64)
    w = z if coord == "z" else np.hypot(x, y)   # ring coordinate: z on a cylinder, r on a disk
    k0 = np.round((w - zc[0]) / (zc[1] - zc[0])).astype(np.int64)
    cand = []
    for dj in (-1, 0, 1):
        for dk in (-1, 0, 1):
            j = np.mod(j0 + dj, nphi)
            k = k0 + dk
            ok = (k >= 0) & (k < zc.size)
            m = np.where(ok, first + np.clip(k, 0, zc.size - 1) * nphi + j, -1)
            cand.append(m)
    cand = np.stack(cand, 1)                       # [T, 9]
    T = x.size
    sig = np.full(cand.shape, np.nan)
    pts = np.zeros(cand.shape + (3,))
    for q in range(cand.shape[1]):
        m = cand[:, q]
        val = m >= 0
        mm = np.where(val, m, 0)
        c, n = mods.c[mm], mods.n[mm]
        sg = np.zeros(T)
        for _ in range(8):
            xn, yn, zn, ps = _move(x, y, z, psi, th, om, sg)
            g = (xn - c[:, 0]) * n[:, 0] + (yn - c[:, 1]) * n[:, 1] + (zn - c[:, 2]) * n[:, 2]
            dg = np.cos(ps) * n[:, 0] + np.sin(ps) * n[:, 1] + n[:, 2] / np.tan(th)
            sg = sg - g / np.where(np.abs(dg) > 1e-6, dg, np.nan)
        xn, yn, zn, _ = _move(x, y, z, psi, th, om, sg)
        d = np.stack([xn, yn, zn], -1) - c
        a = np.einsum("ij,ij->i", d, mods.u[mm])
        b = np.einsum("ij,ij->i", d, mods.v[mm])
        inside = val & np.isfinite(sg) & (np.abs(sg) < 10.0) & (np.abs(a) <= mods.hw[mm]) & (np.abs(b) <= mods.hl[mm])
        sig[:, q] = np.where(inside, sg, np.nan)
        pts[:, q] = np.stack([xn, yn, zn], -1)
    order = np.argsort(np.where(np.isfinite(sig), sig, np.inf), axis=1)
    out = []
    for r in range(2):
        q = order[:, r]
        sr = sig[np.arange(T), q]
        mr = np.where(np.isfinite(sr), cand[np.arange(T), q], -1)
        out.append((mr, pts[np.arange(T), q]))
    return out


def _module_cov6(mods: Modules, m, sig):
    """Packed 3x3 covariance of hits on modules m with resolutions (normal, u, v) = sig."""
    n, u, v = mods.n[m], mods.u[m], mods.v[m]
    M = (sig[0] ** 2 * n[:, :, None] * n[:, None, :] + sig[1] ** 2 * u[:, :, None] * u[:, None, :]
         + sig[2] ** 2 * v[:, :, None] * v[:, None, :])
    return np.stack([M[:, 0, 0], M[:, 1, 0], M[:, 1, 1], M[:, 2, 0], M[:, 2, 1], M[:, 2, 2]], -1)


SIG_MODULE = (30e-4, 30e-4, 100e-4)   # (normal, phi-direction u, v): 30 um in u, 100 um in v


def geometry_barrel(n_layers=10, zmax=120.0, x_over_x0=0.02, n_eta=32, n_phi=128,
                    bz=3.8) -> Geometry:
    """Phase-1-like barrel: cylinders at r = 4..100 cm, |z| <= zmax; one region."""
    rows = [(BARREL, r, -zmax, zmax, x_over_x0, SIG_BARREL, n_eta, n_phi)
            for r in barrel_radii(n_layers)]
    return _layer_table(rows, [list(range(n_layers))], bz=bz, barrel_eta_max=1e9)


def geometry_phase2(x_over_x0=0.02, eta_bin=0.05, n_phi=256, sides=(+1, -1), bz=3.8,
                    barrel_eta_max=1.0) -> Geometry:
    """Phase-2-like tracker: 10 cylinders plus 12 disks per side covering |eta| < 3.

    Regions (layer plans): 0 barrel = cylinders; 1 endcap+ = cylinders then +z disks;
    2 endcap- = cylinders then -z disks.  With sides=(+1,) it is the 22-layer
    (10 barrel + 12 disk) single-endcap tracker with one plan.
    """
    zmax = 120.0
    rows = []
    for r in barrel_radii():
        e = np.arcsinh(zmax / r)
        rows.append((BARREL, r, -zmax, zmax, x_over_x0, SIG_BARREL,
                     _eta_bins(eta_bin, -e, e), n_phi))
    disk_first = {}
    for side in sides:
        disk_first[side] = len(rows)
        for zd in disk_z():
            rmin = zd / np.sinh(3.0)
            e0, e1 = np.arcsinh(zd / 100.0), np.arcsinh(zd / rmin)
            rows.append((DISK, side * zd, rmin, 100.0, x_over_x0, SIG_DISK,
                         _eta_bins(eta_bin, e0, e1), n_phi))
    cyl = list(range(10))
    if len(sides) == 1:
        plans = [cyl + list(range(disk_first[sides[0]], disk_first[sides[0]] + 12))]
        return _layer_table(rows, plans, bz=bz, barrel_eta_max=-1.0)
    plans = [cyl,
             cyl + list(range(disk_first[+1], disk_first[+1] + 12)),
             cyl + list(range(disk_first[-1], disk_first[-1] + 12))]
    return _layer_table(rows, plans, bz=bz, barrel_eta_max=barrel_eta_max)


# --------------------------------------------------------------------------- params

def default_params(**kw) -> dict:
    """Search parameters (Sec. 3.2 IterationParams / IterationLayerConfig), one set for all layers."""
    p = dict(chi2_cut=30.0, max_cands=6, max_holes=3, win_nsigma=3.5,
             deta_min=0.002, deta_max=0.1, dphi_min=0.002, dphi_max=0.1,
             score_hit=4.0, score_hole=8.0, material=1, precision=0, kappa_fp64=2.0 ** 24, fit_outlier_chi2=0.0,
             score_overlap=2.0)
    p.update(kw)
    return p


# --------------------------------------------------------------------------- physics of the simulated detector

def _bethe_bloch_loss(p, t):
    """Mean energy lost [GeV] by a pion of momentum p crossing t radiation lengths of silicon."""
    m = M_PION
    e = np.sqrt(p * p + m * m)
    bg2 = (p / m) ** 2
    b2 = bg2 / (1.0 + bg2)
    gam = e / m
    me = M_ELECTRON
    tmax = 2.0 * me * bg2 / (1.0 + 2.0 * gam * me / m + (me / m) ** 2)
    dedx = SI_K * SI_Z_OVER_A / b2 * (0.5 * np.log(2.0 * me * bg2 * tmax / (SI_I * SI_I)) - b2)
    return dedx * SI_RHO * (t * SI_X0) * 1e-3


def _highland(p, t):
    beta = p / np.sqrt(p * p + M_PION * M_PION)
    return 0.0136 / (beta * p) * np.sqrt(t) * (1.0 + 0.038 * np.log(t / (beta * beta)))


def _local_cov6(phi, sig):
    """3x3 covariance (packed) of a hit whose local axes are (r-hat, phi-hat, z-hat) at azimuth phi."""
    c, s = np.cos(phi), np.sin(phi)
    sr2, sp2, sz2 = (np.asarray(sig[..., 0]) ** 2, np.asarray(sig[..., 1]) ** 2,
                     np.asarray(sig[..., 2]) ** 2)
    out = np.zeros(np.broadcast(phi, sr2).shape + (6,))
    out[..., 0] = sr2 * c * c + sp2 * s * s
    out[..., 1] = (sr2 - sp2) * c * s
    out[..., 2] = sr2 * s * s + sp2 * c * c
    out[..., 5] = sz2
    return out


def _smear(x, y, z, sig, rng):
    phi = np.arctan2(y, x)
    g = rng.standard_normal((3,) + np.shape(x))
    dr, dp, dz = g[0] * sig[..., 0], g[1] * sig[..., 1], g[2] * sig[..., 2]
    c, s = np.cos(phi), np.sin(phi)
    return x + dr * c - dp * s, y + dr * s + dp * c, z + dz


class _Tracks:
    """Vectorised truth state: position, transverse direction phi, polar angle, |p|, charge."""

    def __init__(self, q, pt, eta, phi, x=None, y=None, z=None):
        n = q.shape[0]
        self.q = q.astype(np.float64)
        self.theta = 2.0 * np.arctan(np.exp(-eta))
        self.p = pt / np.sin(self.theta)
        self.phi = phi.astype(np.float64)
        self.x = np.zeros(n) if x is None else x
        self.y = np.zeros(n) if y is None else y
        self.z = np.zeros(n) if z is None else z

    def omega(self, bz, idx):
        pt = self.p[idx] * np.sin(self.theta[idx])
        return -self.q[idx] * C_LIGHT * bz / pt


def _cylinder_crossing(x, y, phi, om, R):
    """First positive transverse path to radius R along circles given by centre (returns nan if none)."""
    n = x.shape[0]
    s_out = np.full(n, np.nan)
    straight = np.abs(om) < 1e-15
    if np.any(straight):
        i = straight
        b = x[i] * np.cos(phi[i]) + y[i] * np.sin(phi[i])
        d2 = R * R - (x[i] * np.sin(phi[i]) - y[i] * np.cos(phi[i])) ** 2
        s = -b + np.sqrt(np.maximum(d2, 0.0))
        s_out[i] = np.where((d2 >= 0) & (s > 0), s, np.nan)
    i = ~straight
    if np.any(i):
        w = om[i]
        cx = x[i] - np.sin(phi[i]) / w
        cy = y[i] + np.cos(phi[i]) / w
        rho = 1.0 / np.abs(w)
        d = np.hypot(cx, cy)
        ok = (d > 0) & (np.abs(d - rho) <= R) & (R <= d + rho)
        dd = np.where(d > 0, d, 1.0)
        a = (rho * rho - R * R + dd * dd) / (2.0 * dd)
        h = np.sqrt(np.maximum(rho * rho - a * a, 0.0))
        ex, ey = -cx / dd, -cy / dd
        best = np.full(w.shape, np.inf)
        for sgn in (+1.0, -1.0):
            px = cx + a * ex - sgn * h * ey
            py = cy + a * ey + sgn * h * ex
            psi = np.arctan2(w * (px - cx), -w * (py - cy))
            turn = np.mod((psi - phi[i]) * np.sign(w), 2.0 * np.pi)
            s = turn * rho
            s = np.where(s > 1e-9, s, np.inf)
            best = np.minimum(best, s)
        best = np.where(ok & np.isfinite(best), best, np.nan)
        s_out[i] = best
    return s_out


def _path_to_apex(x, y, phi, om):
    """Transverse path to the track circle's point farthest from the z axis (inf if straight)."""
    straight = np.abs(om) < 1e-15
    w = np.where(straight, 1.0, om)
    cx = x - np.sin(phi) / w
    cy = y + np.cos(phi) / w
    sg = np.sign(w)
    psi_far = np.arctan2(sg * cx, -sg * cy)
    turn = np.mod((psi_far - phi) * sg, 2.0 * np.pi)
    return np.where(straight, np.inf, turn / np.abs(w))


def _move(x, y, z, phi, theta, om, s):
    """Position and direction after transverse path s (circle-centre form)."""
    straight = np.abs(om) < 1e-15
    w = np.where(straight, 1.0, om)
    cx = x - np.sin(phi) / w
    cy = y + np.cos(phi) / w
    psi = phi + om * s
    xn = np.where(straight, x + s * np.cos(phi), cx + np.sin(psi) / w)
    yn = np.where(straight, y + s * np.sin(phi), cy - np.cos(psi) / w)
    zn = z + s / np.tan(theta)
    return xn, yn, zn, psi


# --------------------------------------------------------------------------- events

@dataclass
class Event:
    """One event's hits grouped by layer, truth, and seeds (event-local hit indices)."""
    hit_xyz: np.ndarray        # float32 [H,3]
    hit_cov: np.ndarray        # float32 [H,6]
    layer_off: np.ndarray      # int64 [L+1]
    hit_track: np.ndarray      # int32 [H], -1 for noise
    track_q: np.ndarray
    track_pt: np.ndarray
    track_eta: np.ndarray
    track_phi: np.ndarray
    track_hits: np.ndarray     # int32 [T, maxh] local hit indices in crossing order, -1 padded
    track_layers: np.ndarray   # int32 [T, maxh]
    track_truth: np.ndarray    # float64 [T, maxh, 6] state (x,y,z,q/pT,phi,theta) leaving each hit's layer
    seed_hits: np.ndarray      # int32 [S,3]
    seed_track: np.ndarray     # int32 [S]
    hit_mod: np.ndarray = None     # int32 [H]: module of each hit, -1 on a layer's own surface
    track_ovl: np.ndarray = None   # int32 [T, maxh]: second hit (an overlapping module) on that layer, -1

    @property
    def n_hits(self):
        return int(self.hit_xyz.shape[0])


def _traversal(geom: Geometry, side: int):
    cyl = sorted([i for i in range(geom.n_layers) if geom.kind[i] == BARREL], key=lambda i: geom.pos[i])
    dsk = sorted([i for i in range(geom.n_layers) if geom.kind[i] == DISK and np.sign(geom.pos[i]) == side],
                 key=lambda i: abs(geom.pos[i]))
    return cyl + dsk


def sample_pt_loguniform(rng, n, lo, hi):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n))


def sample_pt_phase2(rng, n, frac_low=0.7):
    """70% log-uniform in [0.5, 2] GeV, the rest log-uniform in [2, 50] GeV."""
    low = rng.random(n) < frac_low
    return np.where(low, sample_pt_loguniform(rng, n, 0.5, 2.0), sample_pt_loguniform(rng, n, 2.0, 50.0))


def sample_pt_loopers(rng, n, frac_loop=0.1):
    """A fraction frac_loop uniform in [0.5, 0.7] GeV (tracks that curl inside the tracker at
    3.8 T), the rest as sample_pt_phase2."""
    loop = rng.random(n) < frac_loop
    return np.where(loop, rng.uniform(0.5, 0.7, n), sample_pt_phase2(rng, n))


def simulate_event(geom: Geometry, n_tracks: int, seed: int = 0, event: int = 0, *,
                   pt_sampler=None, eta_max=1.0, eta_min=None, noise_per_layer=None,
                   noise_total=None, material=True, smear=True, min_hits_seed=3) -> Event:
    """Simulate one event.  Random streams depend only on (seed, event)."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, event])))
    L = geom.n_layers
    q = rng.choice(np.array([-1.0, 1.0]), n_tracks)
    pt = (pt_sampler(rng, n_tracks) if pt_sampler is not None
          else sample_pt_loguniform(rng, n_tracks, 0.5, 10.0))
    lo_eta = -eta_max if eta_min is None else eta_min
    eta = rng.uniform(lo_eta, eta_max, n_tracks)
    phi0 = rng.uniform(-np.pi, np.pi, n_tracks)
    trk = _Tracks(q, pt, eta, phi0)
    plus = _traversal(geom, +1)
    minus = _traversal(geom, -1)
    nstep = max(len(plus), len(minus))
    side_plus = trk.theta < 0.5 * np.pi

    maxh = nstep
    t_layers = np.full((n_tracks, maxh), -1, np.int32)
    t_truth = np.zeros((n_tracks, maxh, 6))
    t_xyz = np.zeros((n_tracks, maxh, 3))
    t_mod = np.full((n_tracks, maxh), -1, np.int64)
    t_oxyz = np.zeros((n_tracks, maxh, 3))
    t_omod = np.full((n_tracks, maxh), -1, np.int64)
    mods = geom.modules
    nh = np.zeros(n_tracks, np.int32)
    alive = np.ones(n_tracks, bool)

    for j in range(nstep):
        for side_mask, trav in ((side_plus, plus), (~side_plus, minus)):
            if j >= len(trav):
                continue
            lay = trav[j]
            idx = np.nonzero(side_mask & alive)[0]
            if idx.size == 0:
                continue
            om = trk.omega(geom.bz, idx)
            x, y, z, ph, th = trk.x[idx], trk.y[idx], trk.z[idx], trk.phi[idx], trk.theta[idx]
            if geom.kind[lay] == BARREL:
                s = _cylinder_crossing(x, y, ph, om, geom.pos[lay])
            else:
                s = (geom.pos[lay] - z) * np.tan(th)
                # a curling track is followed only up to its point of largest radius: a disk it
                # would reach later ends the track
                past = np.isfinite(s) & (s > 0) & (s > _path_to_apex(x, y, ph, om))
                alive[idx[past]] = False
                s = np.where((s > 0) & ~past, s, np.nan)
            ok = np.isfinite(s)
            s = np.where(ok, s, 0.0)
            xn, yn, zn, psi = _move(x, y, z, ph, th, om, s)
            if geom.kind[lay] == BARREL:
                ok &= (zn >= geom.lo[lay]) & (zn <= geom.hi[lay])
            else:
                rn = np.hypot(xn, yn)
                ok &= (rn >= geom.lo[lay]) & (rn <= geom.hi[lay])
            sel = idx[ok]
            if sel.size == 0:
                continue
            xn, yn, zn, psi = xn[ok], yn[ok], zn[ok], psi[ok]
            th = th[ok]
            hit = np.ones(sel.size, bool)
            if mods is not None and lay in mods.grid:
                # the hits lie where the track crosses the modules around its cylinder crossing
                (m1, x1), (m2, x2) = _module_crossings(mods, lay, xn, yn, zn, psi, th, om[ok])
                hit = m1 >= 0
                k = nh[sel[hit]]
                t_mod[sel[hit], k] = m1[hit]
                t_omod[sel[hit], k] = m2[hit]
                t_oxyz[sel[hit], k] = x2[hit]
            selh = sel[hit]
            k = nh[selh]
            t_layers[selh, k] = lay
            t_xyz[selh, k] = x1[hit] if (mods is not None and lay in mods.grid) else np.stack([xn, yn, zn], -1)
            # material: Highland kick at fixed |p|, then mean energy loss
            p = trk.p[sel]
            if material and geom.x_over_x0[lay] > 0:
                ux, uy, uz = np.sin(th) * np.cos(psi), np.sin(th) * np.sin(psi), np.cos(th)
                if geom.kind[lay] == BARREL:
                    rr = np.hypot(xn, yn)
                    cosi = np.abs((xn * ux + yn * uy) / rr)
                else:
                    cosi = np.abs(uz)
                t = geom.x_over_x0[lay] * np.minimum(1.0 / np.maximum(cosi, 1e-300), INCIDENCE_CAP)
                th0 = _highland(p, t)
                g = rng.standard_normal((2, sel.size))
                th_new = th + th0 * g[0]
                psi = psi + th0 * g[1] / np.sin(th)
                th = np.clip(th_new, 1e-6, np.pi - 1e-6)
                e = np.sqrt(p * p + M_PION ** 2) - _bethe_bloch_loss(p, t)
                p = np.sqrt(np.maximum(e * e - M_PION ** 2, 1e-12))
            psi = np.mod(psi + np.pi, 2.0 * np.pi) - np.pi
            trk.x[sel], trk.y[sel], trk.z[sel] = xn, yn, zn
            trk.phi[sel], trk.theta[sel], trk.p[sel] = psi, th, p
            t_truth[selh, k] = np.stack([xn, yn, zn, trk.q[sel] / (p * np.sin(th)), psi, th], -1)[hit]
            nh[selh] += 1

    # assemble hits per layer: signal + noise, shuffled within the layer
    if noise_total is not None:
        area = np.where(geom.kind == BARREL, 2 * np.pi * np.abs(geom.pos) * (geom.hi - geom.lo),
                        np.pi * (geom.hi ** 2 - geom.lo ** 2))
        n_noise = np.floor(noise_total * area / area.sum()).astype(np.int64)
        n_noise[: int(noise_total - n_noise.sum())] += 1
    else:
        n_noise = np.full(L, 0 if noise_per_layer is None else int(noise_per_layer), np.int64)

    xyz_parts, cov_parts, trk_parts, mod_parts = [], [], [], []
    local_of = np.full((n_tracks, maxh), -1, np.int64)
    local_ovl = np.full((n_tracks, maxh), -1, np.int64)
    layer_off = np.zeros(L + 1, np.int64)
    for lay in range(L):
        ti, ki = np.nonzero(t_layers == lay)
        nn = int(n_noise[lay])
        if mods is not None and lay in mods.grid:
            # primary and overlap hits on their modules, noise uniform over the layer's modules
            oi, ok_ = np.nonzero((t_layers == lay) & (t_omod >= 0))
            first, nphi, zc, _ = mods.grid[lay]
            nm = rng.integers(first, first + nphi * zc.size, nn)
            ab = rng.uniform(-1.0, 1.0, (2, nn))
            npos = mods.c[nm] + (ab[0] * mods.hw[nm])[:, None] * mods.u[nm] + (ab[1] * mods.hl[nm])[:, None] * mods.v[nm]
            pos = np.concatenate([t_xyz[ti, ki], t_oxyz[oi, ok_], npos])
            mid = np.concatenate([t_mod[ti, ki], t_omod[oi, ok_], nm]).astype(np.int64)
            owner = np.concatenate([ti, oi, np.full(nn, -1)]).astype(np.int32)
            if smear:
                g = rng.standard_normal((3, mid.size))
                pos = pos + sum((g[a] * SIG_MODULE[a])[:, None] * (mods.n, mods.u, mods.v)[a][mid] for a in range(3))
            perm = rng.permutation(mid.size)
            pos, mid, owner = pos[perm], mid[perm], owner[perm]
            inv = np.empty_like(perm)
            inv[perm] = np.arange(perm.size)
            base = layer_off[lay]
            local_of[ti, ki] = base + inv[: ti.size]
            local_ovl[oi, ok_] = base + inv[ti.size: ti.size + oi.size]
            xyz_parts.append(pos)
            cov_parts.append(_module_cov6(mods, mid, SIG_MODULE))
            trk_parts.append(owner)
            mod_parts.append(mid)
            layer_off[lay + 1] = base + mid.size
            continue
        sx, sy, sz = t_xyz[ti, ki, 0], t_xyz[ti, ki, 1], t_xyz[ti, ki, 2]
        u = rng.random((2, nn))
        nphi = -np.pi + 2 * np.pi * u[0]
        if geom.kind[lay] == BARREL:
            r = np.full(nn, geom.pos[lay])
            nz = geom.lo[lay] + (geom.hi[lay] - geom.lo[lay]) * u[1]
        else:
            r = np.sqrt(geom.lo[lay] ** 2 + (geom.hi[lay] ** 2 - geom.lo[lay] ** 2) * u[1])
            nz = np.full(nn, geom.pos[lay])
        ax = np.concatenate([sx, r * np.cos(nphi)])
        ay = np.concatenate([sy, r * np.sin(nphi)])
        az = np.concatenate([sz, nz])
        owner = np.concatenate([ti, np.full(nn, -1)]).astype(np.int32)
        sig = np.broadcast_to(geom.sig[lay], (ax.size, 3))
        if smear:
            ax, ay, az = _smear(ax, ay, az, sig, rng)
        perm = rng.permutation(ax.size)
        ax, ay, az, owner = ax[perm], ay[perm], az[perm], owner[perm]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        base = layer_off[lay]
        local_of[ti, ki] = base + inv[: ti.size]
        cov = _local_cov6(np.arctan2(ay, ax), np.broadcast_to(geom.sig[lay], (ax.size, 3)))
        xyz_parts.append(np.stack([ax, ay, az], -1))
        cov_parts.append(cov)
        trk_parts.append(owner)
        mod_parts.append(np.full(ax.size, -1, np.int64))
        layer_off[lay + 1] = base + ax.size

    hit_xyz = np.concatenate(xyz_parts).astype(np.float32) if xyz_parts else np.zeros((0, 3), np.float32)
    hit_cov = np.concatenate(cov_parts).astype(np.float32) if cov_parts else np.zeros((0, 6), np.float32)
    hit_track = np.concatenate(trk_parts).astype(np.int32) if trk_parts else np.zeros(0, np.int32)
    track_hits = np.where(t_layers >= 0, local_of, -1).astype(np.int32)
    has_seed = nh >= min_hits_seed
    seed_track = np.nonzero(has_seed)[0].astype(np.int32)
    seed_hits = track_hits[seed_track, :3].astype(np.int32)
    hit_mod = np.concatenate(mod_parts).astype(np.int32) if mod_parts else np.zeros(0, np.int32)
    return Event(hit_xyz, hit_cov, layer_off, hit_track, q, pt, eta, phi0,
                 track_hits, t_layers, t_truth, seed_hits, seed_track, hit_mod,
                 np.where(t_layers >= 0, local_ovl, -1).astype(np.int32))


@dataclass
class Batch:
    """Several events concatenated: global hit index = hit_off[e*L] + event-local index."""
    n_events: int
    n_layers: int
    hit_xyz: np.ndarray
    hit_cov: np.ndarray
    hit_off: np.ndarray        # int64 [E*L+1]
    hit_track: np.ndarray
    seed_hits: np.ndarray      # int32 [S,3] global hit indices
    seed_event: np.ndarray     # int32 [S]
    seed_track: np.ndarray     # int32 [S] event-local track index
    events: list = field(default_factory=list)
    hit_mod: np.ndarray = None # int32 [H]: module of each hit, -1 on a layer's own surface


def concat_events(events, n_layers) -> Batch:
    offs = [0]
    for ev in events:
        offs.append(offs[-1] + ev.n_hits)
    hit_off = np.concatenate([[0]] + [offs[e] + ev.layer_off[1:] for e, ev in enumerate(events)]).astype(np.int64)
    seeds = [ev.seed_hits + offs[e] for e, ev in enumerate(events)]
    return Batch(len(events), n_layers,
                 np.concatenate([ev.hit_xyz for ev in events]),
                 np.concatenate([ev.hit_cov for ev in events]),
                 hit_off,
                 np.concatenate([ev.hit_track for ev in events]),
                 np.concatenate(seeds).astype(np.int32) if seeds else np.zeros((0, 3), np.int32),
                 np.concatenate([np.full(ev.seed_hits.shape[0], e, np.int32) for e, ev in enumerate(events)]),
                 np.concatenate([ev.seed_track for ev in events]).astype(np.int32),
                 list(events),
                 np.concatenate([ev.hit_mod for ev in events]).astype(np.int32))


def fit_workload(ev: Event, seed: int = 0, *, sig_pos=0.005, sig_z=0.01, rel_k=0.05,
                 sig_ang=0.002, min_hits=1, event_offset=0):
    """Tracks with their true hit assignment and a starting state drawn around the truth at the origin.

    Returns (layers [T,maxh] int32 (-1 end), hits [T,maxh] int32 global indices, p0 [T,6], c0 [T,21],
    truth_last [T,6], n_hits [T]).  p0 ~ N(truth at vertex, C0) so that a consistent fit has unit pulls.
    """
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 7919])))
    nh = (ev.track_layers >= 0).sum(1)
    sel = np.nonzero(nh >= min_hits)[0]
    T = sel.size
    theta = 2.0 * np.arctan(np.exp(-ev.track_eta[sel]))
    k = ev.track_q[sel] / ev.track_pt[sel]
    truth0 = np.stack([np.zeros(T), np.zeros(T), np.zeros(T), k, ev.track_phi[sel], theta], -1)
    sig = np.stack([np.full(T, sig_pos), np.full(T, sig_pos), np.full(T, sig_z),
                    rel_k * np.abs(k), np.full(T, sig_ang), np.full(T, sig_ang)], -1)
    p0 = truth0 + sig * rng.standard_normal((T, 6))
    c0 = np.zeros((T, 21))
    for i in range(6):
        c0[:, i * (i + 1) // 2 + i] = sig[:, i] ** 2
    layers = ev.track_layers[sel].copy()
    hits = np.where(ev.track_hits[sel] >= 0, ev.track_hits[sel] + event_offset, -1).astype(np.int32)
    last = nh[sel] - 1
    truth_last = ev.track_truth[sel, last]
    return layers, hits, p0, c0, truth_last, nh[sel].astype(np.int32), sel


def workload_small_barrel(seed=0):
    """1,000 tracks through 10 barrel cylinders, pT log-uniform 0.5-10 GeV, |eta| < 1,
    2% X0 per layer, 200 uniform noise hits per layer."""
    g = geometry_barrel()
    ev = simulate_event(g, 1000, seed, 0, eta_max=1.0, noise_per_layer=200)
    return g, ev


def workload_phase2(n_events=64, n_tracks=20000, seed=0, noise_total=50000):
    """Phase-2-like events: 10 cylinders + 2x12 disks, |eta| < 3, pT 0.5-50 GeV (70% below 2)."""
    g = geometry_phase2()
    evs = [simulate_event(g, n_tracks, seed, e, pt_sampler=sample_pt_phase2, eta_max=3.0,
                          noise_total=noise_total) for e in range(n_events)]
    return g, evs


def uneven_counts(n_events=256, mean=8000, lo=200, hi=25000, seed=0):
    """Poisson track counts of the uneven-batch workload, clipped to [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 104729])))
    return np.clip(rng.poisson(mean, n_events), lo, hi)


def _uneven_event(args):
    n, seed, e, noise_per_track = args
    return simulate_event(geometry_phase2(), int(n), seed, e, pt_sampler=sample_pt_phase2, eta_max=3.0,
                          noise_total=int(noise_per_track * n))


def workload_uneven(n_events=256, mean=8000, lo=200, hi=25000, seed=0, noise_per_track=2.5, counts=None,
                    processes=None):
    """Events with Poisson track counts (clipped to [lo, hi]; or the given counts) on the
    Phase-2-like geometry, noise in proportion to the tracks (50,000 per 20,000 tracks).
    processes > 1: the events are simulated in a spawn pool of that many processes (the same
    events: each depends only on (seed, event))."""
    g = geometry_phase2()
    if counts is None:
        counts = uneven_counts(n_events, mean, lo, hi, seed)
    jobs = [(int(n), seed, e, noise_per_track) for e, n in enumerate(counts)]
    if processes and processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            evs = pool.map(_uneven_event, jobs)
    else:
        evs = [_uneven_event(j) for j in jobs]
    return g, evs


def workload_loopers(n_events=50, n_tracks=20000, seed=0):
    """Phase-2-like events with 10% of the tracks at 0.5-0.7 GeV (curling, ill-conditioned S)."""
    g = geometry_phase2()
    evs = [simulate_event(g, n_tracks, seed, e, pt_sampler=sample_pt_loopers, eta_max=3.0, noise_total=0)
           for e in range(n_events)]
    return g, evs


def move_hits(geom: Geometry, ev: Event, align) -> Event:
    """The event with the hits of every layer l moved by align[l] = (d, w): h' = h + d + w x (h - c_l),
    c_l the origin for a cylinder and (0, 0, z_l) for a disk; covariances unchanged."""
    import dataclasses
    X = ev.hit_xyz.astype(np.float64)
    for l in range(geom.n_layers):
        a, b = int(ev.layer_off[l]), int(ev.layer_off[l + 1])
        if a == b:
            continue
        c = np.array([0.0, 0.0, float(geom.pos[l]) if geom.kind[l] == DISK else 0.0])
        X[a:b] = X[a:b] + align[l, :3] + np.cross(align[l, 3:], X[a:b] - c)
    return dataclasses.replace(ev, hit_xyz=X.astype(np.float32))


def workload_aligned_fit(n_tracks=100_000, seed=0, sig_shift=50e-4, sig_rot=1e-4, mat_frac=0.2,
                         tracks_per_event=20_000):
    """Known-assignment fit workload with a misaligned detector: tracks with eta in [0, 3) cross
    the 10 cylinders and the 12 disks at +z (22 layers); each layer carries a random alignment
    (shifts of sigma 50 um, rotations of sigma 0.1 mrad) and a material thickness off by a
    uniform factor in [0.8, 1.2].  Hits are simulated through the true material and moved by
    the true alignment; the fit uses the nominal geometry.  Returns (nominal geometry, events,
    true alignment [L, 6], true thickness scales [L])."""
    import dataclasses
    g = geometry_phase2()
    L = g.n_layers
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, 15485863])))
    align = np.zeros((L, 6))
    align[:, :3] = rng.normal(0.0, sig_shift, (L, 3))
    align[:, 3:] = rng.normal(0.0, sig_rot, (L, 3))
    xscale = rng.uniform(1.0 - mat_frac, 1.0 + mat_frac, L)
    g_true = dataclasses.replace(g, x_over_x0=_f32(g.x_over_x0 * xscale))
    evs = []
    for e in range(int(np.ceil(n_tracks / tracks_per_event))):
        nt = min(tracks_per_event, n_tracks - e * tracks_per_event)
        ev = simulate_event(g_true, nt, seed, e, pt_sampler=sample_pt_phase2, eta_min=0.0, eta_max=3.0,
                            noise_total=0)
        evs.append(move_hits(g, ev, align))
    return g, evs, align, xscale
