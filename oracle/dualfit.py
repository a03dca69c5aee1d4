"""Exact derivative of the fit's total chi2 by forward-mode dual numbers (test infrastructure).

The oracle's Kalman fit over a known assignment (orc_fit_batch in mkoracle.c: crossing, helix
step, Jacobian, transport J C J^T, Highland scattering and mean energy loss, chi2 and the
Joseph-form update), written again here on dual numbers: every quantity carries its value (FP64)
and its gradient with respect to the fit's parameters (the track's 6 starting parameters, and per
layer l the alignment (d_x, d_y, d_z, w_x, w_y, w_z) moving the layer's hits as
h' = h + d + w x (h - c_l), c_l the origin for a cylinder and (0, 0, z_l) for a disk, and the
thickness scale m_l multiplying x/X0).  The steps follow the C oracle one for one, so the value of
the total chi2 equals the C oracle's (a pin); the derivative is exact up to FP64 rounding:
  - the barrel crossing s* is found by the C oracle's bracketed Newton iteration on values only,
    then receives its derivative from the implicit function theorem through one final Newton step
    taken on dual numbers, ds*/dq = -(dg/dq) / (dg/ds) for the surface equation g(s, q) = 0;
  - branch decisions (which root, layer extent, incidence cap, charge sign) are taken on values.
Module planes are not covered (layers-only geometries).  Pure Python loops: small cases only.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 0.00299792458
M_PION = 0.13957039
M_ELEC = 0.51099895e-3
SI_K, SI_ZA, SI_RHO, SI_X0, SI_I = 0.307075, 0.49848, 2.329, 9.37, 173.0e-9
INC_CAP = 10.0
PI = math.pi


class D:
    """A dual number: value v and gradient g (numpy vector)."""
    __slots__ = ("v", "g")

    def __init__(self, v, g):
        self.v = float(v)
        self.g = g

    # arithmetic
    def __add__(self, o):
        if isinstance(o, D):
            return D(self.v + o.v, self.g + o.g)
        return D(self.v + o, self.g)

    __radd__ = __add__

    def __sub__(self, o):
        if isinstance(o, D):
            return D(self.v - o.v, self.g - o.g)
        return D(self.v - o, self.g)

    def __rsub__(self, o):
        return D(o - self.v, -self.g)

    def __neg__(self):
        return D(-self.v, -self.g)

    def __mul__(self, o):
        if isinstance(o, D):
            return D(self.v * o.v, self.g * o.v + o.g * self.v)
        return D(self.v * o, self.g * o)

    __rmul__ = __mul__

    def __truediv__(self, o):
        if isinstance(o, D):
            return D(self.v / o.v, (self.g * o.v - o.g * self.v) / (o.v * o.v))
        return D(self.v / o, self.g / o)

    def __rtruediv__(self, o):
        return D(o / self.v, -o * self.g / (self.v * self.v))


def const(v, k):
    return D(v, np.zeros(k))


def val(x):
    return x.v if isinstance(x, D) else float(x)


def sin(x):
    return D(math.sin(x.v), math.cos(x.v) * x.g)


def cos(x):
    return D(math.cos(x.v), -math.sin(x.v) * x.g)


def sqrt(x):
    r = math.sqrt(x.v)
    return D(r, x.g / (2.0 * r))


def log(x):
    return D(math.log(x.v), x.g / x.v)


def fabs(x):
    return x if x.v >= 0 else -x


def hypot(a, b):
    return sqrt(a * a + b * b)


def ix(i, j):
    return i * (i + 1) // 2 + j if i >= j else j * (j + 1) // 2 + i


def wrap_phi(a):
    w = a.v
    while w > PI:
        w -= 2 * PI
    while w <= -PI:
        w += 2 * PI
    return D(w, a.g)


# ---------------------------------------------------------------- helix and crossing

def s1c1(a):
    if abs(a.v) < 1e-8:
        return 1.0 - a * a / 6.0, 0.5 * a - a * a * a / 24.0
    h = sin(0.5 * a)
    return sin(a) / a, 2.0 * h * h / a


def s1c1_deriv(a):
    if abs(a.v) < 0.05:
        a2 = a * a
        dS1 = a * (-1.0 / 3.0 + a2 * (1.0 / 30.0 + a2 * (-1.0 / 840.0 + a2 * (1.0 / 45360.0 - a2 / 3991680.0))))
        dC1 = 0.5 + a2 * (-1.0 / 8.0 + a2 * (1.0 / 144.0 + a2 * (-1.0 / 5760.0 + a2 / 403200.0)))
        return dS1, dC1
    S1, C1 = s1c1(a)
    return (cos(a) - S1) / a, (sin(a) - C1) / a


def helix(bz, p, s):
    om = -C_LIGHT * bz * p[3]
    a = om * s
    S1, C1 = s1c1(a)
    cf, sf = cos(p[4]), sin(p[4])
    return [p[0] + s * (cf * S1 - sf * C1), p[1] + s * (sf * S1 + cf * C1), p[2] + s * cos(p[5]) / sin(p[5]),
            p[3], p[4] + a, p[5]]


def path_value(geom, layer, pv, bz):
    """The C oracle's crossing on values: (crossed, s)."""
    kind, R = int(geom.kind[layer]), float(geom.pos[layer])
    om = -C_LIGHT * bz * pv[3]
    if kind == 1:
        ct, st = math.cos(pv[5]), math.sin(pv[5])
        if abs(ct) < 1e-15:
            return False, 0.0
        s = (R - pv[2]) * st / ct
        if not s > 0:
            return False, 0.0
        if abs(om) >= 1e-14:
            sf, cf = math.sin(pv[4]), math.cos(pv[4])
            cx, cy = pv[0] - sf / om, pv[1] + cf / om
            d = math.hypot(cx, cy)
            sg = 1.0 if om > 0 else -1.0
            turn = math.fmod((math.atan2(sg * cx / d, -sg * cy / d) - pv[4]) * sg, 2 * PI)
            if turn < 0:
                turn += 2 * PI
            s_far = turn / abs(om)
            q = [x.v for x in helix(bz, [const(v, 1) for v in pv], const(s, 1))]
            vr = (q[0] * math.cos(q[4]) + q[1] * math.sin(q[4])) / max(math.hypot(q[0], q[1]), 1e-300)
            if s > s_far or vr < 0:
                return False, 0.0
    else:
        x, y, cf, sf = pv[0], pv[1], math.cos(pv[4]), math.sin(pv[4])
        if x * x + y * y >= R * R:
            return False, 0.0
        b, c = x * cf + y * sf, x * sf - y * cf
        s0 = -b + math.sqrt(R * R - c * c)
        if abs(om) < 1e-14:
            s = s0
        else:
            rho = 1.0 / abs(om)
            cx, cy = x - sf / om, y + cf / om
            d = math.hypot(cx, cy)
            if d + rho - R < 0:
                return False, 0.0
            sg = 1.0 if om > 0 else -1.0
            psi_far = math.atan2(sg * cx / d, -sg * cy / d)
            turn = math.fmod((psi_far - pv[4]) * sg, 2 * PI)
            if turn < 0:
                turn += 2 * PI
            lo, hi = 0.0, turn * rho
            s = s0 if lo < s0 < hi else 0.5 * (lo + hi)
            pc = [const(v, 1) for v in pv]
            for _ in range(300):
                q = [t.v for t in helix(bz, pc, const(s, 1))]
                gv = q[0] * q[0] + q[1] * q[1] - R * R
                if gv < 0:
                    lo = s
                else:
                    hi = s
                dg = 2.0 * (q[0] * math.cos(q[4]) + q[1] * math.sin(q[4]))
                sn = s - gv / dg if dg > 0 else 0.5 * (lo + hi)
                if not (lo < sn < hi):
                    sn = 0.5 * (lo + hi)
                ds = sn - s
                s = sn
                if abs(ds) < 1e-12 * R or hi - lo < 1e-13 * R:
                    break
    q = [t.v for t in helix(bz, [const(v, 1) for v in pv], const(s, 1))]
    v = q[2] if kind == 0 else math.hypot(q[0], q[1])
    return (geom.lo[layer] <= v <= geom.hi[layer]), s


def crossing(geom, layer, p, bz):
    """s* on dual numbers: the value from the C oracle's iteration, the derivative from the
    implicit function theorem (one Newton step on dual numbers at the converged value)."""
    ok, sv = path_value(geom, layer, [x.v for x in p], bz)
    if not ok:
        return None
    k = len(p[0].g)
    if int(geom.kind[layer]) == 1:
        return (float(geom.pos[layer]) - p[2]) * sin(p[5]) / cos(p[5])
    R = float(geom.pos[layer])
    s0 = const(sv, k)
    q = helix(bz, p, s0)
    gq = q[0] * q[0] + q[1] * q[1] - R * R          # g(s*, p): value ~0, gradient dg/dp
    dgds = 2.0 * (q[0].v * math.cos(q[4].v) + q[1].v * math.sin(q[4].v))
    return D(sv, -gq.g / dgds)


def jacobian(geom, layer, p, s, bz):
    cB = C_LIGHT * bz
    a = -cB * p[3] * s
    S1, C1 = s1c1(a)
    dS1, dC1 = s1c1_deriv(a)
    cf, sf, st = cos(p[4]), sin(p[4]), sin(p[5])
    k = len(p[0].g)
    A = [[const(1.0 if i == j else 0.0, k) for j in range(6)] for i in range(6)]
    dx, dy = s * (cf * S1 - sf * C1), s * (sf * S1 + cf * C1)
    A[0][3] = s * (cf * dS1 - sf * dC1) * (-cB * s)
    A[0][4] = -dy
    A[1][3] = s * (sf * dS1 + cf * dC1) * (-cB * s)
    A[1][4] = dx
    A[2][5] = -s / (st * st)
    A[4][3] = -cB * s
    q = helix(bz, p, s)
    om = -C_LIGHT * bz * p[3]
    dfds = [cos(q[4]), sin(q[4]), cos(q[5]) / sin(q[5]), const(0.0, k), om, const(0.0, k)]
    grad = [const(0.0, k)] * 6
    if int(geom.kind[layer]) == 0:
        grad = [2.0 * q[0], 2.0 * q[1]] + [const(0.0, k)] * 4
    else:
        grad = [const(0.0, k)] * 2 + [const(1.0, k)] + [const(0.0, k)] * 3
    gs = const(0.0, k)
    for i in range(6):
        gs = gs + grad[i] * dfds[i]
    J = [[None] * 6 for _ in range(6)]
    for j in range(6):
        gp = const(0.0, k)
        for i in range(6):
            gp = gp + grad[i] * A[i][j]
        for i in range(6):
            J[i][j] = A[i][j] - dfds[i] * gp / gs
    return J


def transport(J, C):
    M = [[C[ix(i, j)] for j in range(6)] for i in range(6)]
    T = [[sum((J[i][l] * M[l][j] for l in range(1, 6)), J[i][0] * M[0][j]) for j in range(6)] for i in range(6)]
    R = [[sum((T[i][l] * J[j][l] for l in range(1, 6)), T[i][0] * J[j][0]) for j in range(6)] for i in range(6)]
    return [R[i][j] for i in range(6) for j in range(i + 1)]


def theta0(pm, t):
    beta = pm / sqrt(pm * pm + M_PION * M_PION)
    return 0.0136 / (beta * pm) * sqrt(t) * (1.0 + 0.038 * log(t / (beta * beta)))


def eloss(pm, t):
    m = M_PION
    e = sqrt(pm * pm + m * m)
    bg2 = (pm / m) * (pm / m)
    b2 = bg2 / (1.0 + bg2)
    gam = e / m
    tmax = 2.0 * M_ELEC * bg2 / (1.0 + 2.0 * gam * M_ELEC / m + (M_ELEC / m) * (M_ELEC / m))
    dedx = SI_K * SI_ZA / b2 * (0.5 * log(2.0 * M_ELEC * bg2 * tmax / (SI_I * SI_I)) - b2)
    return dedx * SI_RHO * (t * SI_X0) * 1e-3


def material(geom, layer, p, C, xscale):
    st, ct = sin(p[5]), cos(p[5])
    ux, uy, uz = st * cos(p[4]), st * sin(p[4]), ct
    if int(geom.kind[layer]) == 0:
        r = hypot(p[0], p[1])
        cosi = fabs((p[0] * ux + p[1] * uy) / r)
    else:
        cosi = fabs(uz)
    fac = 1.0 / cosi if cosi.v * INC_CAP > 1.0 else INC_CAP
    t = xscale * float(geom.x_over_x0[layer]) * fac
    k = p[3]
    if not val(t) > 0 or k.v == 0.0:
        return True
    pm = 1.0 / (fabs(k) * st)
    th0 = theta0(pm, t)
    th02, cot = th0 * th0, ct / st
    C[ix(4, 4)] = C[ix(4, 4)] + th02 / (st * st)
    C[ix(5, 5)] = C[ix(5, 5)] + th02
    C[ix(3, 3)] = C[ix(3, 3)] + k * k * cot * cot * th02
    C[ix(5, 3)] = C[ix(5, 3)] + (-k) * cot * th02
    e = sqrt(pm * pm + M_PION * M_PION)
    e2 = e - eloss(pm, t)
    if not e2.v > M_PION:
        return False
    p2 = sqrt(e2 * e2 - M_PION * M_PION)
    a = pm / p2
    p[3] = k * a
    for j in range(6):
        if j != 3:
            C[ix(3, j)] = C[ix(3, j)] * a
    C[ix(3, 3)] = C[ix(3, 3)] * (a * a)
    return True


def chol3(S):
    if not S[0].v > 0:
        return None
    l00 = sqrt(S[0])
    l10, l20 = S[1] / l00, S[3] / l00
    d1 = S[2] - l10 * l10
    if not d1.v > 0:
        return None
    l11 = sqrt(d1)
    l21 = (S[4] - l20 * l10) / l11
    d2 = S[5] - l20 * l20 - l21 * l21
    if not d2.v > 0:
        return None
    return [l00, l10, l11, l20, l21, sqrt(d2)]


def update(p, C, m, V):
    """Joseph-form update and the predicted chi2, as orc_update (joseph = 1)."""
    S = [C[i] + V[i] for i in range(6)]
    Lc = chol3(S)
    if Lc is None:
        return None
    r = [m[0] - p[0], m[1] - p[1], m[2] - p[2]]
    y0 = r[0] / Lc[0]
    y1 = (r[1] - Lc[1] * y0) / Lc[2]
    y2 = (r[2] - Lc[3] * y0 - Lc[4] * y1) / Lc[5]
    chi2 = y0 * y0 + y1 * y1 + y2 * y2
    i00, i11, i22 = 1.0 / Lc[0], 1.0 / Lc[2], 1.0 / Lc[5]
    i10 = -Lc[1] * i00 * i11
    i21 = -Lc[4] * i11 * i22
    i20 = -(Lc[3] * i00 + Lc[4] * i10) * i22
    Mi = [[i00, None, None], [i10, i11, None], [i20, i21, i22]]
    Si = [[None] * 3 for _ in range(3)]
    for a in range(3):
        for b in range(3):
            acc = None
            for l in range(3):
                if Mi[l][a] is None or Mi[l][b] is None:
                    continue
                t = Mi[l][a] * Mi[l][b]
                acc = t if acc is None else acc + t
            Si[a][b] = acc
    B = [[C[ix(i, a)] for a in range(3)] for i in range(6)]
    K = [[B[i][0] * Si[0][a] + B[i][1] * Si[1][a] + B[i][2] * Si[2][a] for a in range(3)] for i in range(6)]
    pout = [p[i] + K[i][0] * r[0] + K[i][1] * r[1] + K[i][2] * r[2] for i in range(6)]
    k = len(p[0].g)
    A = [[const(1.0 if i == j else 0.0, k) for j in range(6)] for i in range(6)]
    for i in range(6):
        for a in range(3):
            A[i][a] = A[i][a] - K[i][a]
    M = [[C[ix(i, j)] for j in range(6)] for i in range(6)]
    Vf = [[V[ix(i, j)] for j in range(3)] for i in range(3)]
    T = [[sum((A[i][l] * M[l][j] for l in range(1, 6)), A[i][0] * M[0][j]) for j in range(6)] for i in range(6)]
    Cout = []
    for i in range(6):
        for j in range(i + 1):
            acc = sum((T[i][l] * A[j][l] for l in range(1, 6)), T[i][0] * A[j][0])
            for a in range(3):
                for b in range(3):
                    acc = acc + K[i][a] * Vf[a][b] * K[j][b]
            Cout.append(acc)
    pout[4] = wrap_phi(pout[4])
    if not (0.0 < pout[5].v < PI):
        return None
    return pout, Cout, chi2


def fit_track(geom, layers, hits, hit_xyz, hit_cov, p0, c0, align=None, xscale=None, material_on=True):
    """One track's fit on dual numbers.  Parameters (gradient components): [0, 6) the starting
    parameters, then per layer l in 0..L-1: 6 + 7 l + (0..5) its alignment, 6 + 7 l + 6 its
    thickness scale.  Returns (status, total chi2 as a dual number) with status as orc_fit_batch
    (0 ok, 1 a layer not crossed, 2 stopped, 3 update failed)."""
    L = int(geom.n_layers)
    K = 6 + 7 * L
    align = np.zeros((L, 6)) if align is None else np.asarray(align, np.float64)
    xscale = np.ones(L) if xscale is None else np.asarray(xscale, np.float64)
    eye = np.eye(K)
    p = [D(float(p0[i]), eye[i].copy()) for i in range(6)]
    C = [const(float(c0[i]), K) for i in range(21)]
    bz = float(geom.bz)
    total = const(0.0, K)
    for j, lay in enumerate(layers):
        lay = int(lay)
        if lay < 0:
            break
        s = crossing(geom, lay, p, bz)
        if s is None:
            return 1, total
        J = jacobian(geom, lay, p, s, bz)
        q = helix(bz, p, s)
        C = transport(J, C)
        if material_on:
            xs = D(float(xscale[lay]), eye[6 + 7 * lay + 6].copy())
            if not material(geom, lay, q, C, xs):
                return 2, total
        q[4] = wrap_phi(q[4])
        p = q
        h = int(hits[j])
        if h < 0:
            continue
        base = 6 + 7 * lay
        hx = np.asarray(hit_xyz[h], np.float64)
        c = np.array([0.0, 0.0, float(geom.pos[lay]) if int(geom.kind[lay]) == 1 else 0.0])
        rel = hx - c
        d, w = align[lay, :3], align[lay, 3:]
        mv = hx + d + np.cross(w, rel)
        m = []
        for a in range(3):
            g = np.zeros(K)
            g[base + a] = 1.0                       # d h'_a / d d_a
            # d (w x rel)_a / d w_b: (w x rel)_a = eps_abc w_b rel_c
            e = np.zeros(3)
            e[a] = 1.0
            g[base + 3: base + 6] = np.cross(rel, e)
            m.append(D(mv[a], g))
        V = [const(float(v), K) for v in hit_cov[h]]
        u = update(p, C, m, V)
        if u is None:
            return 3, total
        p, C, x2 = u
        total = total + x2
    return 0, total


def gradient(geom, layers, hits, hit_xyz, hit_cov, p0, c0, align=None, xscale=None, material_on=True):
    """All tracks: (chi2 per track, status, d/dp0 [n, 6], d/dalign [L, 6], d/dxscale [L]), the
    layer derivatives summed over the tracks with status 0 (the total chi2's), as
    oracle.gradient.fd_gradient returns them."""
    n = len(layers)
    L = int(geom.n_layers)
    chi2, status = np.zeros(n), np.zeros(n, np.int32)
    dp0, dal, dxs = np.zeros((n, 6)), np.zeros((L, 6)), np.zeros(L)
    X, V = np.asarray(hit_xyz, np.float64), np.asarray(hit_cov, np.float64)
    for i in range(n):
        st, tot = fit_track(geom, layers[i], hits[i], X, V, np.asarray(p0[i], np.float64),
                            np.asarray(c0[i], np.float64), align, xscale, material_on)
        status[i] = st
        if st != 0:
            continue
        chi2[i] = tot.v
        dp0[i] = tot.g[:6]
        gl = tot.g[6:].reshape(L, 7)
        dal += gl[:, :6]
        dxs += gl[:, 6]
    return chi2, status, dp0, dal, dxs
