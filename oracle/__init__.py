"""FP64 CPU oracle (ctypes wrapper around mkoracle.c).

TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the CPU-baseline legs of
bench.py may import this package.  It shares no code with the CUDA library and never
imports it.  Each wrapper names the step of the method it computes; the C source states
the formula.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mkoracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MISS, SKIP, STOP, PRE = -1, -2, -3, -4


def build(force: bool = False) -> str:
    """Compile the oracle with plain ISO C flags (no fused multiply-add contraction, no
    machine-specific code) so results agree between x86-64 and aarch64 hosts."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "mkoracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_eta", C.c_int), ("n_phi", C.c_int), ("pad", C.c_int),
                ("pos", C.c_double), ("lo", C.c_double), ("hi", C.c_double), ("x_over_x0", C.c_double),
                ("sig", C.c_double * 3), ("eta_lo", C.c_double), ("eta_hi", C.c_double)]


class Modules(C.Structure):
    _fields_ = [("n", C.c_int), ("c", C.POINTER(C.c_double)), ("nrm", C.POINTER(C.c_double)),
                ("hit_mod", C.POINTER(C.c_int))]


class Geom(C.Structure):
    _fields_ = [("bz", C.c_double), ("barrel_eta_max", C.c_double), ("n_layers", C.c_int),
                ("n_regions", C.c_int), ("layers", C.POINTER(Layer)), ("plan", C.POINTER(C.c_int)),
                ("plan_off", C.POINTER(C.c_int)), ("mods", C.POINTER(Modules))]


class Params(C.Structure):
    _fields_ = [("chi2_cut", C.c_double), ("win_nsigma", C.c_double), ("deta_min", C.c_double),
                ("deta_max", C.c_double), ("dphi_min", C.c_double), ("dphi_max", C.c_double),
                ("score_hit", C.c_double), ("score_hole", C.c_double), ("max_cands", C.c_int),
                ("max_holes", C.c_int), ("material", C.c_int), ("binned", C.c_int),
                ("score_overlap", C.c_double)]


class Tie(C.Structure):
    _fields_ = [("chi2_rel", C.c_double), ("win_abs", C.c_double), ("win_rel", C.c_double),
                ("score_abs", C.c_double), ("score_rel", C.c_double), ("edge_rel", C.c_double),
                ("kappa", C.c_double)]


class BuildOut(C.Structure):
    _fields_ = [("params", C.POINTER(C.c_double)), ("cov", C.POINTER(C.c_double)),
                ("score", C.POINTER(C.c_double)), ("chi2", C.POINTER(C.c_double)),
                ("nfound", C.POINTER(C.c_int)), ("nholes", C.POINTER(C.c_int)),
                ("hits", C.POINTER(C.c_int)), ("max_plan", C.c_int), ("tie_step", C.POINTER(C.c_int)),
                ("region", C.POINTER(C.c_int)), ("start", C.POINTER(C.c_int)),
                ("counters", C.POINTER(C.c_longlong)), ("ovl", C.POINTER(C.c_int))]


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


def lib():
    """The oracle library.  MKORACLE_LIB may name another build of the same source (the
    mutation test uses it to load copies with planted mistakes)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(os.environ.get("MKORACLE_LIB") or build())
            d, i = C.POINTER(C.c_double), C.POINTER(C.c_int)
            _lib.orc_path.restype = C.c_int
            _lib.orc_propagate.restype = C.c_int
            _lib.orc_path_inward.restype = C.c_int
            _lib.orc_propagate_backward.restype = C.c_int
            _lib.orc_chi2.restype = C.c_int
            _lib.orc_update.restype = C.c_int
            _lib.orc_seed.restype = C.c_int
            _lib.orc_material.restype = C.c_int
            _lib.orc_eloss.restype = C.c_double
            _lib.orc_eloss.argtypes = [C.c_double, C.c_double]
            _lib.orc_ms_theta0.argtypes = [C.c_double, C.c_double, d]
            _lib.orc_helix.argtypes = [C.c_double, d, C.c_double, d]
            _lib.orc_jacobian_fixed_s.argtypes = [C.c_double, d, C.c_double, d]
            _lib.orc_build_event.restype = C.c_int
            _lib.orc_path_plane.restype = C.c_int
            _lib.orc_propagate_plane.restype = C.c_int
            del i
    return _lib


class Oracle:
    """Holds the ctypes views of one geometry (layers, plans) and a parameter set."""

    def __init__(self, geom, params: dict | None = None, tie: dict | None = None):
        self.geom = geom
        L = geom.n_layers
        self._layers = (Layer * L)()
        for i in range(L):
            ly = self._layers[i]
            ly.kind = int(geom.kind[i]); ly.n_eta = int(geom.n_eta[i]); ly.n_phi = int(geom.n_phi[i])
            ly.pos = float(geom.pos[i]); ly.lo = float(geom.lo[i]); ly.hi = float(geom.hi[i])
            ly.x_over_x0 = float(geom.x_over_x0[i])
            for j in range(3):
                ly.sig[j] = float(geom.sig[i, j])
            ly.eta_lo = float(geom.eta_lo[i]); ly.eta_hi = float(geom.eta_hi[i])
        self._plan, self._plan_off = geom.plan_arrays()
        self.g = Geom(float(geom.bz), float(geom.barrel_eta_max), L, len(geom.plans),
                      self._layers, _p(self._plan, C.c_int), _p(self._plan_off, C.c_int))
        self.set_params(params or {})
        t = dict(chi2_rel=1e-3, win_abs=1e-5, win_rel=1e-4, score_abs=2e-3, score_rel=1e-4, edge_rel=1e-5,
                 kappa=2.0 ** 24)
        t.update(tie or {})
        self.tie = Tie(**t)
        self.lib = lib()

    def set_params(self, params: dict):
        from paper_2312_11728_gb300.synth import default_params
        p = default_params(**params)
        self.params = p
        self.P = Params(p["chi2_cut"], p["win_nsigma"], p["deta_min"], p["deta_max"], p["dphi_min"],
                        p["dphi_max"], p["score_hit"], p["score_hole"], int(p["max_cands"]),
                        int(p["max_holes"]), int(p["material"]), int(p.get("binned", 1)),
                        float(p["score_overlap"]))

    @property
    def gp(self):
        return C.byref(self.g)

    def set_modules(self, mod_c, mod_n, hit_mod):
        """Module planes (Sec. 3.1: position and normal) and the module of every global hit id
        (-1: on the layer's own surface) for the following calls; None clears them."""
        if mod_c is None:
            self._mods = None
            self.g.mods = None
            return
        self._mod_arrays = (np.ascontiguousarray(mod_c, np.float64), np.ascontiguousarray(mod_n, np.float64),
                            np.ascontiguousarray(hit_mod, np.int32))
        c, n, h = self._mod_arrays
        self._mods = Modules(int(c.shape[0]), _p(c), _p(n), _p(h, C.c_int))
        self.g.mods = C.pointer(self._mods)

    def path_plane(self, p, c, n):
        """Crossing of the helix from p with the module plane n.(x - c) = 0 nearest to p."""
        s, m = C.c_double(0.0), C.c_double(0.0)
        ok = self.lib.orc_path_plane(C.c_double(self.geom.bz), _p(np.ascontiguousarray(p, np.float64)),
                                     _p(np.ascontiguousarray(c, np.float64)), _p(np.ascontiguousarray(n, np.float64)),
                                     C.byref(s), C.byref(m))
        return bool(ok), s.value, m.value

    def jacobian_plane(self, p, s, n):
        J = np.zeros(36)
        self.lib.orc_jacobian_plane(C.c_double(self.geom.bz), _p(np.ascontiguousarray(p, np.float64)),
                                    C.c_double(s), _p(np.ascontiguousarray(n, np.float64)), _p(J))
        return J.reshape(6, 6)

    def propagate_plane(self, p, c21, c, n):
        """Step to a module plane (no material): (reached, p', C', s)."""
        po, co, s = np.zeros(6), np.zeros(21), C.c_double(0.0)
        r = self.lib.orc_propagate_plane(C.c_double(self.geom.bz), _p(np.ascontiguousarray(p, np.float64)),
                                         _p(np.ascontiguousarray(c21, np.float64)),
                                         _p(np.ascontiguousarray(c, np.float64)),
                                         _p(np.ascontiguousarray(n, np.float64)), _p(po), _p(co), C.byref(s))
        return bool(r), po, co, s.value

    # ---- single steps (float64 numpy in/out)
    def helix(self, p, s):
        out = np.zeros(6)
        self.lib.orc_helix(C.c_double(self.geom.bz), _p(np.ascontiguousarray(p, np.float64)), C.c_double(s), _p(out))
        return out

    def path(self, layer, p):
        s = C.c_double(0.0)
        m = C.c_double(0.0)
        ok = self.lib.orc_path(self.gp, int(layer), _p(np.ascontiguousarray(p, np.float64)), C.byref(s), C.byref(m))
        return bool(ok), s.value, m.value

    def path_inward(self, layer, p):
        """Inward crossing of a state moving inward (the reversed state of the backward fit)."""
        s = C.c_double(0.0)
        m = C.c_double(0.0)
        ok = self.lib.orc_path_inward(self.gp, int(layer), _p(np.ascontiguousarray(p, np.float64)), C.byref(s),
                                      C.byref(m))
        return bool(ok), s.value, m.value

    def reverse(self, p, c21):
        """The same trajectory traversed in the opposite direction (backward fit, Sec. 2.2)."""
        pr, cr = np.zeros(6), np.zeros(21)
        self.lib.orc_reverse(_p(np.ascontiguousarray(p, np.float64)), _p(np.ascontiguousarray(c21, np.float64)),
                             _p(pr), _p(cr))
        return pr, cr

    def propagate_backward(self, layer, p, c21, material=None):
        """Backward-fit propagation step to an inner layer (Sec. 2.2)."""
        mat = self.params["material"] if material is None else int(material)
        po, co, s = np.zeros(6), np.zeros(21), C.c_double(0.0)
        r = self.lib.orc_propagate_backward(self.gp, int(layer), _p(np.ascontiguousarray(p, np.float64)),
                                            _p(np.ascontiguousarray(c21, np.float64)), int(mat), _p(po), _p(co),
                                            C.byref(s))
        return r, po, co, s.value

    def jacobian(self, layer, p, s):
        J = np.zeros(36)
        self.lib.orc_jacobian(self.gp, int(layer), _p(np.ascontiguousarray(p, np.float64)), C.c_double(s), _p(J))
        return J.reshape(6, 6)

    def jacobian_fixed_s(self, p, s):
        A = np.zeros(36)
        self.lib.orc_jacobian_fixed_s(C.c_double(self.geom.bz), _p(np.ascontiguousarray(p, np.float64)),
                                      C.c_double(s), _p(A))
        return A.reshape(6, 6)

    def transport(self, J, c21):
        out = np.zeros(21)
        self.lib.orc_transport(_p(np.ascontiguousarray(J, np.float64).ravel()),
                               _p(np.ascontiguousarray(c21, np.float64)), _p(out))
        return out

    def material(self, layer, p, c21, direction=1.0):
        p = np.array(p, np.float64)
        c = np.array(c21, np.float64)
        ok = self.lib.orc_material(C.byref(self._layers[layer]), _p(p), _p(c), C.c_double(direction))
        return bool(ok), p, c

    def theta0(self, pmag, t):
        out = C.c_double(0.0)
        self.lib.orc_ms_theta0(C.c_double(pmag), C.c_double(t), C.byref(out))
        return out.value

    def eloss(self, pmag, t):
        return self.lib.orc_eloss(pmag, t)

    def propagate(self, layer, p, c21, material=None):
        mat = self.params["material"] if material is None else int(material)
        po, co, s = np.zeros(6), np.zeros(21), C.c_double(0.0)
        r = self.lib.orc_propagate(self.gp, int(layer), _p(np.ascontiguousarray(p, np.float64)),
                                   _p(np.ascontiguousarray(c21, np.float64)), int(mat), _p(po), _p(co), C.byref(s))
        return r, po, co, s.value

    def window(self, layer, p, c21):
        out = np.zeros(4)
        self.lib.orc_window(C.byref(self._layers[layer]), C.byref(self.P),
                            _p(np.ascontiguousarray(p, np.float64)), _p(np.ascontiguousarray(c21, np.float64)), _p(out))
        return out

    def chi2(self, p, c21, m, v6):
        x = C.c_double(0.0)
        ok = self.lib.orc_chi2(_p(np.ascontiguousarray(p, np.float64)), _p(np.ascontiguousarray(c21, np.float64)),
                               _p(np.ascontiguousarray(m, np.float64)), _p(np.ascontiguousarray(v6, np.float64)), C.byref(x))
        return bool(ok), x.value

    def update(self, p, c21, m, v6, joseph=False):
        po, co, x = np.zeros(6), np.zeros(21), C.c_double(0.0)
        ok = self.lib.orc_update(_p(np.ascontiguousarray(p, np.float64)), _p(np.ascontiguousarray(c21, np.float64)),
                                 _p(np.ascontiguousarray(m, np.float64)), _p(np.ascontiguousarray(v6, np.float64)),
                                 int(joseph), _p(po), _p(co), C.byref(x))
        return bool(ok), po, co, x.value

    def seed(self, h9, v18, layers3, material=None):
        mat = self.params["material"] if material is None else int(material)
        p, c, pi = np.zeros(6), np.zeros(21), np.zeros(6)
        ok = self.lib.orc_seed(self.gp, int(mat), _p(np.ascontiguousarray(h9, np.float64)),
                               _p(np.ascontiguousarray(v18, np.float64)),
                               _p(np.ascontiguousarray(layers3, np.int32), C.c_int), _p(p), _p(c), _p(pi))
        return bool(ok), p, c, pi

    def surfaces(self):
        """(kind, position) of every layer surface: the frames in which results are compared."""
        return np.asarray(self.geom.kind).copy(), np.asarray(self.geom.pos, np.float64).copy()

    # ---- batches
    def seed_batch(self, seed_hits, seed_layers, xyz, cov, material=None):
        mat = self.params["material"] if material is None else int(material)
        n = int(seed_hits.shape[0])
        sh = np.ascontiguousarray(seed_hits, np.int32)
        sl = np.ascontiguousarray(seed_layers, np.int32)
        x = np.ascontiguousarray(xyz, np.float64)
        cv = np.ascontiguousarray(cov, np.float64)
        p, c, pi = np.zeros((n, 6)), np.zeros((n, 21)), np.zeros((n, 6))
        reg, st, status = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        self.lib.orc_seed_batch(self.gp, int(mat), n, _p(sh, C.c_int), _p(sl, C.c_int), _p(x), _p(cv),
                                _p(p), _p(c), _p(pi), _p(reg, C.c_int), _p(st, C.c_int), _p(status, C.c_int))
        return dict(p=p, c=c, pinit=pi, region=reg, start=st, status=status, surf=self.surfaces())

    def fit_batch(self, layers, hits, xyz, cov, p0, c0, material=None, outlier_chi2=None):
        """Kalman fit over a known assignment (Sec. 4); outlier_chi2 > 0 rejects hits above it."""
        mat = self.params["material"] if material is None else int(material)
        cut = float(self.params.get("fit_outlier_chi2", 0.0) if outlier_chi2 is None else outlier_chi2)
        n, m = layers.shape
        la = np.ascontiguousarray(layers, np.int32)
        hi = np.ascontiguousarray(hits, np.int32)
        x = np.ascontiguousarray(xyz, np.float64)
        cv = np.ascontiguousarray(cov, np.float64)
        q0 = np.ascontiguousarray(p0, np.float64)
        d0 = np.ascontiguousarray(c0, np.float64)
        p, c, chi2 = np.zeros((n, 6)), np.zeros((n, 21)), np.zeros(n)
        nupd, status, near = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        ctr = np.zeros(4, np.int64)
        self.lib.orc_fit_batch(self.gp, int(mat), int(n), int(m), _p(la, C.c_int), _p(hi, C.c_int), _p(x), _p(cv),
                               _p(q0), _p(d0), C.c_double(cut), _p(p), _p(c), _p(chi2), _p(nupd, C.c_int),
                               _p(status, C.c_int), _p(near, C.c_int), _p(ctr, C.c_longlong))
        return dict(p=p, c=c, chi2=chi2, nupd=nupd, status=status, near_cut=near, counters=ctr, surf=self.surfaces())

    def bkfit_batch(self, layers, hits, xyz, cov, p_start, c_start, cov_scale, material=None, outlier_chi2=None):
        """Backward fit (Sec. 2.2) of tracks listed in forward order, from their state on the
        last listed layer (covariance scaled by cov_scale) to the innermost listed layer."""
        mat = self.params["material"] if material is None else int(material)
        cut = float(self.params.get("fit_outlier_chi2", 0.0) if outlier_chi2 is None else outlier_chi2)
        n, m = layers.shape
        la = np.ascontiguousarray(layers, np.int32)
        hi = np.ascontiguousarray(hits, np.int32)
        x = np.ascontiguousarray(xyz, np.float64)
        cv = np.ascontiguousarray(cov, np.float64)
        q0 = np.ascontiguousarray(p_start, np.float64)
        d0 = np.ascontiguousarray(c_start, np.float64)
        p, c, chi2 = np.zeros((n, 6)), np.zeros((n, 21)), np.zeros(n)
        nupd, status, near = np.zeros(n, np.int32), np.zeros(n, np.int32), np.zeros(n, np.int32)
        ctr = np.zeros(4, np.int64)
        self.lib.orc_bkfit_batch(self.gp, int(mat), int(n), int(m), _p(la, C.c_int), _p(hi, C.c_int), _p(x),
                                 _p(cv), _p(q0), _p(d0), C.c_double(cov_scale), C.c_double(cut), _p(p), _p(c),
                                 _p(chi2), _p(nupd, C.c_int), _p(status, C.c_int), _p(near, C.c_int),
                                 _p(ctr, C.c_longlong))
        return dict(p=p, c=c, chi2=chi2, nupd=nupd, status=status, near_cut=near, counters=ctr, surf=self.surfaces())

    def build_event(self, layer_off, xyz, cov, seed_hits, seed_layers, binned=True):
        """Combinatorial forward search for the seeds of one event (hits [layer_off[0], layer_off[-1]))."""
        self.P.binned = int(binned)
        S = int(seed_hits.shape[0])
        mp = max(len(p) for p in self.geom.plans)
        lo = np.ascontiguousarray(layer_off, np.int64)
        x = np.ascontiguousarray(xyz, np.float64)
        cv = np.ascontiguousarray(cov, np.float64)
        sh = np.ascontiguousarray(seed_hits, np.int32)
        sl = np.ascontiguousarray(seed_layers, np.int32)
        res, out = _build_out(S, mp)
        rc = self.lib.orc_build_event(self.gp, C.byref(self.P), C.byref(self.tie), _p(lo, C.c_longlong), _p(x), _p(cv),
                                      S, _p(sh, C.c_int), _p(sl, C.c_int), C.byref(out))
        if rc != 0:
            raise RuntimeError(f"orc_build_event failed ({rc})")
        return res

    def build_backward_event(self, layer_off, xyz, cov, p_start, c_start, first_layer, binned=True):
        """Combinatorial backward search (Sec. 2.2) for tracks of one event from their state on
        their innermost found layer; hits indexed by the steps of the reversed region plan."""
        self.P.binned = int(binned)
        S = int(np.asarray(first_layer).shape[0])
        mp = max(len(p) for p in self.geom.plans)
        lo = np.ascontiguousarray(layer_off, np.int64)
        x = np.ascontiguousarray(xyz, np.float64)
        cv = np.ascontiguousarray(cov, np.float64)
        ps = np.ascontiguousarray(p_start, np.float64)
        cs = np.ascontiguousarray(c_start, np.float64)
        fl = np.ascontiguousarray(first_layer, np.int32)
        res, out = _build_out(S, mp)
        rc = self.lib.orc_build_backward_event(self.gp, C.byref(self.P), C.byref(self.tie), _p(lo, C.c_longlong),
                                               _p(x), _p(cv), S, _p(ps), _p(cs), _p(fl, C.c_int), C.byref(out))
        if rc != 0:
            raise RuntimeError(f"orc_build_backward_event failed ({rc})")
        return res


def clean_seeds(seed_hits, n_hits):
    """Seed cleaning (Sec. 2.2): keep flags; a seed sharing >= 2 hits with a lower-index seed is dropped."""
    lib_ = lib()
    sh = np.ascontiguousarray(seed_hits, np.int32)
    keep = np.zeros(sh.shape[0], np.int32)
    lib_.orc_clean_seeds(int(sh.shape[0]), _p(sh, C.c_int), C.c_longlong(int(n_hits)), _p(keep, C.c_int))
    return keep


def remove_duplicates(hits, score, n_hits, min_hits=0, frac=0.5):
    """Quality filter and duplicate removal (Sec. 2.2): keep flags over the rows of `hits`."""
    lib_ = lib()
    h = np.ascontiguousarray(hits, np.int32)
    sc = np.ascontiguousarray(score, np.float64)
    keep = np.zeros(h.shape[0], np.int32)
    lib_.orc_remove_duplicates(int(h.shape[0]), int(h.shape[1]), _p(h, C.c_int), _p(sc), C.c_longlong(int(n_hits)),
                              int(min_hits), C.c_double(frac), _p(keep, C.c_int))
    return keep


def _build_out(S, mp):
    res = dict(params=np.zeros((S, 6)), cov=np.zeros((S, 21)), score=np.zeros(S), chi2=np.zeros(S),
               nfound=np.zeros(S, np.int32), nholes=np.zeros(S, np.int32),
               hits=np.zeros((S, mp), np.int32), tie_step=np.zeros(S, np.int32),
               region=np.zeros(S, np.int32), start=np.zeros(S, np.int32), counters=np.zeros(4, np.int64),
               ovl=np.zeros((S, mp), np.int32))
    out = BuildOut(_p(res["params"]), _p(res["cov"]), _p(res["score"]), _p(res["chi2"]),
                   _p(res["nfound"], C.c_int), _p(res["nholes"], C.c_int), _p(res["hits"], C.c_int), mp,
                   _p(res["tie_step"], C.c_int), _p(res["region"], C.c_int), _p(res["start"], C.c_int),
                   _p(res["counters"], C.c_longlong), _p(res["ovl"], C.c_int))
    return res, out


def hit_layers(layer_off, ids):
    """Layer of each (global) hit id given the per-layer offsets of its event (host bookkeeping)."""
    return (np.searchsorted(np.asarray(layer_off), np.asarray(ids), side="right") - 1).astype(np.int32)
