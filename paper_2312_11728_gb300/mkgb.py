"""Python binding of libmkgb.so (include/mkgb.h): argument marshalling only.

Every step of the build and the fit runs in the library's CUDA kernels.  Arrays may be
torch CUDA tensors (passed as device pointers, calls asynchronous on the context's
stream) or numpy arrays (host pointers; the library copies them and returns after its
outputs are written).  Loading fails loudly if the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmkgb.so")

BARREL, DISK = 0, 1
FP32, FP64 = 0, 2
MAX_CANDS = 8
HIT_MISS, HIT_SKIP, HIT_STOP, HIT_PRE = -1, -2, -3, -4
ERRORS = {-1: "MKGB_EINVAL", -2: "MKGB_ENOMEM", -3: "MKGB_ECUDA", -5: "MKGB_ESTATE"}


class Layer(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pos", C.c_float), ("lo", C.c_float), ("hi", C.c_float),
                ("x_over_x0", C.c_float), ("sig_local", C.c_float * 3), ("n_eta_bins", C.c_int32),
                ("n_phi_bins", C.c_int32), ("eta_lo", C.c_float), ("eta_hi", C.c_float)]


class Params(C.Structure):
    _fields_ = [("chi2_cut", C.c_float), ("max_cands", C.c_int32), ("max_holes", C.c_int32),
                ("win_nsigma", C.c_float), ("deta_min", C.c_float), ("deta_max", C.c_float),
                ("dphi_min", C.c_float), ("dphi_max", C.c_float), ("score_hit", C.c_float),
                ("score_hole", C.c_float), ("barrel_eta_max", C.c_float), ("material", C.c_int32),
                ("precision", C.c_int32), ("kappa_fp64", C.c_float), ("fit_outlier_chi2", C.c_float),
                ("score_overlap", C.c_float)]


class Tracks(C.Structure):
    _fields_ = [("params", C.c_void_p), ("cov", C.c_void_p), ("chi2", C.c_void_p), ("score", C.c_void_p),
                ("nfound", C.c_void_p), ("nholes", C.c_void_p), ("hits", C.c_void_p), ("max_plan", C.c_int32),
                ("ovl_hits", C.c_void_p)]


EXPORTS = ["mkgb_create", "mkgb_destroy", "mkgb_last_error", "mkgb_version", "mkgb_load_geometry",
           "mkgb_set_params", "mkgb_load_hits", "mkgb_load_modules", "mkgb_load_hits_modular", "mkgb_seed", "mkgb_build", "mkgb_build_backward", "mkgb_fit",
           "mkgb_fit_backward",
           "mkgb_fit_static", "mkgb_fit_grad", "mkgb_run", "mkgb_run_host", "mkgb_run_modular", "mkgb_set_launch",
           "mkgb_autotune",
           "mkgb_probe_peak", "mkgb_clean_seeds", "mkgb_remove_duplicates", "mkgb_propagate", "mkgb_update",
           "mkgb_counters"]

_lib = None


class MkgbError(RuntimeError):
    pass


def load_library(path: str = LIB_PATH):
    """Loads libmkgb.so (raises if it is missing: there is no fallback path)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise MkgbError(f"{path} not built: run `python -m paper_2312_11728_gb300.build` "
                        "(or __graft_entry__.build()); there is no CPU fallback")
    lib = C.CDLL(path)
    vp, i32, f32 = C.c_void_p, C.c_int, C.c_float
    lib.mkgb_create.argtypes = [C.POINTER(vp), i32, vp]
    lib.mkgb_destroy.argtypes = [vp]
    lib.mkgb_destroy.restype = None
    lib.mkgb_last_error.argtypes = [vp]
    lib.mkgb_last_error.restype = C.c_char_p
    lib.mkgb_version.restype = C.c_char_p
    lib.mkgb_load_geometry.argtypes = [vp, C.POINTER(Layer), i32, vp, vp, i32, f32]
    lib.mkgb_set_params.argtypes = [vp, C.POINTER(Params)]
    lib.mkgb_load_hits.argtypes = [vp, i32, vp, vp, vp, i32]
    lib.mkgb_seed.argtypes = [vp, i32, vp, i32, vp, vp, vp]
    lib.mkgb_build.argtypes = [vp, C.POINTER(Tracks), i32]
    lib.mkgb_fit.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.mkgb_fit_backward.argtypes = [vp, i32, i32, vp, vp, vp, vp, f32, vp, vp, vp, vp, i32]
    lib.mkgb_build_backward.argtypes = [vp, i32, vp, vp, vp, vp, C.POINTER(Tracks), i32]
    lib.mkgb_fit_static.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
    lib.mkgb_fit_grad.argtypes = [vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, i32]
    lib.mkgb_run.argtypes = [vp, i32, vp, vp, vp, i32, vp, C.POINTER(Tracks), i32, i32, vp, vp, vp, vp, vp, vp, vp,
                             vp]
    lib.mkgb_run_host.argtypes = [vp, i32, vp, vp, vp, i32, vp, C.POINTER(Tracks), i32, i32, vp, vp, vp, vp, vp, vp,
                                  vp, vp]
    lib.mkgb_set_launch.argtypes = [vp, i32, i32, i32]
    lib.mkgb_autotune.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(f32)]
    lib.mkgb_probe_peak.argtypes = [vp, i32, C.POINTER(C.c_double)]
    lib.mkgb_clean_seeds.argtypes = [vp, i32, vp, vp, i32]
    lib.mkgb_remove_duplicates.argtypes = [vp, i32, i32, vp, vp, i32, f32, vp, i32]
    lib.mkgb_propagate.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, i32]
    lib.mkgb_update.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp, vp, i32]
    lib.mkgb_counters.argtypes = [vp, i32, vp]
    lib.mkgb_load_modules.argtypes = [vp, i32, vp, vp, vp]
    lib.mkgb_load_hits_modular.argtypes = [vp, i32, vp, vp, vp, vp, i32]
    lib.mkgb_run_modular.argtypes = [vp, i32, vp, vp, vp, vp, i32, vp, C.POINTER(Tracks), i32, i32, vp, vp, vp, vp,
                                     vp, vp, vp, vp]
    lib.mkgb_version.argtypes = []
    # every entry point is declared: an undeclared one would pass a host pointer given as a Python
    # int as a 32-bit C int, truncating any address above 2 GB
    missing = [n for n in EXPORTS if getattr(lib, n).argtypes is None]
    if missing:
        raise MkgbError(f"entry points without argument types: {missing}")
    _lib = lib
    return lib


def _is_torch(a):
    return type(a).__module__.startswith("torch")


_keep = []   # host copies made for the call in progress


def _ptr(a, dtype, out=False):
    """(pointer, on_device) of an array argument; None -> (None, None).  Host inputs of another
    dtype or layout are copied; outputs must already be contiguous arrays of the right dtype."""
    if a is None:
        return None, None
    if _is_torch(a):
        import torch
        want = {np.float32: torch.float32, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise MkgbError(f"tensor must be contiguous {want}, got {a.dtype}")
        return C.c_void_p(a.data_ptr()), a.is_cuda
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous):
        if out:
            raise MkgbError(f"output must be a C-contiguous numpy {np.dtype(dtype).name} array")
        a = np.ascontiguousarray(a, dtype)
        _keep.append(a)
    return C.c_void_p(a.ctypes.data), False


def _same(*flags):
    fl = {f for f in flags if f is not None}
    if len(fl) > 1:
        raise MkgbError("mix of device tensors and host arrays in one call")
    return int(fl.pop()) if fl else 0


class Context:
    """One mkgb context on a CUDA device, launching on a given stream (default: torch's current)."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        h = C.c_void_p()
        s = None
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream(device)
            except ImportError:
                pass
        if stream is not None:
            handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
            # torch's default stream has handle 0, which the library reads as "create a stream":
            # pass cudaStreamLegacy (1) so both launch on the same stream
            s = C.c_void_p(handle if handle else 1)
        rc = self.lib.mkgb_create(C.byref(h), int(device), s)
        if rc != 0:
            raise MkgbError(f"mkgb_create failed ({ERRORS.get(rc, rc)})")
        self.h = h
        self.device = device
        self.max_plan = 0
        self.n_seeds = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.mkgb_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        _keep.clear()
        if rc != 0:
            msg = self.lib.mkgb_last_error(self.h).decode()
            raise MkgbError(f"{what} failed ({ERRORS.get(rc, rc)}): {msg}")

    # ---- setup
    def load_geometry(self, geom):
        L = geom.n_layers
        arr = (Layer * L)()
        for i in range(L):
            arr[i] = Layer(int(geom.kind[i]), float(geom.pos[i]), float(geom.lo[i]), float(geom.hi[i]),
                           float(geom.x_over_x0[i]), (C.c_float * 3)(*[float(v) for v in geom.sig[i]]),
                           int(geom.n_eta[i]), int(geom.n_phi[i]), float(geom.eta_lo[i]), float(geom.eta_hi[i]))
        plan, off = geom.plan_arrays()
        self._check(self.lib.mkgb_load_geometry(self.h, arr, L, plan.ctypes.data, off.ctypes.data, len(geom.plans),
                                                float(geom.bz)), "mkgb_load_geometry")
        self.max_plan = geom.max_plan
        self.barrel_eta_max = float(geom.barrel_eta_max)

    def set_params(self, params: dict):
        p = Params(float(params["chi2_cut"]), int(params["max_cands"]), int(params["max_holes"]),
                   float(params["win_nsigma"]), float(params["deta_min"]), float(params["deta_max"]),
                   float(params["dphi_min"]), float(params["dphi_max"]), float(params["score_hit"]),
                   float(params["score_hole"]), float(params.get("barrel_eta_max", self.barrel_eta_max)),
                   int(params["material"]), int(params.get("precision", 0)),
                   float(params.get("kappa_fp64", 0.0)), float(params.get("fit_outlier_chi2", 0.0)),
                   float(params.get("score_overlap", 0.0)))
        self._check(self.lib.mkgb_set_params(self.h, C.byref(p)), "mkgb_set_params")

    # ---- data
    def load_modules(self, modules):
        """mkgb_load_modules: module planes (layer, position, unit normal) of a synth.Modules
        table (None removes them)."""
        if modules is None:
            self._check(self.lib.mkgb_load_modules(self.h, 0, None, None, None), "mkgb_load_modules")
            return
        lay = np.ascontiguousarray(modules.layer, np.int32)
        pos = np.ascontiguousarray(modules.c, np.float32)
        nrm = np.ascontiguousarray(modules.n, np.float32)
        self._check(self.lib.mkgb_load_modules(self.h, int(lay.shape[0]), lay.ctypes.data, pos.ctypes.data,
                                               nrm.ctypes.data), "mkgb_load_modules")

    def load_hits(self, n_events, seg_off, xyz, cov, hit_module=None):
        """mkgb_load_hits, or mkgb_load_hits_modular when hit_module (module per hit) is given."""
        so = np.ascontiguousarray(seg_off, np.int64)
        px, dx = _ptr(xyz, np.float32)
        pc, dc = _ptr(cov, np.float32)
        if hit_module is not None:
            pm, dm = _ptr(hit_module, np.int32)
            self._check(self.lib.mkgb_load_hits_modular(self.h, int(n_events), so.ctypes.data, px, pc, pm,
                                                        _same(dx, dc, dm)), "mkgb_load_hits_modular")
            return
        self._check(self.lib.mkgb_load_hits(self.h, int(n_events), so.ctypes.data, px, pc, _same(dx, dc)),
                    "mkgb_load_hits")

    def seed(self, seed_hits, state=None, cov=None, info=None):
        n = int(seed_hits.shape[0])
        ps, d0 = _ptr(seed_hits, np.int32)
        p1, d1 = _ptr(state, np.float32, out=True)
        p2, d2 = _ptr(cov, np.float32, out=True)
        p3, d3 = _ptr(info, np.int32, out=True)
        self._check(self.lib.mkgb_seed(self.h, n, ps, _same(d0, d1, d2, d3), p1, p2, p3), "mkgb_seed")
        self.n_seeds = n

    def build(self, out: dict):
        """out: dict of arrays params (n,6) cov (n,21) chi2 score nfound nholes hits (n, max_plan), and
        optionally ovl (n, max_plan): the overlap hits on modular layers."""
        f, i = np.float32, np.int32
        ptrs = [_ptr(out[k], t, out=True) for k, t in (("params", f), ("cov", f), ("chi2", f), ("score", f),
                                              ("nfound", i), ("nholes", i), ("hits", i))]
        if "ovl" in out:
            ptrs.append(_ptr(out["ovl"], i, out=True))
        t = Tracks(*[p for p, _ in ptrs[:7]], int(out["hits"].shape[1]), ptrs[7][0] if len(ptrs) > 7 else None)
        self._check(self.lib.mkgb_build(self.h, C.byref(t), _same(*[d for _, d in ptrs])), "mkgb_build")
        return out

    def build_backward(self, track_event, first_layer, p_start, c_start, out: dict):
        """mkgb_build_backward: the backward search of tracks from their state on their innermost
        found layer; out as for build (hits and the optional ovl indexed by the reversed plan's
        steps)."""
        f, i = np.float32, np.int32
        args = [_ptr(track_event, i), _ptr(first_layer, i), _ptr(p_start, f), _ptr(c_start, f)]
        ptrs = [_ptr(out[k], t, out=True) for k, t in (("params", f), ("cov", f), ("chi2", f), ("score", f),
                                              ("nfound", i), ("nholes", i), ("hits", i))]
        if "ovl" in out:
            ptrs.append(_ptr(out["ovl"], i, out=True))
        t = Tracks(*[p for p, _ in ptrs[:7]], int(out["hits"].shape[1]), ptrs[7][0] if len(ptrs) > 7 else None)
        n = int(np.asarray(first_layer).shape[0]) if not _is_torch(first_layer) else int(first_layer.shape[0])
        self._check(self.lib.mkgb_build_backward(self.h, n, *[p for p, _ in args], C.byref(t),
                                                 _same(*[d for _, d in args + ptrs])), "mkgb_build_backward")
        return out

    def fit(self, layers, hits, p0, c0, p_out, c_out, chi2_out, status_out=None):
        n, m = layers.shape
        args = [_ptr(layers, np.int32), _ptr(hits, np.int32), _ptr(p0, np.float32), _ptr(c0, np.float32),
                _ptr(p_out, np.float32, True), _ptr(c_out, np.float32, True), _ptr(chi2_out, np.float32, True),
                _ptr(status_out, np.int32, True)]
        self._check(self.lib.mkgb_fit(self.h, int(n), int(m), *[p for p, _ in args], _same(*[d for _, d in args])),
                    "mkgb_fit")

    def run(self, n_events, seg_off, xyz, cov, seed_hits, out: dict, layers, hits, p0, c0, p_out, c_out, chi2_out,
            status_out=None, hit_module=None):
        """mkgb_run: load_hits + seed + build + fit in one call, device tensors only; the fit runs
        beside the seed fit and the search inside the call.  With hit_module (module per hit):
        mkgb_run_modular, and out may hold ovl."""
        so = np.ascontiguousarray(seg_off, np.int64)
        f, i = np.float32, np.int32
        ptrs = [_ptr(out[k], t, out=True) for k, t in (("params", f), ("cov", f), ("chi2", f), ("score", f),
                                              ("nfound", i), ("nholes", i), ("hits", i))]
        if "ovl" in out:
            ptrs.append(_ptr(out["ovl"], i, out=True))
        t = Tracks(*[p for p, _ in ptrs[:7]], int(out["hits"].shape[1]), ptrs[7][0] if len(ptrs) > 7 else None)
        args = [_ptr(xyz, f), _ptr(cov, f), _ptr(seed_hits, i), _ptr(layers, i), _ptr(hits, i), _ptr(p0, f),
                _ptr(c0, f), _ptr(p_out, f, True), _ptr(c_out, f, True), _ptr(chi2_out, f, True),
                _ptr(status_out, i, True)]
        if _same(*[d for _, d in args + ptrs]) != 1:
            raise MkgbError("mkgb_run takes CUDA tensors only")
        (px, _), (pc, _), (ps, _), (pl, _), (ph, _), (pp, _), (pq, _), (po, _), (pco, _), (px2, _), (pst, _) = args
        n, m = layers.shape
        if hit_module is not None:
            pm, dm = _ptr(hit_module, i)
            if dm != 1:
                raise MkgbError("mkgb_run_modular takes CUDA tensors only")
            self._check(self.lib.mkgb_run_modular(self.h, int(n_events), so.ctypes.data, px, pc, pm,
                                                  int(seed_hits.shape[0]), ps, C.byref(t), int(n), int(m), pl, ph,
                                                  pp, pq, po, pco, px2, pst), "mkgb_run_modular")
        else:
            self._check(self.lib.mkgb_run(self.h, int(n_events), so.ctypes.data, px, pc, int(seed_hits.shape[0]),
                                          ps, C.byref(t), int(n), int(m), pl, ph, pp, pq, po, pco, px2, pst),
                        "mkgb_run")
        self.n_seeds = int(seed_hits.shape[0])
        return out

    def run_host(self, n_events, seg_off, xyz, cov, seed_hits, out: dict, layers, hits, p0, c0, p_out, c_out,
                 chi2_out, status_out=None):
        """mkgb_run_host: the one-call pass with every array in host memory (numpy arrays or CPU
        tensors; page-locked ones let the library overlap its copies with the kernels)."""
        so = np.ascontiguousarray(seg_off, np.int64)
        f, i = np.float32, np.int32
        ptrs = [_ptr(out[k], t, out=True) for k, t in (("params", f), ("cov", f), ("chi2", f), ("score", f),
                                              ("nfound", i), ("nholes", i), ("hits", i))]
        if "ovl" in out:
            ptrs.append(_ptr(out["ovl"], i, out=True))
        t = Tracks(*[p for p, _ in ptrs[:7]], int(out["hits"].shape[1]), ptrs[7][0] if len(ptrs) > 7 else None)
        args = [_ptr(xyz, f), _ptr(cov, f), _ptr(seed_hits, i), _ptr(layers, i), _ptr(hits, i), _ptr(p0, f),
                _ptr(c0, f), _ptr(p_out, f, True), _ptr(c_out, f, True), _ptr(chi2_out, f, True),
                _ptr(status_out, i, True)]
        if _same(*[d for _, d in args + ptrs]) != 0:
            raise MkgbError("mkgb_run_host takes host arrays only")
        (px, _), (pc, _), (ps, _), (pl, _), (ph, _), (pp, _), (pq, _), (po, _), (pco, _), (px2, _), (pst, _) = args
        n, m = layers.shape
        self._check(self.lib.mkgb_run_host(self.h, int(n_events), so.ctypes.data, px, pc, int(seed_hits.shape[0]),
                                           ps, C.byref(t), int(n), int(m), pl, ph, pp, pq, po, pco, px2, pst),
                    "mkgb_run_host")
        self.n_seeds = int(seed_hits.shape[0])
        return out

    def fit_backward(self, layers, hits, p_start, c_start, p_out, c_out, chi2_out, status_out=None,
                     cov_scale: float = 100.0):
        """mkgb_fit_backward: tracks listed in forward order, from their state on the last listed
        layer (covariance x cov_scale) back to the first listed layer (outputs written in place)."""
        n, m = layers.shape
        args = [_ptr(layers, np.int32), _ptr(hits, np.int32), _ptr(p_start, np.float32), _ptr(c_start, np.float32)]
        outs = [_ptr(p_out, np.float32, True), _ptr(c_out, np.float32, True), _ptr(chi2_out, np.float32, True),
                _ptr(status_out, np.int32, True)]
        self._check(self.lib.mkgb_fit_backward(self.h, int(n), int(m), *[p for p, _ in args], float(cov_scale),
                                               *[p for p, _ in outs], _same(*[d for _, d in args + outs])),
                    "mkgb_fit_backward")

    def fit_static(self, layers, hits, p0, c0, p_out, c_out, chi2_out, status_out=None):
        """mkgb_fit_static: the fit without device allocations (device tensors only, at most
        65536 tracks; calls on one device must not overlap in time)."""
        n, m = layers.shape
        args = [_ptr(layers, np.int32), _ptr(hits, np.int32), _ptr(p0, np.float32), _ptr(c0, np.float32),
                _ptr(p_out, np.float32, True), _ptr(c_out, np.float32, True), _ptr(chi2_out, np.float32, True),
                _ptr(status_out, np.int32, True)]
        if _same(*[d for _, d in args]) != 1:
            raise MkgbError("mkgb_fit_static takes CUDA tensors only")
        self._check(self.lib.mkgb_fit_static(self.h, int(n), int(m), *[p for p, _ in args]), "mkgb_fit_static")

    def fit_grad(self, layers, hits, p0, c0, align, xscale, chi2_out, d_p0, d_align, d_xscale, status_out=None,
                 mode: int = 0):
        """mkgb_fit_grad: per-track chi2 at the given alignment / thickness scales and the
        derivatives of the total chi2 (outputs written in place); mode 0 reverse sweep, 1 forward."""
        n, m = layers.shape
        args = [_ptr(layers, np.int32), _ptr(hits, np.int32), _ptr(p0, np.float32), _ptr(c0, np.float32),
                _ptr(align, np.float32), _ptr(xscale, np.float32), _ptr(chi2_out, np.float32, True),
                _ptr(d_p0, np.float32, True), _ptr(d_align, np.float32, True), _ptr(d_xscale, np.float32, True),
                _ptr(status_out, np.int32, True)]
        self._check(self.lib.mkgb_fit_grad(self.h, int(n), int(m), *[p for p, _ in args], int(mode),
                                           _same(*[d for _, d in args])), "mkgb_fit_grad")

    def set_launch(self, find_shape: int = 0, select_shape: int = 0, use_graph: bool = True):
        """mkgb_set_launch: block shapes of the search kernels and CUDA-graph replay."""
        self._check(self.lib.mkgb_set_launch(self.h, int(find_shape), int(select_shape), int(bool(use_graph))),
                    "mkgb_set_launch")

    def autotune(self, reps: int = 3):
        """mkgb_autotune over the loaded seeds: returns (find_shape, select_shape, ms per search)
        and keeps the fastest shapes for later searches."""
        f, s, ms = C.c_int(0), C.c_int(0), C.c_float(0.0)
        self._check(self.lib.mkgb_autotune(self.h, int(reps), C.byref(f), C.byref(s), C.byref(ms)),
                    "mkgb_autotune")
        return f.value, s.value, ms.value

    def probe_peak(self, kind: int = 0) -> float:
        """mkgb_probe_peak: measured FMA throughput in TFLOP/s (kind 0 FP32, 1 FP64)."""
        r = C.c_double(0.0)
        self._check(self.lib.mkgb_probe_peak(self.h, int(kind), C.byref(r)), "mkgb_probe_peak")
        return r.value

    def clean_seeds(self, seed_hits, keep_out):
        """mkgb_clean_seeds: keep flags (written in place)."""
        args = [_ptr(seed_hits, np.int32), _ptr(keep_out, np.int32, True)]
        self._check(self.lib.mkgb_clean_seeds(self.h, int(seed_hits.shape[0]), *[p for p, _ in args],
                                              _same(*[d for _, d in args])), "mkgb_clean_seeds")
        return keep_out

    def remove_duplicates(self, hits, score, keep_out, min_hits: int = 0, frac: float = 0.5):
        """mkgb_remove_duplicates: keep flags over the rows of hits (written in place)."""
        args = [_ptr(hits, np.int32), _ptr(score, np.float32), _ptr(keep_out, np.int32, True)]
        self._check(self.lib.mkgb_remove_duplicates(self.h, int(hits.shape[0]), int(hits.shape[1]), args[0][0],
                                                    args[1][0], int(min_hits), float(frac), args[2][0],
                                                    _same(*[d for _, d in args])), "mkgb_remove_duplicates")
        return keep_out

    def propagate(self, layers, p_in, c_in, p_out, c_out, crossed):
        args = [_ptr(layers, np.int32), _ptr(p_in, np.float32), _ptr(c_in, np.float32), _ptr(p_out, np.float32, True),
                _ptr(c_out, np.float32, True), _ptr(crossed, np.int32, True)]
        self._check(self.lib.mkgb_propagate(self.h, int(layers.shape[0]), *[p for p, _ in args],
                                            _same(*[d for _, d in args])), "mkgb_propagate")

    def update(self, p_in, c_in, hxyz, hcov, p_out, c_out, chi2, ok):
        args = [_ptr(p_in, np.float32), _ptr(c_in, np.float32), _ptr(hxyz, np.float32), _ptr(hcov, np.float32),
                _ptr(p_out, np.float32, True), _ptr(c_out, np.float32, True), _ptr(chi2, np.float32, True),
                _ptr(ok, np.int32, True)]
        self._check(self.lib.mkgb_update(self.h, int(p_in.shape[0]), *[p for p, _ in args],
                                         _same(*[d for _, d in args])), "mkgb_update")

    def counters(self, kind: int = 0):
        out = np.zeros(5, np.int64)
        self._check(self.lib.mkgb_counters(self.h, int(kind), out.ctypes.data), "mkgb_counters")
        return out


def alloc_tracks(n, max_plan, device=None, ovl=False):
    """Output arrays of Context.build: numpy (device None) or torch CUDA tensors; ovl adds the
    overlap-hit array."""
    shapes = dict(params=((n, 6), np.float32), cov=((n, 21), np.float32), chi2=((n,), np.float32),
                  score=((n,), np.float32), nfound=((n,), np.int32), nholes=((n,), np.int32),
                  hits=((n, max_plan), np.int32))
    if ovl:
        shapes["ovl"] = ((n, max_plan), np.int32)
    if device is None:
        return {k: np.zeros(s, t) for k, (s, t) in shapes.items()}
    import torch
    tt = {np.float32: torch.float32, np.int32: torch.int32}
    return {k: torch.zeros(s, dtype=tt[t], device=device) for k, (s, t) in shapes.items()}
