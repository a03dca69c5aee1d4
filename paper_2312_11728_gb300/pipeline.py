"""One pass of the hot path over a batch of events through the C ABI.

    bin the hits of every (event, layer)        mkgb_load_hits   (a2)
    seed states, regions, (eta, phi) order      mkgb_seed        (a1, a3)
    combinatorial forward search               mkgb_build       (a4-a11, a13)
    Kalman fit over a known hit assignment      mkgb_fit         (a12)

Arrays live on the GPU (torch tensors) or on the host (numpy / pinned torch CPU tensors);
the library does all arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import mkgb
from .synth import Batch, fit_workload


@dataclass
class FitInputs:
    layers: np.ndarray   # int32 [T, M], -1 ends a list
    hits: np.ndarray     # int32 [T, M] global hit indices, -1 none
    p0: np.ndarray       # float32 [T, 6]
    c0: np.ndarray       # float32 [T, 21]
    event: np.ndarray    # int32 [T] event of each track


def fit_inputs(batch: Batch, seed: int = 0) -> FitInputs:
    """Known-assignment fit workload of a batch: every track with its true hits, started from a
    state drawn around its truth at the origin (host bookkeeping of the generator's output)."""
    parts = []
    m = 0
    for e, ev in enumerate(batch.events):
        layers, hits, p0, c0, *_ = fit_workload(ev, seed=seed + e, event_offset=int(batch.hit_off[e * batch.n_layers]))
        parts.append((layers, hits, p0, c0))
        m = max(m, layers.shape[1])
    L = np.concatenate([np.pad(p[0], ((0, 0), (0, m - p[0].shape[1])), constant_values=-1) for p in parts])
    H = np.concatenate([np.pad(p[1], ((0, 0), (0, m - p[1].shape[1])), constant_values=-1) for p in parts])
    return FitInputs(L.astype(np.int32), H.astype(np.int32),
                     np.concatenate([p[2] for p in parts]).astype(np.float32),
                     np.concatenate([p[3] for p in parts]).astype(np.float32),
                     np.concatenate([np.full(p[0].shape[0], e, np.int32) for e, p in enumerate(parts)]))


def outer_fit_inputs(fi: FitInputs, n_skip: int) -> FitInputs:
    """The fit workload without each track's first n_skip listed layers (the lists shifted left):
    the tracks as a search seeded further out would have found them, the input of a backward
    search that should find the inner hits again (host bookkeeping)."""
    L = np.full_like(fi.layers, -1)
    H = np.full_like(fi.hits, -1)
    m = fi.layers.shape[1] - n_skip
    L[:, :m] = fi.layers[:, n_skip:]
    H[:, :m] = fi.hits[:, n_skip:]
    return FitInputs(L, H, fi.p0, fi.c0, fi.event)


def plant_wrong_hits(batch: Batch, fi: FitInputs, frac: float, seed: int):
    """Known assignments with wrong hits planted: for a fraction of the tracks one listed hit
    (not the first) is replaced by a random hit of the same layer and event (host bookkeeping
    for the outlier rejection's tests).  Returns the new hit lists and the (track, step) swaps."""
    rng = np.random.default_rng(seed)
    hits = fi.hits.copy()
    L = batch.n_layers
    swaps = []
    for i in np.nonzero(rng.random(hits.shape[0]) < frac)[0]:
        n = int((fi.layers[i] >= 0).sum())
        if n < 4:
            continue
        j = int(rng.integers(1, n))
        e, l = int(fi.event[i]), int(fi.layers[i, j])
        lo, hi = batch.hit_off[e * L + l], batch.hit_off[e * L + l + 1]
        h = int(rng.integers(lo, hi))
        if h == hits[i, j]:
            continue
        hits[i, j] = h
        swaps.append((i, j))
    return hits, swaps


def to_device(a, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


class DeviceBatch:
    """A batch's inputs resident in GPU memory plus preallocated outputs."""

    def __init__(self, batch: Batch, fit: FitInputs | None, max_plan: int, device="cuda"):
        import torch
        self.n_events = batch.n_events
        self.seg_off = np.ascontiguousarray(batch.hit_off, np.int64)
        self.xyz = to_device(batch.hit_xyz, device)
        self.cov = to_device(batch.hit_cov, device)
        self.seeds = to_device(batch.seed_hits, device)
        self.out = mkgb.alloc_tracks(batch.seed_hits.shape[0], max_plan, device)
        self.fit = None
        if fit is not None:
            T = fit.layers.shape[0]
            self.fit = dict(layers=to_device(fit.layers, device), hits=to_device(fit.hits, device),
                            p0=to_device(fit.p0, device), c0=to_device(fit.c0, device),
                            p=torch.zeros((T, 6), dtype=torch.float32, device=device),
                            c=torch.zeros((T, 21), dtype=torch.float32, device=device),
                            chi2=torch.zeros(T, dtype=torch.float32, device=device),
                            status=torch.zeros(T, dtype=torch.int32, device=device))


def run_step(ctx: mkgb.Context, db: DeviceBatch):
    """Enqueues one pass of the hot path on the context's stream (asynchronous)."""
    ctx.load_hits(db.n_events, db.seg_off, db.xyz, db.cov)
    ctx.seed(db.seeds)
    ctx.build(db.out)
    if db.fit is not None:
        f = db.fit
        ctx.fit(f["layers"], f["hits"], f["p0"], f["c0"], f["p"], f["c"], f["chi2"], f["status"])


def run_step_fused(ctx: mkgb.Context, db: DeviceBatch):
    """The same pass as run_step through mkgb_run (one call; the fit overlaps the seed fit and
    the search inside it)."""
    f = db.fit
    ctx.run(db.n_events, db.seg_off, db.xyz, db.cov, db.seeds, db.out, f["layers"], f["hits"], f["p0"], f["c0"],
            f["p"], f["c"], f["chi2"], f["status"])


def run_host(ctx: mkgb.Context, batch: Batch, max_plan: int, fit: FitInputs | None = None):
    """Same pass with host arrays (the library copies in and out); returns numpy results."""
    ctx.load_hits(batch.n_events, batch.hit_off, np.ascontiguousarray(batch.hit_xyz, np.float32),
                  np.ascontiguousarray(batch.hit_cov, np.float32))
    n = batch.seed_hits.shape[0]
    state = np.zeros((n, 6), np.float32)
    cov = np.zeros((n, 21), np.float32)
    info = np.zeros((n, 3), np.int32)
    ctx.seed(np.ascontiguousarray(batch.seed_hits, np.int32), state, cov, info)
    out = ctx.build(mkgb.alloc_tracks(n, max_plan))
    res = dict(build=out, seed_state=state, seed_cov=cov, seed_info=info, build_counters=ctx.counters(0))
    if fit is not None:
        T = fit.layers.shape[0]
        p, c = np.zeros((T, 6), np.float32), np.zeros((T, 21), np.float32)
        x2, st = np.zeros(T, np.float32), np.zeros(T, np.int32)
        ctx.fit(fit.layers, fit.hits, fit.p0, fit.c0, p, c, x2, st)
        res["fit"] = dict(p=p, c=c, chi2=x2, status=st, counters=ctx.counters(1))
    return res


def make_context(geom, params: dict, device: int = 0, stream=None) -> mkgb.Context:
    ctx = mkgb.Context(device, stream)
    ctx.load_geometry(geom)
    if geom.modules is not None:   # modular layers: their hits are loaded with load_hits(hit_module=...)
        ctx.load_modules(geom.modules)
    ctx.set_params(dict(params, barrel_eta_max=params.get("barrel_eta_max", geom.barrel_eta_max)))
    return ctx


def replica_throughput(seconds: float, units: int, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas (one process per GPU, each on its own
    events): the units of all ranks / the slowest rank's time.  Returns (value, max seconds,
    total units).  dist: torch.distributed (initialised) or None for one process."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    wall, total = float(t.item()), float(u.item())
    return total / wall, wall, total
