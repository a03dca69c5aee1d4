"""Seed cleaning and the quality filter with duplicate removal (Sec. 2.2; mkgb_clean_seeds,
mkgb_remove_duplicates) against the oracle's, bit for bit (integer decisions on the same hit
lists and scores), on Phase-2-like events with two seeds per track."""
import numpy as np
import pytest

import oracle
from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mkgb.load_library()


def _duplicate_seed_batch(n_events=3, n_tracks=1500, seed=61):
    """Events with, per track with four or more hits, the seeds from its first three crossed
    layers and from its first, second and fourth (global hit ids)."""
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, n_tracks, seed, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=4000)
           for e in range(n_events)]
    batch = S.concat_events(evs, g.n_layers)
    rows, trk = [], []
    for e, ev in enumerate(evs):
        base = batch.hit_off[e * g.n_layers]
        for t in range(ev.track_hits.shape[0]):
            h = ev.track_hits[t]
            if (h >= 0).sum() < 4:
                continue
            rows += [h[[0, 1, 2]] + base, h[[0, 1, 3]] + base]
            trk += [(e, t), (e, t)]
    return g, batch, np.array(rows, np.int32), trk


def test_seed_cleaning_matches_oracle(lib):
    g, batch, seeds, trk = _duplicate_seed_batch()
    ctx = pipeline.make_context(g, S.default_params())
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    keep = ctx.clean_seeds(seeds, np.zeros(seeds.shape[0], np.int32))
    ref = oracle.clean_seeds(seeds, batch.hit_xyz.shape[0])
    assert np.array_equal(keep, ref)
    assert np.all(keep[0::2] == 1) and np.all(keep[1::2] == 0)
    # shuffled order: the lower index wins whichever seed it is
    perm = np.random.default_rng(1).permutation(seeds.shape[0])
    keep2 = ctx.clean_seeds(np.ascontiguousarray(seeds[perm]), np.zeros(seeds.shape[0], np.int32))
    assert np.array_equal(keep2, oracle.clean_seeds(seeds[perm], batch.hit_xyz.shape[0]))


def test_duplicate_removal_matches_oracle(lib):
    """The GPU search from both seeds of every track, then the quality filter and duplicate
    removal over (seed hits + found hits): the same keep flags as the oracle's on those lists,
    and one track of each particle's pair survives."""
    g, batch, seeds, trk = _duplicate_seed_batch()
    ctx = pipeline.make_context(g, S.default_params())
    ctx.load_hits(batch.n_events, batch.hit_off, batch.hit_xyz, batch.hit_cov)
    ctx.seed(seeds)
    out = ctx.build(mkgb.alloc_tracks(seeds.shape[0], g.max_plan))
    hits = np.ascontiguousarray(np.concatenate([seeds, np.where(out["hits"] >= 0, out["hits"], -1)], axis=1))
    ok = np.isfinite(out["score"])
    score = np.where(ok, out["score"], np.float32(-1e30)).astype(np.float32)
    keep = ctx.remove_duplicates(hits, score, np.zeros(seeds.shape[0], np.int32), min_hits=6, frac=0.5)
    ref = oracle.remove_duplicates(hits, score.astype(np.float64), batch.hit_xyz.shape[0], min_hits=6, frac=0.5)
    assert np.array_equal(keep, ref)
    pairs = ok[0::2] & ok[1::2]
    one = (keep[0::2] + keep[1::2]) == 1
    assert one[pairs].mean() > 0.9, one[pairs].mean()
    with pytest.raises(mkgb.MkgbError):
        ctx.remove_duplicates(hits, score, np.zeros(seeds.shape[0], np.int32), frac=0.0)
