"""Pins of seed cleaning and of the quality filter with duplicate removal (Sec. 2.2).  Readings:
a seed sharing at least two of its three hits with a seed of lower index is dropped; a track with
fewer than min_hits hits is dropped, and a track is dropped if a better one (higher score, ties to
the lower index) shares at least half of the smaller hit count; every item is judged against all
others.  Pins: brute force over all pairs on small random sets (the oracle enumerates pairs through
a hit -> items index), and workloads with two seeds per true track."""
import itertools

import numpy as np

import oracle
from paper_2312_11728_gb300 import synth as S


def _shared(a, b):
    return len(set(int(x) for x in a if x >= 0) & set(int(x) for x in b if x >= 0))


def test_cleaning_equals_brute_force_over_all_pairs():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n, n_hits = 60, 40
        seeds = np.stack([rng.choice(n_hits, 3, replace=False) for _ in range(n)]).astype(np.int32)
        keep = oracle.clean_seeds(seeds, n_hits)
        ref = np.ones(n, np.int32)
        for t, u in itertools.product(range(n), range(n)):
            if u < t and _shared(seeds[t], seeds[u]) >= 2:
                ref[t] = 0
        assert np.array_equal(keep, ref), trial
        w = 8
        tracks = np.full((n, w), -1, np.int32)
        for t in range(n):
            k = int(rng.integers(1, w + 1))
            tracks[t, :k] = rng.choice(n_hits, k, replace=False)
        score = rng.integers(0, 6, n).astype(np.float64)   # ties included
        keep = oracle.remove_duplicates(tracks, score, n_hits, min_hits=2, frac=0.5)
        ref = np.array([(tracks[t] >= 0).sum() >= 2 for t in range(n)], np.int32)
        for t, u in itertools.product(range(n), range(n)):
            if t == u:
                continue
            better = score[u] > score[t] or (score[u] == score[t] and u < t)
            nt, nu = (tracks[t] >= 0).sum(), (tracks[u] >= 0).sum()
            if better and _shared(tracks[t], tracks[u]) >= 0.5 * min(nt, nu):
                ref[t] = 0
        assert np.array_equal(keep, ref), trial


def duplicate_seeds(ev):
    """Two seeds per track with at least four hits: its hits on its first three crossed layers,
    and on its first, second and fourth (event-local hit ids, and the seed's track)."""
    rows, trk = [], []
    for t in range(ev.track_hits.shape[0]):
        h = ev.track_hits[t]
        if (h >= 0).sum() < 4:
            continue
        rows += [h[[0, 1, 2]], h[[0, 1, 3]]]
        trk += [t, t]
    return np.array(rows, np.int32), np.array(trk, np.int32)


def test_seed_cleaning_keeps_one_seed_per_track():
    g = S.geometry_barrel()
    ev = S.simulate_event(g, 500, 51, 0, eta_max=1.0, noise_per_layer=100)
    seeds, trk = duplicate_seeds(ev)
    keep = oracle.clean_seeds(seeds, ev.hit_xyz.shape[0])
    assert keep.sum() == len(np.unique(trk))
    assert np.all(keep[0::2] == 1) and np.all(keep[1::2] == 0)


def test_duplicate_removal_keeps_one_track_per_particle():
    """The oracle's forward search from both seeds of every track finds each particle twice;
    duplicate removal over (seed hits + found hits) keeps one of each pair and no fewer."""
    g = S.geometry_barrel()
    o = oracle.Oracle(g)
    ev = S.simulate_event(g, 400, 52, 0, eta_max=1.0, noise_per_layer=100,
                          pt_sampler=lambda rng, n: S.sample_pt_loguniform(rng, n, 1.0, 10.0))
    seeds, trk = duplicate_seeds(ev)
    X, V = ev.hit_xyz.astype(np.float64), ev.hit_cov.astype(np.float64)
    r = o.build_event(ev.layer_off, X, V, seeds, oracle.hit_layers(ev.layer_off, seeds))
    hits = np.concatenate([seeds, np.where(r["hits"] >= 0, r["hits"], -1)], axis=1)
    ok = np.isfinite(r["score"])
    score = np.where(ok, r["score"], -1e30)
    keep = oracle.remove_duplicates(hits, score, ev.hit_xyz.shape[0], min_hits=6, frac=0.5)
    pairs = ok[0::2] & ok[1::2]
    # exactly one of the two tracks of a particle survives
    one = (keep[0::2] + keep[1::2]) == 1
    assert one[pairs].mean() > 0.95, one[pairs].mean()
    # the survivor is the better-scored of the two
    best = np.where(score[0::2] >= score[1::2], 0, 1)
    surv = np.where(keep[0::2] == 1, 0, 1)
    assert (best == surv)[pairs & one].mean() > 0.99
