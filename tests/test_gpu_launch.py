"""Launch configuration of the search (library service; changes no arithmetic): the CUDA-graph
replay of the search rounds, the block shapes of the two-kernel rounds and of the fused round
kernel, and the autotuner give the plain two-kernel launches' results bit for bit, and a changed
batch re-records the graph."""
import numpy as np
import pytest

from paper_2312_11728_gb300 import build as B
from paper_2312_11728_gb300 import mkgb, pipeline, synth as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    B.build()
    return mkgb.load_library()


def _batch(n_events, seed):
    g = S.geometry_phase2()
    evs = [S.simulate_event(g, seed, 0, e, pt_sampler=S.sample_pt_phase2, eta_max=3.0, noise_total=4000)
           for e in range(n_events)]
    return g, S.concat_events(evs, g.n_layers)


def _search(ctx, db):
    import torch
    pipeline.run_step(ctx, db)
    torch.cuda.current_stream().synchronize()
    return {k: v.cpu().clone() for k, v in db.out.items()}


def _equal(a, b):
    import torch
    return all(torch.equal(a[k], b[k]) for k in a)


def test_graph_and_shapes_match_plain_launches(lib):
    import torch
    g, batch = _batch(3, 2024)
    params = S.default_params()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        db = pipeline.DeviceBatch(batch, None, g.max_plan, "cuda")
        plain = pipeline.make_context(g, params, stream=side)
        plain.set_launch(0, 0, use_graph=False)
        ref = _search(plain, db)
        assert int(ref["nfound"].sum()) > 0
        ctx = pipeline.make_context(g, params, stream=side)
        for f, s in [(0, 0), (1, 1), (2, 2), (1, 2), (2, 0), (3, 0), (4, 0), (5, 0)]:
            ctx.set_launch(f, s, use_graph=True)
            for _ in range(2):   # record, then replay
                assert _equal(_search(ctx, db), ref), (f, s)
            ctx.set_launch(f, s, use_graph=False)
            assert _equal(_search(ctx, db), ref), (f, s, "plain")


def test_graph_rerecords_for_a_new_batch(lib):
    import torch
    params = S.default_params()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ctx = None
        for n_events, seed in [(2, 11), (3, 12), (2, 11)]:
            g, batch = _batch(n_events, seed)
            db = pipeline.DeviceBatch(batch, None, g.max_plan, "cuda")
            if ctx is None:
                ctx = pipeline.make_context(g, params, stream=side)
            fresh = pipeline.make_context(g, params, stream=side)
            fresh.set_launch(0, 0, use_graph=False)
            assert _equal(_search(ctx, db), _search(fresh, db)), (n_events, seed)


def test_graph_inside_a_callers_capture(lib):
    """On a stream that the caller is capturing, the search's launches join the caller's graph,
    which then replays to the same results."""
    import torch
    g, batch = _batch(2, 77)
    params = S.default_params()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        db = pipeline.DeviceBatch(batch, None, g.max_plan, "cuda")
        ctx = pipeline.make_context(g, params, stream=side)
        ref = _search(ctx, db)   # allocates every buffer before the capture
        for v in db.out.values():
            v.zero_()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            ctx.build(db.out)
        graph.replay()
        side.synchronize()
        assert _equal({k: v.cpu() for k, v in db.out.items()}, ref)


def test_autotune_keeps_results(lib):
    import torch
    g, batch = _batch(3, 31)
    params = S.default_params()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        db = pipeline.DeviceBatch(batch, None, g.max_plan, "cuda")
        ctx = pipeline.make_context(g, params, stream=side)
        ref = _search(ctx, db)
        f, s, ms = ctx.autotune(reps=2)
        assert f in range(6) and s in (0, 1, 2) and ms > 0.0
        assert _equal(_search(ctx, db), ref)
        with pytest.raises(mkgb.MkgbError):
            ctx.set_launch(6, 0)
        with pytest.raises(mkgb.MkgbError):
            ctx.autotune(reps=0)


def test_autotune_before_seeds_is_an_error(lib):
    g = S.geometry_phase2()
    ctx = pipeline.make_context(g, S.default_params())
    with pytest.raises(mkgb.MkgbError):
        ctx.autotune()


def test_probe_peak(lib):
    """The FMA-throughput probe returns plausible rates (FP32 above FP64)."""
    g = S.geometry_phase2()
    ctx = pipeline.make_context(g, S.default_params())
    f32 = ctx.probe_peak(0)
    f64 = ctx.probe_peak(1)
    assert 5.0 < f32 < 500.0, f32
    assert 0.01 < f64 < f32, (f64, f32)
    with pytest.raises(mkgb.MkgbError):
        ctx.probe_peak(2)
