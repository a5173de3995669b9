"""The batched pipeline (tkf_pipeline_*) and the work-tile autotuner: a CUDA-graph replay of
the whole step gives exactly the results of the direct call sequence, replays reuse one
capture, and building results do not depend on how seeds are split into work tiles."""
import numpy as np
import pytest

from _gpu import device_hits
from synth import Detector, EventSpec, event_sizes, generate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402


def _batch(seed, n_events=8, det=Detector()):
    sizes, noise = event_sizes(seed, n_events, median=600, lo=50, hi=3000)
    return generate(EventSpec(seed=seed, n_events=n_events, n_tracks=sizes, noise_frac=noise), det)


def _direct(ctx, b, dh, sh, se):
    """The pipeline's step as separate C-ABI calls."""
    L = ctx.cfg.n_layers
    n = b.n_tracks
    seeds = tkf.DeviceTracks.empty(n, L)
    built = tkf.DeviceTracks.empty(n, L)
    final = tkf.DeviceTracks.empty(n, L)
    idx = ctx.build_hit_index(dh)
    ctx.seed_fit(dh, sh, 2, seeds)
    seeds.event = se
    ctx.build_tracks(idx, seeds, built)
    ctx.fit(dh, seeds, 3, L - 1, final, hit_idx=built.hit_idx, continue_fit=True)
    ctx.sync_status()
    return built, final


def _pipe_out(pipe, L, n):
    _, built, fitted = pipe.outputs()
    bt = tkf.tracks_tensors(built, L)
    ft = tkf.tracks_tensors(fitted, L)
    return ({k: v[..., :n].clone() for k, v in bt.items()}, {k: v[..., :n].clone() for k, v in ft.items()})


def test_graph_replay_equals_direct_calls():
    b = _batch(61)
    b2 = _batch(62)
    # same sizes for the in-place update below
    n = min(b.n_tracks, b2.n_tracks)
    ctx = tkf.Context(tkf.default_config())
    L = ctx.cfg.n_layers
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    se = torch.as_tensor(b.trk_event, dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, max(b.n_hits, b2.n_hits), b.n_events, b.n_tracks, use_graph=True)
    for _ in range(3):
        pipe.run(dh, sh, se, b.n_tracks)
    torch.cuda.synchronize()
    ctx.sync_status()
    assert pipe.captures() == 1
    gb, gf = _pipe_out(pipe, L, b.n_tracks)
    db, df = _direct(ctx, b, dh, sh, se)
    assert torch.equal(gb["hit_idx"], db.hit_idx)
    assert torch.equal(gb["par"], db.par) and torch.equal(gb["chi2"], db.chi2) and torch.equal(gb["nhits"], db.nhits)
    assert torch.equal(gf["par"], df.par) and torch.equal(gf["cov"], df.cov) and torch.equal(gf["chi2"], df.chi2)
    assert pipe.build_ms() > 0
    # new data in the same buffers: the replay (no new capture) follows the data
    b2x = device_hits(b2)
    m = min(b.n_hits, b2.n_hits)
    for k in ("x", "y", "z", "var_u", "var_v", "layer"):
        getattr(dh, k)[:m].copy_(getattr(b2x, k)[:m])
    pipe.run(dh, sh, se, b.n_tracks)
    torch.cuda.synchronize()
    assert pipe.captures() == 1
    gb2, _ = _pipe_out(pipe, L, b.n_tracks)
    db2, _ = _direct(ctx, b, dh, sh, se)
    assert torch.equal(gb2["hit_idx"], db2.hit_idx) and torch.equal(gb2["par"], db2.par)
    assert not torch.equal(gb2["par"], gb["par"])
    del n


@pytest.mark.parametrize("prec", [tkf.FP32, tkf.MIXED], ids=["fp32", "mixed"])
def test_results_do_not_depend_on_the_work_tile(prec):
    """The same hit lists and parameters bit for bit for every work tile.  In MIXED a block's
    updates run packed into whichever of its warps the rotation picks, and the tile decides which
    seeds share a block: the packing must not change any result."""
    b = _batch(63, n_events=12)
    ctx = tkf.Context(tkf.default_config(precision=prec))
    L = ctx.cfg.n_layers
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    se = torch.as_tensor(b.trk_event, dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, b.n_tracks, use_graph=True)
    pipe.run(dh, sh, se, b.n_tracks)
    ref_b, ref_f = _pipe_out(pipe, L, b.n_tracks)
    seeds, _, _ = pipe.outputs()

    class _T:
        def struct(self):
            return seeds
    out = tkf.DeviceTracks.empty(b.n_tracks, L, prec)
    tiles = [1, 5, 10, 37, 128]
    best, ms = ctx.autotune_build(pipe.index(), _T(), out, tiles, repeats=2)
    assert best in tiles and len(ms) == len(tiles) and all(x > 0 for x in ms)
    assert ctx.config().seeds_per_block == best
    for tile in tiles:
        c2 = tkf.Context(tkf.default_config(seeds_per_block=tile, precision=prec))
        p2 = tkf.DevicePipeline(c2, b.n_hits, b.n_events, b.n_tracks, use_graph=True)
        p2.run(dh, sh, se, b.n_tracks)
        gb, gf = _pipe_out(p2, L, b.n_tracks)
        assert torch.equal(gb["hit_idx"], ref_b["hit_idx"]) and torch.equal(gb["par"], ref_b["par"]), tile
        assert torch.equal(gf["par"], ref_f["par"]), tile
        p2.close()


@pytest.mark.parametrize("prec", [tkf.MIXED, tkf.FP64], ids=["mixed", "fp64"])
def test_graph_replay_equals_direct_calls_other_precisions(prec):
    b = _batch(64, n_events=6)
    ctx = tkf.Context(tkf.default_config(precision=prec))
    L, n = ctx.cfg.n_layers, b.n_tracks
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    se = torch.as_tensor(b.trk_event, dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, n, use_graph=True)
    for _ in range(2):
        pipe.run(dh, sh, se, n)
    ctx.sync_status()
    assert pipe.captures() == 1
    _, built, fitted = pipe.outputs()
    gb, gf = tkf.tracks_tensors(built, L, prec), tkf.tracks_tensors(fitted, L, prec)
    seeds, db, df = (tkf.DeviceTracks.empty(n, L, prec) for _ in range(3))
    idx = ctx.build_hit_index(dh)
    ctx.seed_fit(dh, sh, 2, seeds)
    seeds.event = se
    ctx.build_tracks(idx, seeds, db)
    ctx.fit(dh, seeds, 3, L - 1, df, hit_idx=db.hit_idx, continue_fit=True)
    ctx.sync_status()
    assert torch.equal(gb["hit_idx"][:, :n], db.hit_idx[:, :n])
    assert torch.equal(gf["par"][:, :n], df.par[:, :n]) and torch.equal(gf["cov"][:, :n], df.cov[:, :n])
    pipe.close()


@pytest.mark.parametrize("prec", [tkf.FP32, tkf.FP64], ids=["fp32", "fp64"])
def test_seed_fit_and_continued_fit_agree_with_the_separate_calls(prec):
    """tkf_seed_fit equals tkf_seed_state + tkf_fit, and a fit continued over layers 3..9 from
    the seed fit equals one fit over 0..9, within rounding of the fused arithmetic (bit for
    bit is not promised: the compiler may fuse multiply-adds differently in the two kernels).
    In FP32 each form carries its own rounding error against the exact fit, up to about 5e-5
    relative in q/pT on the precision sweep, so two forms may differ by the parity tolerance
    (1e-4) on a few tracks (up to 2e-5 here); nearly all tracks agree far closer (99 % within
    1e-5), which a dropped layer, update or scattering term would not give."""
    from _gpu import CHI2_REL, PAR_FLOOR, PAR_REL
    b = _batch(65, n_events=4)
    ctx = tkf.Context(tkf.default_config(precision=prec))
    L, n = ctx.cfg.n_layers, b.n_tracks
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    hid = torch.as_tensor(np.ascontiguousarray(b.trk_hits.T), dtype=torch.int32, device="cuda")
    init, sep, fused, full, cont = (tkf.DeviceTracks.empty(n, L, prec) for _ in range(5))
    ctx.seed_state(dh, sh, init)
    ctx.fit(dh, init, 0, 2, sep)
    ctx.seed_fit(dh, sh, 2, fused)
    ctx.fit(dh, init, 0, L - 1, full, hit_idx=hid)
    ctx.fit(dh, fused, 3, L - 1, cont, hit_idx=hid, continue_fit=True)
    ctx.sync_status()
    rel = PAR_REL if prec == tkf.FP32 else 1e-12
    floor = torch.as_tensor(PAR_FLOOR, device="cuda", dtype=sep.par.dtype)[:, None]
    for a_, b_ in ((sep, fused), (full, cont)):
        assert torch.equal(a_.nhits, b_.nhits)
        d = (a_.par - b_.par).abs() / torch.maximum(a_.par.abs(), floor)
        d[4] = torch.remainder(d[4] + np.pi, 2 * np.pi) - np.pi
        assert float(d.abs().max()) < rel
        if prec == tkf.FP32:
            assert float(torch.quantile(d.abs().max(dim=0).values.double(), 0.99)) < 1e-5
        dc = (a_.chi2 - b_.chi2).abs() / torch.clamp(a_.chi2.abs(), min=1.0)
        assert float(dc.max()) < (CHI2_REL if prec == tkf.FP32 else 1e-11)
    assert torch.equal(fused.hit_idx[:3], sh) and bool((fused.hit_idx[3:] == -1).all())


def test_backward_stage_equals_the_separate_call():
    """tkf_pipeline_set_backward adds the backward pass as the step's last stage: its states on
    layer 1 equal tkf_fit_backward on the pipeline's own fitted tracks (the same kernel, bit for
    bit), in the graph and with direct launches; enabling and disabling each capture anew."""
    b = _batch(64)
    n = b.n_tracks
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    se = torch.as_tensor(b.trk_event, dtype=torch.int32, device="cuda")

    class _Raw:
        def __init__(self, t):
            self.t = t

        def struct(self):
            return self.t
    for use_graph in (True, False):
        ctx = tkf.Context(tkf.default_config())
        L = ctx.cfg.n_layers
        pipe = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, n, use_graph=use_graph)
        with pytest.raises(tkf.TkfError):
            pipe.backward_outputs()  # no backward stage yet
        pipe.run(dh, sh, se, n)
        pipe.set_backward(1e4)
        for _ in range(2):
            pipe.run(dh, sh, se, n)
        torch.cuda.synchronize()
        ctx.sync_status()
        if use_graph:
            assert pipe.captures() == 2
        got = tkf.tracks_tensors(pipe.backward_outputs(), L)
        _, built, fitted = pipe.outputs()
        ref = tkf.DeviceTracks.empty(n, L)
        ctx.fit_backward(dh, _Raw(fitted), L - 1, 0, ref, cov_scale=1e4, hit_idx=tkf.tracks_tensors(built, L)["hit_idx"])
        ctx.sync_status()
        assert torch.equal(got["par"][:, :n], ref.par) and torch.equal(got["cov"][:, :n], ref.cov)
        assert torch.equal(got["chi2"][:n], ref.chi2) and torch.equal(got["nhits"][:n], ref.nhits)
        pipe.set_backward(0)
        pipe.run(dh, sh, se, n)
        if use_graph:
            assert pipe.captures() == 3
        with pytest.raises(tkf.TkfError):
            pipe.set_backward(-1.0)
        pipe.close()
        ctx.close()


def test_two_step_pipeline_equals_direct_calls():
    """Hits on modules off the layers' cylinders (hit_dr = 0.5 cm): the graph step equals the
    same calls made one by one, bit for bit, and its builds keep most tracks' own hits."""
    b = _batch(63, det=Detector(module_dr=1.0))
    ctx = tkf.Context(tkf.default_config(hit_dr=0.5))
    L = ctx.cfg.n_layers
    dh = device_hits(b)
    sh = torch.as_tensor(np.ascontiguousarray(b.trk_hits[:, :3].T), dtype=torch.int32, device="cuda")
    se = torch.as_tensor(b.trk_event, dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, b.n_hits, b.n_events, b.n_tracks, use_graph=True)
    for _ in range(2):
        pipe.run(dh, sh, se, b.n_tracks)
    torch.cuda.synchronize()
    ctx.sync_status()
    gb, gf = _pipe_out(pipe, L, b.n_tracks)
    db, df = _direct(ctx, b, dh, sh, se)
    assert torch.equal(gb["hit_idx"], db.hit_idx) and torch.equal(gb["par"], db.par)
    assert torch.equal(gf["par"], df.par) and torch.equal(gf["cov"], df.cov) and torch.equal(gf["chi2"], df.chi2)
    ids = gb["hit_idx"].T.cpu().numpy()  # global hit ids
    assert np.all(ids == b.trk_hits, axis=1).mean() >= 0.97
    pipe.close()
    ctx.close()
