"""The serving loop (tkf_server_*): every event's result is the same when it runs alone, in a
mixed continuous batch, and through the plain pipeline; the host queue admits by its byte
budget; unreleased results hold back new batches once they fill the result memory; polling,
release and timestamps behave as documented."""
import time

import numpy as np
import pytest

from _gpu import device_hits
from synth import Detector, EventSpec, event_sizes, generate

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from paper_1702_06359_gb300 import tkf  # noqa: E402


def _events(seed, n_events=12, det=Detector()):
    sizes, noise = event_sizes(seed, n_events, median=800, lo=100, hi=4000)
    b = generate(EventSpec(seed=seed, n_events=n_events, n_tracks=sizes, noise_frac=noise), det)
    evs = []
    for e in range(n_events):
        h0, h1 = b.hit_off[e], b.hit_off[e + 1]
        t0, t1 = b.trk_off[e], b.trk_off[e + 1]
        evs.append(tkf.HostEvent(b.x[h0:h1], b.y[h0:h1], b.z[h0:h1], b.var_u[h0:h1], b.var_v[h0:h1], b.layer[h0:h1],
                                 (b.trk_hits[t0:t1, :3] - h0).T))
    return b, evs


def _wait(sv, ticket):
    code, r = sv.poll(ticket, timeout_us=10_000_000)
    assert code == tkf.OK and r["status"] == tkf.OK
    return r


def test_result_is_the_same_alone_and_in_the_mix():
    b, evs = _events(71)
    sv = tkf.Server(n_slots=1, max_batch_events=16, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    code, t = sv.submit(evs[5])
    assert code == tkf.OK
    alone = _wait(sv, t)
    sv.release(t)
    tickets = []
    for ev in evs:  # submitted back to back: the queue fills while the slot is busy
        code, t = sv.submit(ev)
        assert code == tkf.OK
        tickets.append(t)
    results = [_wait(sv, t) for t in tickets]
    st = sv.stats()
    assert st["events_done"] == len(evs) + 1 and st["max_batch_events"] >= 2
    mixed = results[5]
    for k in ("par", "cov", "chi2", "nhits", "hit_idx"):
        assert np.array_equal(mixed[k], alone[k]), k
    for r in results:
        assert r["t_submit_ns"] <= r["t_start_ns"] <= r["t_done_ns"]
    # the same event through the plain pipeline on its own
    e = 5
    h0, h1 = b.hit_off[e], b.hit_off[e + 1]
    t0, t1 = b.trk_off[e], b.trk_off[e + 1]
    one = b
    ctx = tkf.Context(tkf.default_config())
    dh = device_hits(one)
    dh = tkf.DeviceHits(dh.x[h0:h1], dh.y[h0:h1], dh.z[h0:h1], dh.var_u[h0:h1], dh.var_v[h0:h1], dh.layer[h0:h1],
                        torch.tensor([0, h1 - h0], dtype=torch.int32, device="cuda"))
    sh = torch.as_tensor(np.ascontiguousarray((b.trk_hits[t0:t1, :3] - h0).T), dtype=torch.int32, device="cuda")
    se = torch.zeros(t1 - t0, dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, h1 - h0, 1, t1 - t0, use_graph=False)
    pipe.run(dh, sh, se, t1 - t0)
    torch.cuda.synchronize()
    _, built, fitted = pipe.outputs()
    ft = tkf.tracks_tensors(fitted, 10)
    bt = tkf.tracks_tensors(built, 10)
    assert np.array_equal(ft["par"].cpu().numpy(), alone["par"])
    hid = bt["hit_idx"].cpu().numpy()
    assert np.array_equal(hid, alone["hit_idx"])
    for t in tickets:
        assert sv.release(t) == tkf.OK
    assert sv.release(tickets[0]) == tkf.ERR_INVALID
    sv.close()


def test_batches_overlap_on_the_device_and_each_result_equals_its_alone_run():
    """Continuous batching with three slots of two events: twelve events of 1500-6000 tracks
    submitted together run as several batches in flight at once -- at least two batches' launch-to-completion host
    intervals intersect, and so do their device intervals (CUDA event times from before the
    first input copy to after the last result copy on each slot's stream) -- and every event's
    result is bit for bit the one it gets alone (one event per batch, one slot)."""
    # events of 1500-6000 tracks: a batch of two keeps the GPU busy for a few tenths of a
    # millisecond, longer than the host takes to launch the next slot's batch
    sizes, noise = event_sizes(74, 12, median=3000, lo=1500, hi=6000)
    b = generate(EventSpec(seed=74, n_events=12, n_tracks=sizes, noise_frac=noise), Detector())
    evs = []
    for e in range(b.n_events):
        h0, h1 = b.hit_off[e], b.hit_off[e + 1]
        t0, t1 = b.trk_off[e], b.trk_off[e + 1]
        evs.append(tkf.HostEvent(b.x[h0:h1], b.y[h0:h1], b.z[h0:h1], b.var_u[h0:h1], b.var_v[h0:h1], b.layer[h0:h1],
                                 (b.trk_hits[t0:t1, :3] - h0).T))
    sv1 = tkf.Server(n_slots=1, max_batch_events=1, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    alone = []
    for ev in evs:
        code, t = sv1.submit(ev)
        assert code == tkf.OK
        alone.append(_wait(sv1, t))
        sv1.release(t)
    sv1.close()
    sv = tkf.Server(n_slots=3, max_batch_events=2, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    arr = (tkf.Event * len(evs))(*[ev.struct for ev in evs])
    code, tickets = sv.submit_many(arr)
    assert code == tkf.OK and len(tickets) == len(evs)
    results = [_wait(sv, t) for t in tickets]
    for r, r0 in zip(results, alone):
        for k in ("par", "cov", "chi2", "nhits", "hit_idx"):
            assert np.array_equal(r[k], r0[k]), k
    batches = {}
    for r in results:
        assert r["gpu_start_ms"] >= 0 and r["gpu_done_ms"] >= r["gpu_start_ms"]
        batches[(r["t_start_ns"], r["gpu_start_ms"])] = (r["t_start_ns"], r["t_done_ns"], r["gpu_start_ms"],
                                                         r["gpu_done_ms"])
    iv = sorted(batches.values())
    assert len(iv) >= len(evs) // 2 - 1
    host = [(a, c) for a in range(len(iv)) for c in range(a + 1, len(iv))
            if iv[a][0] < iv[c][1] and iv[c][0] < iv[a][1]]
    dev = [(a, c) for a, c in host if iv[a][2] < iv[c][3] and iv[c][2] < iv[a][3]]
    assert host, "no two batches were in flight at once"
    assert dev, "no two batches overlapped on the device"
    for t in tickets:
        sv.release(t)
    sv.close()


def test_borrowed_inputs_give_the_same_results():
    b, evs = _events(73, n_events=6)
    sv = tkf.Server(n_slots=2, max_batch_events=8, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    ref = []
    for ev in evs:
        code, t = sv.submit(ev)
        ref.append(_wait(sv, t))
        sv.release(t)
    lent = []
    for e, ev in enumerate(evs):
        a = ev.arrays
        lent.append(tkf.HostEvent(a[0], a[1], a[2], a[3], a[4], a[5], a[6], borrow=True))
    tickets = [sv.submit(ev)[1] for ev in lent]
    for t, r0 in zip(tickets, ref):
        r = _wait(sv, t)
        for k in ("par", "cov", "chi2", "nhits", "hit_idx"):
            assert np.array_equal(r[k], r0[k]), k
        sv.release(t)
    sv.close()


def test_admission_polling_and_errors():
    b, evs = _events(72, n_events=3)
    ev_bytes = len(evs[0].arrays[0]) * 24 + evs[0].arrays[6].shape[1] * 12  # copied (not borrowed) events
    sv = tkf.Server(n_slots=1, max_batch_events=4, max_batch_hits=1 << 20, max_batch_tracks=1 << 16,
                    queue_bytes=ev_bytes - 1)
    code, _ = sv.submit(evs[0])
    assert code == tkf.ERR_AGAIN  # does not fit the host queue budget
    assert sv.stats()["rejected"] == 1
    sv.close()
    sv = tkf.Server(n_slots=2, max_batch_events=4, max_batch_hits=1000, max_batch_tracks=1 << 16)
    code, _ = sv.submit(evs[0])
    assert code == tkf.ERR_INVALID  # larger than a batch
    code, _ = sv.poll(12345)
    assert code == tkf.ERR_INVALID
    sv.close()
    sv = tkf.Server(n_slots=2, max_batch_events=4, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    code, t = sv.submit(evs[1])
    assert code == tkf.OK
    code, _ = sv.poll(t, timeout_us=0, copy=False)
    assert code in (tkf.OK, tkf.ERR_NOTREADY)
    r = _wait(sv, t)
    assert r["n_tracks"] == evs[1].arrays[6].shape[1]
    assert np.all(r["nhits"] > 0)
    sv.close()


def test_unreleased_results_hold_back_new_batches():
    b, evs = _events(74, n_events=10)
    T = 4096
    sv = tkf.Server(n_slots=1, max_batch_events=1, max_batch_hits=1 << 20, max_batch_tracks=T,
                    result_bytes=T * (29 + 10) * 4)  # room for one full-size batch only
    tickets = [sv.submit(ev)[1] for ev in evs]
    done, blocked = [], None
    for t in tickets:
        code, _ = sv.poll(t, timeout_us=500_000, copy=False)
        if code == tkf.ERR_TIMEOUT:
            blocked = t
            break
        assert code == tkf.OK
        done.append(t)
    assert blocked is not None and len(done) >= 1  # ten events need more than the budget
    for t in done:
        assert sv.release(t) == tkf.OK
    for t in tickets[len(done):]:
        r = _wait(sv, t)
        assert r["n_tracks"] > 0
        sv.release(t)
    assert sv.stats()["events_done"] == len(evs)
    sv.close()


def test_batch_submit_wait_release_match_single_calls():
    import ctypes as C
    b, evs = _events(75, n_events=8)
    sv = tkf.Server(n_slots=2, max_batch_events=4, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    single = []
    for ev in evs:
        code, t = sv.submit(ev)
        single.append(_wait(sv, t))
        sv.release(t)
    arr = (tkf.Event * len(evs))(*[ev.struct for ev in evs])
    code, tickets = sv.submit_many(arr)
    assert code == tkf.OK and len(tickets) == len(evs)
    code, res = sv.wait_all(tickets, timeout_us=10_000_000)
    assert code == tkf.OK
    for r, ref in zip(res, single):
        assert r.status == tkf.OK and r.n_tracks == ref["n_tracks"]
        n, st = r.n_tracks, r.stride
        par = np.ctypeslib.as_array(C.cast(r.par, C.POINTER(C.c_float)), shape=(5 * st + n,))
        assert np.array_equal(np.stack([par[k * st:k * st + n] for k in range(6)]), ref["par"])
    assert sv.release_many(tickets) == tkf.OK
    assert sv.release_many(tickets[:1]) == tkf.ERR_INVALID  # already released
    sv.close()


@pytest.mark.parametrize("prec,module_dr", [(tkf.MIXED, 0.0), (tkf.FP32, 1.0)], ids=["mixed", "two_step"])
def test_server_equals_the_pipeline_of_its_configuration(prec, module_dr):
    """The server's results equal the plain pipeline's under the same configuration, bit for bit:
    MIXED precision, and hits on modules 0.5 cm off the layers' cylinders (hit_dr = 0.5 cm)."""
    b, evs = _events(76, n_events=3, det=Detector(module_dr=module_dr))
    kw = dict(precision=prec, hit_dr=0.5 * module_dr)
    cfg = tkf.default_config(**kw)
    sv = tkf.Server(cfg, n_slots=2, max_batch_events=4, max_batch_hits=1 << 20, max_batch_tracks=1 << 16)
    tickets = [sv.submit(ev)[1] for ev in evs]
    res = [_wait(sv, t) for t in tickets]
    sv.release_many(tickets)
    sv.close()
    e = 1
    h0, h1, t0, t1 = b.hit_off[e], b.hit_off[e + 1], b.trk_off[e], b.trk_off[e + 1]
    ctx = tkf.Context(tkf.default_config(**kw))
    dh = device_hits(b)
    dh = tkf.DeviceHits(dh.x[h0:h1], dh.y[h0:h1], dh.z[h0:h1], dh.var_u[h0:h1], dh.var_v[h0:h1], dh.layer[h0:h1],
                        torch.tensor([0, h1 - h0], dtype=torch.int32, device="cuda"))
    sh = torch.as_tensor(np.ascontiguousarray((b.trk_hits[t0:t1, :3] - h0).T), dtype=torch.int32, device="cuda")
    pipe = tkf.DevicePipeline(ctx, h1 - h0, 1, t1 - t0, use_graph=False)
    pipe.run(dh, sh, torch.zeros(t1 - t0, dtype=torch.int32, device="cuda"), t1 - t0)
    torch.cuda.synchronize()
    _, built, fitted = pipe.outputs()
    assert np.array_equal(tkf.tracks_tensors(fitted, 10)["par"].cpu().numpy()[:, :t1 - t0], res[e]["par"])
    assert np.array_equal(tkf.tracks_tensors(built, 10)["hit_idx"].cpu().numpy()[:, :t1 - t0], res[e]["hit_idx"])
    pipe.close()
