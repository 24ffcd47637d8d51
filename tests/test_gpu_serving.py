"""List calls and the serving loop on the GPU.

* ebof_process_window_list (n windows of arbitrary extents, graph-replayed
  per n) gives the same flow, bit for bit, as one ebof_process_window call
  per window.
* The server: windows of streams of three resolutions and both storage
  modes, submitted interleaved and batched by the dispatcher, give each
  stream exactly the flow it gets alone; streams beyond the memory budget
  wait, are admitted when another stream closes, and still match."""
import ctypes
import time

import numpy as np
import pytest

from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _windows(ev, n):
    out = []
    for k in range(n):
        x, y, t, _, tb, te = ev.window(k)
        out.append((_dev(x), _dev(y), _dev(t), tb, te))
    return out


def _alone(eb, prm, wins):
    """Flow of each window through single-window calls of a fresh stream."""
    p = eb.ebof_params()
    ctypes.memmove(ctypes.byref(p), ctypes.byref(prm), ctypes.sizeof(p))
    p.max_batch = 1
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st)
    W, H = p.width, p.height
    out = []
    for (x, y, t, tb, te) in wins:
        flow = torch.full((2, H, W), float("nan"), dtype=torch.float32, device="cuda")
        eb.check(eb.ebof_process_window(s, x, y, t, None, tb, te, flow))
        out.append(flow)
    torch.cuda.synchronize()
    out = [f.cpu() for f in out]
    s.close()
    return out


def _stream(kind, seed, n):
    if kind == "346x260":
        return synth.translating_segments(n_windows=n, seed=seed, velocity=(2.0, -1.0))
    if kind == "640x480":
        return synth.rigid_objects(width=640, height=480, n_windows=n, n_objects=6, n_edges=120,
                                   radius=(30.0, 120.0), events=(30_000, 90_000), seed=seed)
    return synth.rigid_objects(width=1280, height=720, n_windows=n, events=(60_000, 150_000),
                               seed=seed, lognormal_counts=True)


@pytest.mark.parametrize("storage", [0, 1])
def test_window_list_matches_single_windows(eb, storage):
    n = 12
    ev = _stream("346x260", 40 + storage, n)
    wins = _windows(ev, n)
    prm = eb.ebof_default_params(346, 260)
    prm.storage = storage
    prm.max_batch = 4
    ref = _alone(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    flows = [torch.full((2, 260, 346), float("nan"), device="cuda") for _ in range(n)]
    k = 0
    for m in (1, 3, 2, 4, 1, 1):  # graphs for n = 3, 2, 4, 1 captured, 1 replayed
        r = eb.ebof_process_window_list(s, wins[k:k + m], flows[k:k + m])
        assert r == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        k += m
    st, stats = eb.ebof_stream_sync(s, 1)
    eb.check(st)
    assert stats[0].events == wins[-1][0].numel()
    for i in range(n):
        assert torch.equal(flows[i].cpu(), ref[i]), "window %d" % i
    s.close()


def test_window_list_mixed_with_other_calls(eb):
    """List calls interleave with single-window and batched calls on one
    stream (the pyramid slots move between the call kinds)."""
    n = 10
    ev = _stream("346x260", 50, n)
    wins = _windows(ev, n)
    prm = eb.ebof_default_params(346, 260)
    prm.max_batch = 3
    ref = _alone(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    flows = [torch.full((2, 260, 346), float("nan"), device="cuda") for _ in range(n)]
    eb.check(eb.ebof_process_window_list(s, wins[0:2], flows[0:2]))
    x, y, t, tb, te = wins[2]
    eb.check(eb.ebof_process_window(s, x, y, t, None, tb, te, flows[2]))
    eb.check(eb.ebof_process_window_list(s, wins[3:6], flows[3:6]))
    # two consecutive windows as one batched call over their joined events
    xs = torch.cat([wins[6][0], wins[7][0]])
    ys = torch.cat([wins[6][1], wins[7][1]])
    ts = torch.cat([wins[6][2], wins[7][2]])
    f2 = torch.empty((2, 2, 260, 346), device="cuda")
    eb.check(eb.ebof_process_windows(s, 2, xs, ys, ts, None, wins[6][3], wins[6][4] - wins[6][3],
                                     f2))
    flows[6].copy_(f2[0])
    flows[7].copy_(f2[1])
    eb.check(eb.ebof_process_window_list(s, wins[8:10], flows[8:10]))
    torch.cuda.synchronize()
    for i in range(n):
        assert torch.equal(flows[i].cpu(), ref[i]), "window %d" % i
    s.close()


def test_window_list_degenerate(eb):
    """An image smaller than a patch has no pyramid level: zero flow for
    every window; empty windows are allowed."""
    prm = eb.ebof_default_params(7, 6)
    prm.max_batch = 2
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    e16 = torch.empty(0, dtype=torch.uint16, device="cuda")
    e64 = torch.empty(0, dtype=torch.int64, device="cuda")
    for rep in range(3):
        flows = [torch.full((2, 6, 7), float("nan"), device="cuda") for _ in range(2)]
        w = [(e16, e16, e64, 0, 10), (e16, e16, e64, 10, 20)]
        r = eb.ebof_process_window_list(s, w, flows)
        assert r >= 0
        for f in flows:
            assert torch.count_nonzero(f.cpu()) == 0
    with pytest.raises(ValueError):
        eb.ebof_process_window_list(s, w, flows[:1])
    assert eb.ebof_process_window_list(s, w * 2, flows * 2) == eb.EBOF_ERR_INVALID_ARG
    s.close()


def _serve(eb, server, streams, rng, pace_s=0.0):
    """Submits every stream's windows interleaved (random stream order, each
    stream's windows in order); returns {sid: [flow]} once all completed."""
    flows = {sid: [torch.full((2, p.height, p.width), float("nan"), device="cuda")
                   for _ in wins] for sid, (p, wins) in streams.items()}
    order = [sid for sid, (_, wins) in streams.items() for _ in wins]
    rng.shuffle(order)
    nxt = {sid: 0 for sid in streams}
    for sid in order:
        k = nxt[sid]
        nxt[sid] += 1
        r = eb.ebof_server_submit(server, sid, streams[sid][1][k], flows[sid][k], tag=k)
        assert r == eb.EBOF_OK
        if pace_s:
            time.sleep(pace_s * rng.random())
    return flows


def test_server_mix_matches_alone(eb):
    rng = np.random.default_rng(7)
    kinds = [("346x260", 0, 4), ("346x260", 1, 2), ("640x480", 1, 3), ("1280x720", 0, 2),
             ("640x480", 0, 1)]
    nwin = 6
    cfg = eb.ebof_server_default_config()
    cfg.n_workers = 3
    st, server = eb.ebof_server_create(cfg)
    eb.check(st)
    streams, refs = {}, {}
    for i, (kind, storage, mb) in enumerate(kinds):
        ev = _stream(kind, 60 + i, nwin)
        prm = eb.ebof_default_params(ev.width, ev.height)
        prm.storage = storage
        prm.max_batch = mb
        wins = _windows(ev, nwin)
        refs[i] = _alone(eb, prm, wins)
        r, sid = eb.ebof_server_open_stream(server, prm)
        assert r == eb.EBOF_OK
        streams[sid] = (prm, wins)
        refs[sid] = refs.pop(i)
    flows = _serve(eb, server, streams, rng, pace_s=0.0005)
    assert eb.ebof_server_drain(server, 120000) == eb.EBOF_OK
    comps = []
    while True:
        c = eb.ebof_server_poll(server, 256, 0)
        if not c:
            break
        comps += c
    assert len(comps) == len(streams) * nwin
    seen = {sid: [] for sid in streams}
    for c in comps:
        seen[c.stream_id].append(c.tag)
        assert c.status == (eb.EBOF_NO_PREVIOUS if c.tag == 0 else eb.EBOF_OK)
        assert 1 <= c.batch <= streams[c.stream_id][0].max_batch
        assert c.arrival_ns <= c.launch_ns <= c.done_ns
    for sid in streams:
        assert seen[sid] == list(range(nwin))  # per-stream completion order
        for k in range(nwin):
            assert torch.equal(flows[sid][k].cpu(), refs[sid][k]), "stream %d window %d" % (sid, k)
    info = eb.ebof_server_get_info(server)
    assert info.windows_completed == len(streams) * nwin
    assert info.streams_admitted == len(streams)
    server.close()


def test_server_admission_under_budget(eb):
    rng = np.random.default_rng(3)
    nwin = 4
    prm = eb.ebof_default_params(346, 260)
    prm.max_batch = 2
    one = eb.ebof_stream_device_bytes(prm)
    cfg = eb.ebof_server_default_config()
    cfg.memory_budget = 2 * one + one // 2  # room for two streams
    cfg.n_workers = 2
    st, server = eb.ebof_server_create(cfg)
    eb.check(st)
    streams, refs = {}, {}
    status = []
    for i in range(3):
        wins = _windows(_stream("346x260", 70 + i, nwin), nwin)
        r, sid = eb.ebof_server_open_stream(server, prm)
        status.append(r)
        streams[sid] = (prm, wins)
        refs[sid] = _alone(eb, prm, wins)
    assert status == [eb.EBOF_OK, eb.EBOF_OK, eb.EBOF_QUEUED]
    info = eb.ebof_server_get_info(server)
    assert (info.streams_admitted, info.streams_waiting) == (2, 1)
    assert info.memory_in_use == 2 * one
    flows = _serve(eb, server, streams, rng)
    sids = sorted(streams)
    # only the admitted streams run; then closing the first admits the third
    done = []
    t_end = time.time() + 60
    while len(done) < 2 * nwin and time.time() < t_end:
        done += eb.ebof_server_poll(server, 64, 1000)
    assert len(done) == 2 * nwin and all(c.stream_id != sids[2] for c in done)
    assert eb.ebof_server_close_stream(server, sids[0]) == eb.EBOF_OK
    assert eb.ebof_server_drain(server, 60000) == eb.EBOF_OK
    info = eb.ebof_server_get_info(server)
    assert (info.streams_admitted, info.streams_waiting) == (2, 0)
    for sid in sids:
        for k in range(nwin):
            assert torch.equal(flows[sid][k].cpu(), refs[sid][k]), "stream %d window %d" % (sid, k)
    too_big = eb.ebof_default_params(1280, 720)
    too_big.max_batch = 8
    assert eb.ebof_server_open_stream(server, too_big)[0] == eb.EBOF_ERR_OOM
    server.close()
