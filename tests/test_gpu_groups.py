"""Multi-stream groups: n camera streams of one resolution stepped in lockstep
(one launch per stage for all of them, replayed as a CUDA graph from the
second step); mixed resolutions as separate groups on concurrent CUDA
streams.  Each stream's flow must be bit-identical to a single ebof_stream
fed the same windows."""
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


def _single(eb, prm, ev, nwin):
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    W, H = prm.width, prm.height
    out = []
    for k in range(nwin):
        x, y, t, _, tb, te = ev.window(k)
        flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
        eb.check(eb.ebof_process_window(s, _dev(x), _dev(y), _dev(t), None, tb, te, flow))
        out.append(flow.cpu().numpy())
    s.close()
    return out


@pytest.mark.parametrize("storage", [0, 1])
def test_group_matches_single_streams_through_graph_replays(eb, storage):
    nwin, nstr = 4, 3
    W, H = 346, 260
    streams = [synth.translating_segments(n_windows=nwin, seed=20 + i,
                                          velocity=(1.0 + i, -0.5 * i)) for i in range(nstr)]
    prm = eb.ebof_default_params(W, H)
    prm.storage = storage
    st, g = eb.ebof_group_create(prm, nstr, 0)
    eb.check(st)
    got = []
    for k in range(nwin):
        wins = []
        for ev in streams:
            x, y, t, _, tb, te = ev.window(k)
            wins.append((_dev(x), _dev(y), _dev(t), tb, te))
        flow = torch.empty((nstr, 2, H, W), dtype=torch.float32, device="cuda")
        r = eb.ebof_group_process(g, wins, flow)
        assert r == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        torch.cuda.synchronize()
        got.append(flow.cpu().numpy())
        sst, stats = eb.ebof_group_sync(g)
        eb.check(sst)
        for i, ev in enumerate(streams):
            x, *_ = ev.window(k)
            assert stats[i].events == len(x) and stats[i].in_window == len(x)
    for i, ev in enumerate(streams):
        ref = _single(eb, prm, ev, nwin)
        for k in range(nwin):
            assert np.array_equal(got[k][i], ref[k]), (i, k)
    # the group's own buffer holds the last step
    assert eb.ebof_group_flow(g, 0) != 0
    assert eb.ebof_group_reset(g) == eb.EBOF_OK
    g.close()


def test_two_resolutions_on_concurrent_streams(eb):
    nwin = 3
    small = [synth.translating_segments(n_windows=nwin, seed=40 + i) for i in range(2)]
    big = [synth.rigid_objects(n_windows=nwin, seed=50, events=(20000, 40000), width=640,
                               height=360, n_edges=120)]
    groups, refs, outs = [], [], []
    for evs in (small, big):
        W, H = evs[0].width, evs[0].height
        prm = eb.ebof_default_params(W, H)
        st, g = eb.ebof_group_create(prm, len(evs), 0)
        eb.check(st)
        groups.append((g, evs, torch.cuda.Stream(), prm))
        refs.append([_single(eb, prm, ev, nwin) for ev in evs])
        outs.append([])
    for k in range(nwin):
        for gi, (g, evs, cs, prm) in enumerate(groups):
            wins = []
            for ev in evs:
                x, y, t, _, tb, te = ev.window(k)
                wins.append((_dev(x), _dev(y), _dev(t), tb, te))
            flow = torch.empty((len(evs), 2, prm.height, prm.width), dtype=torch.float32,
                               device="cuda")
            cs.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(cs):
                eb.check(eb.ebof_group_process(g, wins, flow))
            outs[gi].append((flow, cs, wins))  # keep the inputs alive until the sync
    torch.cuda.synchronize()
    for gi in range(2):
        for k in range(nwin):
            f = outs[gi][k][0].cpu().numpy()
            for i in range(len(groups[gi][1])):
                assert np.array_equal(f[i], refs[gi][i][k])
    for g, *_ in groups:
        g.close()
