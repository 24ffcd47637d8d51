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


def _group_flow(eb, g, k, prm):
    """Stream k's flow of the group's last step, read from the group's own
    buffer (ebof_group_flow) through a zero-copy view."""
    class _View:
        pass
    v = _View()
    v.__cuda_array_interface__ = {"shape": (2, prm.height, prm.width), "typestr": "<f4",
                                  "data": (eb.ebof_group_flow(g, k), False), "version": 3}
    return torch.as_tensor(v, device="cuda").cpu().numpy()


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


def test_multigroup_one_graph_matches_single_streams(eb):
    """Two resolutions stepped as one CUDA graph (each group's step a branch):
    every stream's flow bit-identical to a single stream fed the same
    windows, through the eager first step and graph replays of both parity
    patterns."""
    nwin = 5
    small = [synth.translating_segments(n_windows=nwin, seed=60 + i) for i in range(3)]
    big = [synth.rigid_objects(n_windows=nwin, seed=70 + i, events=(20000, 40000), width=640,
                               height=360, n_edges=120) for i in range(2)]
    groups, refs = [], []
    for evs in (small, big):
        prm = eb.ebof_default_params(evs[0].width, evs[0].height)
        st, g = eb.ebof_group_create(prm, len(evs), 0)
        eb.check(st)
        groups.append((g, evs, prm))
        refs.append([_single(eb, prm, ev, nwin) for ev in evs])
    st, mg = eb.ebof_multigroup_create([g for g, _, _ in groups])
    eb.check(st)
    keep = []
    for k in range(nwin):
        wins = []
        for g, evs, _ in groups:
            ws = []
            for ev in evs:
                x, y, t, _, tb, te = ev.window(k)
                ws.append((_dev(x), _dev(y), _dev(t), tb, te))
            wins.append(ws)
        keep.append(wins)
        r = eb.ebof_multigroup_process(mg, wins)
        assert r == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        torch.cuda.synchronize()
        for gi, (g, evs, prm) in enumerate(groups):
            eb.check(eb.ebof_group_sync(g)[0])
            for i in range(len(evs)):
                got = _group_flow(eb, g, i, prm)
                assert np.array_equal(got, refs[gi][i][k]), (gi, i, k)
    mg.close()
    for g, *_ in groups:
        g.close()


@pytest.mark.parametrize("knob,values", [("sor_tma_min_per_sm", (1, 2, 1 << 20)),
                                         ("sor_row_waves", (0, 2, 4)),
                                         ("coeff_cw_min_width", (160, 640, 1 << 20)),
                                         ("var_cluster_max", (2, 8, 16)),
                                         ("coeff_cw_rows", (4, 16))])
def test_layout_knobs_never_change_the_flow(eb, knob, values):
    """The variational layouts (the coefficient kernel's form, the SOR forms,
    the cluster-resident refinement of the small levels) tile the same
    computation differently: single and batched calls give the same flow bit
    for bit under every setting."""
    ev = synth.rigid_objects(n_windows=6, seed=80, events=(60000, 90000), width=1280,
                             height=720)
    W, H, n = 1280, 720, 5
    outs = []
    for v in (None,) + tuple(values):
        prm = eb.ebof_default_params(W, H)
        prm.max_batch = n
        if v is not None:
            setattr(prm, knob, v)
        st, s = eb.ebof_stream_create(prm, 0)
        eb.check(st)
        x, y, t, _, tb, te = ev.window(0)
        f0 = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
        eb.check(eb.ebof_process_window(s, _dev(x), _dev(y), _dev(t), None, tb, te, f0))
        a, b = int(ev.offsets[1]), int(ev.offsets[1 + n])
        flow = torch.empty((n, 2, H, W), dtype=torch.float32, device="cuda")
        eb.check(eb.ebof_process_windows(s, n, _dev(ev.x[a:b]), _dev(ev.y[a:b]),
                                         _dev(ev.t[a:b]), None, int(ev.t_begin[1]), ev.dt,
                                         flow))
        eb.check(eb.ebof_stream_sync(s, 1)[0])
        outs.append(flow.cpu().numpy())
        s.close()
    for v, o in zip(values, outs[1:]):
        assert np.array_equal(o, outs[0]), (knob, v)
