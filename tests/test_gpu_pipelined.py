"""Pipelined windows (ebof_process_window_async): a window's front end runs
on one internal stream, its flow on one of four flow streams in turn (each
with its own scratch buffers), over eight pyramid slots of the stream's own,
so that front ends and the flows of consecutive windows overlap.  The gate
is bit identity with ebof_process_window on the same windows (whose parity
with the oracle the other tests establish): every flow, through graph
replays of all eight slots, with FP16 storage, with
stage timing on (the eager path), mixed with ordinary calls on one stream
(the pyramid handed over both ways) and across a reset.
"""
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


def _windows(ev, n):
    out = []
    for k in range(n):
        x, y, t, _, tb, te = ev.window(k)
        out.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, t))
                   + (tb, te))
    return out


def _ordinary(eb, prm, wins):
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    out = []
    for x, y, t, tb, te in wins:
        f = torch.empty((2, prm.height, prm.width), dtype=torch.float32, device="cuda")
        eb.check(eb.ebof_process_window(s, x, y, t, None, tb, te, f))
        out.append(f)
    torch.cuda.synchronize()
    s.close()
    return [f.cpu().numpy() for f in out]


def _steps(eb, s, prm, wins, kinds):
    """kinds[k]: 'a' pipelined, 'o' ordinary; returns the statuses and flows."""
    flows, sts = [], []
    for (x, y, t, tb, te), kind in zip(wins, kinds):
        f = torch.full((2, prm.height, prm.width), float("nan"), dtype=torch.float32,
                       device="cuda")
        if kind == "a":
            r = eb.ebof_process_window_async(s, x, y, t, None, tb, te, f)
        else:
            r = eb.ebof_process_window(s, x, y, t, None, tb, te, f)
        eb.check(r)
        sts.append(r)
        flows.append(f)
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    torch.cuda.synchronize()
    return sts, [f.cpu().numpy() for f in flows]


@pytest.mark.parametrize("W,H,storage", [(1280, 720, 0), (346, 260, 1)])
def test_pipelined_equals_ordinary_calls(eb, W, H, storage):
    n = 18  # every slot and every flow stream more than once
    if W == 1280:
        ev = synth.rigid_objects(n_windows=n, seed=41, events=(60000, 150000))
    else:
        ev = synth.translating_segments(n_windows=n, seed=42)
    prm = eb.ebof_default_params(W, H)
    prm.storage = storage
    wins = _windows(ev, n)
    ref = _ordinary(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    sts, got = _steps(eb, s, prm, wins, "a" * n)
    assert sts[0] == eb.EBOF_NO_PREVIOUS and all(r == eb.EBOF_OK for r in sts[1:])
    for k in range(n):
        assert np.array_equal(got[k], ref[k]), k
    # the last window's counters, as after an ordinary call
    _, stats = eb.ebof_stream_sync(s, 1)
    assert stats[0].has_flow == 1 and stats[0].events == wins[-1][0].numel()
    s.close()


def test_pipelined_mixed_with_ordinary_calls_and_reset(eb):
    n = 9
    ev = synth.rigid_objects(n_windows=n, seed=43, events=(40000, 90000), width=640,
                             height=360, n_edges=120)
    prm = eb.ebof_default_params(640, 360)
    wins = _windows(ev, n)
    ref = _ordinary(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    # ordinary -> pipelined -> ordinary -> pipelined hand-overs
    kinds = "ooaaoaaao"
    sts, got = _steps(eb, s, prm, wins, kinds)
    assert sts[0] == eb.EBOF_NO_PREVIOUS
    for k in range(n):
        assert np.array_equal(got[k], ref[k]), (k, kinds[k])
    # after a reset the pipeline starts again with no previous window
    assert eb.ebof_stream_reset(s) == eb.EBOF_OK
    sts, got = _steps(eb, s, prm, wins[:4], "aaaa")
    assert sts[0] == eb.EBOF_NO_PREVIOUS
    for k in range(4):
        assert np.array_equal(got[k], ref[k]), k
    s.close()


def test_pipelined_with_stage_timing(eb):
    """Stage timing on: the front ends and flows are enqueued eagerly on the
    pipeline's streams instead of replayed from graphs; the same flows, and
    every stage shows up in the profile."""
    n = 5
    ev = synth.translating_segments(n_windows=n, seed=44)
    prm = eb.ebof_default_params(346, 260)
    wins = _windows(ev, n)
    ref = _ordinary(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    eb.check(eb.ebof_stream_set_profiling(s, True))
    _, got = _steps(eb, s, prm, wins, "a" * n)
    for k in range(n):
        assert np.array_equal(got[k], ref[k]), k
    _, prof = eb.ebof_stream_get_profile(s)
    for stage in ("scatter", "edt_rows_surface", "pyramid", "patch_search", "var_sor",
                  "flow_out"):
        assert prof[stage][1] > 0, stage
    s.close()


def test_pipelined_calls_sharing_one_flow_buffer(eb):
    """Every window into the same flow buffer: the writes follow the call
    order, so the buffer ends with the newest window's flow."""
    n = 7
    ev = synth.rigid_objects(n_windows=n, seed=45, events=(60000, 150000))
    prm = eb.ebof_default_params(1280, 720)
    wins = _windows(ev, n)
    ref = _ordinary(eb, prm, wins)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    f = torch.full((2, 720, 1280), float("nan"), dtype=torch.float32, device="cuda")
    for x, y, t, tb, te in wins:
        eb.check(eb.ebof_process_window_async(s, x, y, t, None, tb, te, f))
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    torch.cuda.synchronize()
    assert np.array_equal(f.cpu().numpy(), ref[-1])
    s.close()



@pytest.mark.parametrize("W,H", [(160, 120), (6, 6)])
def test_pipelined_empty_windows_and_images_without_levels(eb, W, H):
    """A window without events between windows with events, and an image
    smaller than the patch (no pyramid level: the flow is zero): the same
    flows as ordinary calls, with a non-default max_batch (more ordinary
    slots) in the mix."""
    n = 6
    rng = np.random.default_rng(W)
    wins = []
    for k in range(n):
        tb = k * synth.WINDOW_US
        m = 0 if k == 2 else max(20, W * H // 6)
        x, y, t, _ = synth.random_edge_events(rng, W, H, m, t_begin=tb)
        order = np.argsort(t, kind="stable")
        wins.append(tuple(torch.from_numpy(np.ascontiguousarray(a[order])).cuda()
                          for a in (x, y, t)) + (tb, tb + synth.WINDOW_US))
    prm = eb.ebof_default_params(W, H)
    ref = _ordinary(eb, prm, wins)
    prm.max_batch = 3
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    sts, got = _steps(eb, s, prm, wins, "oaaaoa")
    for k in range(n):
        assert np.array_equal(got[k], ref[k]), k
    if W == 6:
        assert all(np.all(g == 0.0) for g in got)
    s.close()
