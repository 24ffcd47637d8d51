"""Fused multigroup steps (ebof_multigroup_set_fused): every stage one launch
for the streams of all groups, whatever their resolutions, storage, patch
sizes and event counts (mode 1), or only the front-end stages fused and
the flow levels as per-group graph branches (mode 2).

The gate is bit identity: each stream's flow, edge counts and dropped-event
counts equal those of the same groups stepped with one launch per stage and
group (the default mode, itself bit-identical to single streams and tested
against them in test_gpu_groups.py, and through them against the oracle),
through graph replays of both parity patterns.  The fused step launches
fewer kernels.  Groups the fused kernels cannot run are refused.
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


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _group_flow(eb, g, k, prm):
    class _View:
        pass
    v = _View()
    v.__cuda_array_interface__ = {"shape": (2, prm.height, prm.width), "typestr": "<f4",
                                  "data": (eb.ebof_group_flow(g, k), False), "version": 3}
    return torch.as_tensor(v, device="cuda").cpu().numpy()


def _noisy_windows(W, H, nwin, n_events, seed):
    """Uniform events with 5 % outside the image or the window, as
    (x, y, t, t_begin, t_end) numpy windows."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(nwin):
        tb = k * synth.WINDOW_US
        x, y, t, _ = synth.random_edge_events(rng, W, H, n_events, t_begin=tb,
                                              out_of_range=0.05)
        order = np.argsort(t, kind="stable")
        out.append((x[order], y[order], t[order], tb, tb + synth.WINDOW_US))
    return out


def _stream_windows(ev, nwin):
    return [tuple(ev.window(k)[i] for i in (0, 1, 2, 4, 5)) for k in range(nwin)]


def _run(eb, specs, nwin, fused):
    """specs: list of (params, [windows of each stream]).  Steps the groups
    as one multigroup; returns per step and group the flows and stats, and
    the kernels launched per steady-state step."""
    groups = []
    for prm, streams in specs:
        st, g = eb.ebof_group_create(prm, len(streams), 0)
        eb.check(st)
        groups.append(g)
    st, mg = eb.ebof_multigroup_create(groups)
    eb.check(st)
    if fused:
        eb.check(eb.ebof_multigroup_set_fused(mg, fused))
    out, launches = [], []
    for k in range(nwin):
        wins = []
        for prm, streams in specs:
            wins.append([tuple(_dev(a) for a in w[k][:3]) + w[k][3:] for w in streams])
        before = eb.load().ebof_kernel_launches()
        r = eb.ebof_multigroup_process(mg, wins)
        launches.append(eb.load().ebof_kernel_launches() - before)
        assert r == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        torch.cuda.synchronize()
        step = []
        for g, (prm, streams) in zip(groups, specs):
            st, stats = eb.ebof_group_sync(g)
            eb.check(st)
            flows = [_group_flow(eb, g, i, prm) for i in range(len(streams))]
            counts = [(s.events, s.in_window, s.dropped_time, s.dropped_oob, s.edge_px,
                       s.levels_used, s.has_flow) for s in stats]
            step.append((flows, counts))
        out.append(step)
    mg.close()
    for g in groups:
        g.close()
    return out, launches


def _compare(a, b):
    for k, (sa, sb) in enumerate(zip(a, b)):
        for gi, ((fa, ca), (fb, cb)) in enumerate(zip(sa, sb)):
            assert ca == cb, (k, gi)
            for i, (x, y) in enumerate(zip(fa, fb)):
                assert np.array_equal(x, y), (k, gi, i)


def test_fused_step_equals_per_group_launches(eb):
    nwin = 5
    specs = []
    # 346x260, uneven event counts per stream, FP32, default patches
    prm = eb.ebof_default_params(346, 260)
    specs.append((prm, [_stream_windows(synth.translating_segments(
        n_windows=nwin, seed=90 + i, events_per_window=n), nwin)
        for i, n in enumerate((4000, 20000, 60000))]))
    # 1280x720, FP32, 12x12 patches, 5 levels
    prm = eb.ebof_default_params(1280, 720)
    specs.append((prm, [_stream_windows(synth.rigid_objects(
        n_windows=nwin, seed=95 + i, events=(40000, 120000)), nwin) for i in range(2)]))
    # 640x480, FP16 storage, 8x8 patches at stride 4
    prm = eb.ebof_default_params(640, 480)
    prm.storage = eb.EBOF_STORAGE_FP16
    prm.patch, prm.stride = 8, 4
    specs.append((prm, [_stream_windows(synth.rigid_objects(
        n_windows=nwin, width=640, height=480, n_edges=150, seed=97 + i,
        events=(20000, 60000)), nwin) for i in range(2)]))
    # 300x200 noise with dropped events; other variational and search settings
    prm = eb.ebof_default_params(300, 200)
    prm.var_outer, prm.var_sor, prm.gn_iters, prm.connectivity = 3, 3, 8, 4
    specs.append((prm, [_noisy_windows(300, 200, nwin, 9000, 99)]))
    ref, l_ref = _run(eb, specs, nwin, 0)
    got, l_got = _run(eb, specs, nwin, 1)
    _compare(ref, got)
    front, l_front = _run(eb, specs, nwin, 2)
    _compare(ref, front)
    print("kernels per steady step: per group %s, fused %s, front end fused %s"
          % (l_ref[2:], l_got[2:], l_front[2:]))
    assert max(l_got[2:]) < min(l_front[2:]) < min(l_ref[2:])


def test_fused_step_with_more_groups_than_a_table_holds(eb):
    """Nine groups of small and odd sizes, one a level too small for any
    patch (its flow is zero): the tables split at eight segments."""
    nwin = 4
    sizes = [(64, 48), (80, 60), (96, 72), (100, 50), (128, 96), (70, 90), (33, 47), (6, 6),
             (160, 120)]
    specs = []
    for i, (W, H) in enumerate(sizes):
        prm = eb.ebof_default_params(W, H)
        specs.append((prm, [_noisy_windows(W, H, nwin, max(50, W * H // 8), 200 + i)]))
    ref, _ = _run(eb, specs, nwin, 0)
    for mode in (1, 2):
        got, _ = _run(eb, specs, nwin, mode)
        _compare(ref, got)


def test_fused_mode_refuses_groups_it_cannot_run(eb):
    prm = eb.ebof_default_params(346, 260)
    prm.var_sor = 13  # more sweeps than a register-resident SOR region holds
    st, g = eb.ebof_group_create(prm, 1, 0)
    eb.check(st)
    st, mg = eb.ebof_multigroup_create([g])
    eb.check(st)
    assert eb.ebof_multigroup_set_fused(mg, 1) == eb.EBOF_ERR_UNSUPPORTED
    assert eb.ebof_multigroup_set_fused(mg, 2) == eb.EBOF_OK  # the flow stays per group
    assert eb.ebof_multigroup_set_fused(mg, 0) == eb.EBOF_OK
    assert eb.ebof_multigroup_set_fused(mg, 3) == eb.EBOF_ERR_INVALID_ARG
    mg.close()
    g.close()
    prm = eb.ebof_default_params(1280, 720)
    prm.levels, prm.patch, prm.stride = 7, 4, 2  # 7 levels: beyond the fused pyramid
    st, g = eb.ebof_group_create(prm, 1, 0)
    eb.check(st)
    st, mg = eb.ebof_multigroup_create([g])
    eb.check(st)
    assert eb.ebof_multigroup_set_fused(mg, True) == eb.EBOF_ERR_UNSUPPORTED
    mg.close()
    g.close()
