"""GPU path vs the FP64 oracle, through the C ABI (needs a GB300).

Gates: edge image and squared EDT bit-exact; surface d_exp within 1e-5
absolute; flow within 0.05 px mean endpoint error of the oracle's flow.
Inputs are seeded synthetic event streams and analytic surfaces.
"""
import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

SURF_TOL = 1e-5
EPE_TOL = 0.05
# p99 of the per-pixel endpoint error on the 1280x720 workload.  DIS is
# chaotic at a few pixels per frame (a patch whose Gauss-Newton path crosses
# the reset radius on one side only moves its neighbourhood by up to a
# pixel), so the tail is wider than the mean; the bar is set from the
# measured GPU-oracle p99 of these frames with a margin.
EPE_P99_TOL = 1.0
# FP16 storage (surfaces, pyramid, gradients as __half): the gate of the
# FP16 tests
FP16_EPE_TOL = 0.06

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def make_stream(eb, W, H, **kw):
    p = eb.ebof_default_params(W, H)
    for k, v in kw.items():
        setattr(p, k, v)
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st, "create")
    return p, s


def run_window(eb, s, x, y, t, tb, te, p=None):
    W, H = s.params.width, s.params.height
    flow = torch.full((2, H, W), float("nan"), dtype=torch.float32, device="cuda:0")
    edge = torch.empty((H, W), dtype=torch.uint8, device="cuda:0")
    edt = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
    surf = torch.empty((H, W), dtype=torch.float32, device="cuda:0")
    pt = dev(p) if p is not None else None
    st = eb.ebof_process_window(s, dev(x), dev(y), dev(t), pt, tb, te, flow, edge, edt, surf)
    eb.check(st, "process_window")
    sst, stats = eb.ebof_stream_sync(s, 1)
    eb.check(sst, "sync")
    return dict(status=st, stats=stats[0], flow=flow.cpu().numpy(), edge=edge.cpu().numpy(),
                edt=edt.cpu().numpy(), surf=surf.cpu().numpy())


def run_k(eb, s, ev, k):
    x, y, t, p, tb, te = ev.window(k)
    return run_window(eb, s, x, y, t, tb, te, p)


def oracle_surface(prm, W, H, x, y, t, tb, te):
    return oracle.surface_from_events(W, H, x, y, t, tb, te, connectivity=prm.connectivity,
                                      n_d=prm.n_d, n_f=prm.n_f, alpha=float(prm.alpha))


def oracle_flow(prm, I0, I1):
    return oracle.flow(I0, I1, levels=prm.levels, patch=prm.patch, stride=prm.stride,
                       gn_iters=prm.gn_iters, gn_damping=float(prm.gn_damping),
                       var_outer=prm.var_outer, var_sor=prm.var_sor,
                       var_delta=float(prm.var_delta), var_gamma=float(prm.var_gamma),
                       var_alpha=float(prm.var_alpha), sor_omega=float(prm.sor_omega))


def epe(a, b):
    return np.hypot(a[0] - b[0], a[1] - b[1])


def check_front(g, o, tag=""):
    assert np.array_equal(g["edge"], o["Edf"]), "edge image differs " + tag
    assert np.array_equal(g["edt"], o["D"]), "EDT differs " + tag
    d = np.abs(g["surf"].astype(np.float64) - o["S"]).max()
    assert d <= SURF_TOL, "surface max diff %g %s" % (d, tag)


# ---------------------------------------------------------------- front end
SMALL = [(1, 1), (1, 17), (23, 1), (5, 7), (33, 20), (64, 48), (100, 37), (129, 65)]


@pytest.mark.parametrize("W,H", SMALL)
def test_front_end_bit_exact_small(eb, W, H):
    rng = np.random.default_rng(W * 1000 + H)
    for conn, nd, nf in ((8, 1, 9), (4, 1, 5), (4, 2, 3), (8, 0, 9), (4, 1, 4)):
        prm, s = make_stream(eb, W, H, connectivity=conn, n_d=nd, n_f=nf)
        for k in range(2):
            n = int(rng.integers(0, 3 * W * H + 5))
            x, y, t, p = synth.random_edge_events(rng, W, H, n, t_begin=1000 * k, dt=1000,
                                                  out_of_range=0.1)
            g = run_window(eb, s, x, y, t, 1000 * k, 1000 * (k + 1), p)
            o = oracle_surface(prm, W, H, x, y, t, 1000 * k, 1000 * (k + 1))
            check_front(g, o, "(%dx%d conn %d nd %d nf %d)" % (W, H, conn, nd, nf))
            st = g["stats"]
            assert (st.events, st.in_window, st.dropped_time, st.dropped_oob) == tuple(
                int(v) for v in o["stats"])
            assert st.edge_px == int(o["Edf"].sum())
            assert g["status"] == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
            if min(W, H) < prm.patch:
                assert np.all(g["flow"] == 0.0)
        s.close()


@pytest.mark.parametrize("W,H,sites", [(1500, 3, 1), (3, 700, 2), (2000, 9, 3),
                                       (1280, 720, 1), (16384, 4, 3), (777, 33, 0),
                                       (1280, 720, 40)])
def test_edt_entry_sparse_wide_and_empty(eb, W, H, sites):
    rng = np.random.default_rng(W + 7 * H + sites)
    E = np.zeros((H, W), np.uint8)
    for _ in range(sites):
        E[rng.integers(H), rng.integers(W)] = 1
    want = oracle.edt_brute(E)
    scratch = torch.empty(W * H, dtype=torch.int32, device="cuda:0")
    D = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
    S = torch.empty((H, W), dtype=torch.float32, device="cuda:0")
    eb.check(eb.ebof_edt(dev(E), W, H, scratch, D, S, 1.08), "ebof_edt")
    torch.cuda.synchronize()
    assert np.array_equal(D.cpu().numpy(), want)
    Sw = oracle.surface(want, 1.08)
    assert np.abs(S.cpu().numpy() - Sw).max() <= SURF_TOL


def test_edt_entry_dense_random(eb):
    rng = np.random.default_rng(12)
    for W, H, dens in ((300, 200, 0.001), (517, 123, 0.05), (64, 64, 0.5), (2048, 16, 0.01)):
        E = (rng.random((H, W)) < dens).astype(np.uint8)
        scratch = torch.empty(W * H, dtype=torch.int32, device="cuda:0")
        D = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
        eb.check(eb.ebof_edt(dev(E), W, H, scratch, D, None, 1.08), "ebof_edt")
        torch.cuda.synchronize()
        assert np.array_equal(D.cpu().numpy(), oracle.edt(E)), (W, H, dens)


@pytest.mark.parametrize("W,H", [(600, 40), (1100, 36), (1280, 24)])
def test_edt_row_layouts_exact(eb, W, H):
    """The EDT row pass serves a row with one warp in batched calls and with
    two (from 512 px) or four (from 1024 px) warps, one row per block, for
    single frames; D must be exact in every layout.  Random pixels plus
    horizontal runs (long stretches of equal column distance next to them)."""
    rng = np.random.default_rng(W + H)
    prm, s = make_stream(eb, W, H, max_batch=3, n_d=0)
    wins = []
    for k in range(3):
        x, y, t, _ = synth.random_edge_events(rng, W, H, int(0.01 * W * H) * (k + 1),
                                              t_begin=1000 * k, dt=1000)
        for _ in range(4):
            r, a0 = int(rng.integers(H)), int(rng.integers(W // 2))
            run = np.arange(a0, min(W, a0 + int(rng.integers(5, W // 2))))
            x = np.concatenate([x, run.astype(np.uint16)])
            y = np.concatenate([y, np.full(run.size, r, np.uint16)])
            t = np.concatenate([t, np.full(run.size, 1000 * k, np.int64)])
        wins.append((x, y, t))
    # shuffled across the windows: warps straddle window boundaries in the
    # scatter's counts (the edge images do not depend on the order)
    perm = rng.permutation(sum(w[0].size for w in wins))
    x, y, t = (np.concatenate([w[i] for w in wins])[perm] for i in range(3))
    flow = torch.empty((3, 2, H, W), dtype=torch.float32, device="cuda:0")
    edge = torch.empty((3, H, W), dtype=torch.uint8, device="cuda:0")
    edt = torch.empty((3, H, W), dtype=torch.int32, device="cuda:0")
    st = eb.ebof_process_windows(s, 3, dev(x), dev(y), dev(t), None, 0, 1000, flow, edge, edt)
    assert st == eb.EBOF_NO_PREVIOUS
    sst, stats = eb.ebof_stream_sync(s, 3)
    eb.check(sst, "sync")
    scratch = torch.empty(W * H, dtype=torch.int32, device="cuda:0")
    D = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
    for k, (xk, yk, tk) in enumerate(wins):
        o = oracle_surface(prm, W, H, xk, yk, tk, 1000 * k, 1000 * (k + 1))
        assert (stats[k].in_window, stats[k].dropped_oob) == (int(o["stats"][1]),
                                                             int(o["stats"][3])), k
        assert stats[k].edge_px == int(o["Edf"].sum()), k
        assert np.array_equal(edge[k].cpu().numpy(), o["Edf"]), k
        assert np.array_equal(edt[k].cpu().numpy(), o["D"]), ("batched", k)
        eb.check(eb.ebof_edt(dev(o["Edf"]), W, H, scratch, D, None, 1.08), "ebof_edt")
        torch.cuda.synchronize()
        assert np.array_equal(D.cpu().numpy(), o["D"]), ("single", k)
    s.close()


# ---------------------------------------------------------------- whole path
def test_pipeline_346x260_parity(eb):
    s_ = synth.workload_346x260()
    W, H = s_.width, s_.height
    prm, s = make_stream(eb, W, H)
    gs = [run_k(eb, s, s_, k) for k in range(2)]
    os_ = [oracle_surface(prm, W, H, *s_.window(k)[:3], *s_.window(k)[4:]) for k in range(2)]
    for g, o in zip(gs, os_):
        check_front(g, o)
    U = oracle_flow(prm, 255.0 * os_[0]["S"], 255.0 * os_[1]["S"])
    e = epe(gs[1]["flow"], U)
    m = os_[1]["Edf"].astype(bool)
    print("346x260 flow vs oracle: mean EPE %.5f, p99 %.5f, on edges %.5f" %
          (e.mean(), np.percentile(e, 99), e[m].mean()))
    assert e.mean() <= EPE_TOL
    assert np.all(gs[0]["flow"] == 0.0) and gs[0]["status"] == eb.EBOF_NO_PREVIOUS
    s.close()


def test_pipeline_1280x720_parity(eb):
    s_ = synth.workload_1280x720(n_windows=2)
    W, H = s_.width, s_.height
    prm, s = make_stream(eb, W, H)
    gs = [run_k(eb, s, s_, k) for k in range(2)]
    os_ = [oracle_surface(prm, W, H, *s_.window(k)[:3], *s_.window(k)[4:]) for k in range(2)]
    for g, o in zip(gs, os_):
        check_front(g, o)
    U = oracle_flow(prm, 255.0 * os_[0]["S"], 255.0 * os_[1]["S"])
    e = epe(gs[1]["flow"], U)
    print("1280x720 flow vs oracle: mean EPE %.5f, p99 %.5f" % (e.mean(), np.percentile(e, 99)))
    assert e.mean() <= EPE_TOL
    assert np.percentile(e, 99) <= EPE_P99_TOL
    s.close()


def test_pipeline_1280x720_graph_path_parity(eb):
    """The path the benchmark times: one ebof_process_window call per window
    with the flow as its only output, so every window after the first
    replays the stream's CUDA graph (one graph per ping-pong slot).  Two flow
    frames, one from each graph, against the oracle."""
    s_ = synth.workload_1280x720(n_windows=3)
    W, H = s_.width, s_.height
    prm, s = make_stream(eb, W, H)
    flows = []
    for k in range(3):
        x, y, t, _, tb, te = s_.window(k)
        f = torch.full((2, H, W), float("nan"), dtype=torch.float32, device="cuda:0")
        st = eb.ebof_process_window(s, dev(x), dev(y), dev(t), None, tb, te, f)
        assert st == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        flows.append(f)
    eb.check(eb.ebof_stream_sync(s, 1)[0], "sync")
    Ss = [255.0 * oracle_surface(prm, W, H, *s_.window(k)[:3], *s_.window(k)[4:])["S"]
          for k in range(3)]
    for k in (1, 2):
        U = oracle_flow(prm, Ss[k - 1], Ss[k])
        e = epe(flows[k].cpu().numpy(), U)
        print("1280x720 graph path, frame %d: mean EPE %.5f, p99 %.5f"
              % (k, e.mean(), np.percentile(e, 99)))
        assert e.mean() <= EPE_TOL
        assert np.percentile(e, 99) <= EPE_P99_TOL
    s.close()


def _texture(W, H, v=(0.0, 0.0)):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    return (127.5 + 60.0 * np.sin(2 * np.pi * (xx - v[0]) / 23.0)
            * np.cos(2 * np.pi * (yy - v[1]) / 17.0)) / 255.0


@pytest.mark.parametrize("v", [(0.3, -0.2), (1.7, 0.9), (3.0, -1.5)])
def test_flow_on_analytic_surfaces(eb, v):
    W, H = 160, 120
    prm, s = make_stream(eb, W, H)
    S0 = _texture(W, H).astype(np.float32)
    S1 = _texture(W, H, v).astype(np.float32)
    flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_surface(s, dev(S0), flow) == eb.EBOF_NO_PREVIOUS
    assert eb.ebof_process_surface(s, dev(S1), flow) == eb.EBOF_OK
    torch.cuda.synchronize()
    F = flow.cpu().numpy()
    U = oracle_flow(prm, 255.0 * S0.astype(np.float64), 255.0 * S1.astype(np.float64))
    assert epe(F, U).mean() <= EPE_TOL
    inner = (slice(None), slice(16, -16), slice(16, -16))
    assert epe(F[inner], np.array(v)[:, None, None]).mean() <= 0.05
    s.close()


@pytest.mark.parametrize("W,H,storage", [(193, 129, 0), (129, 97, 0), (193, 129, 1)])
def test_flow_with_odd_level0_edges(eb, W, H, storage):
    """Widths and heights of 64k + 1 pixels: level 0's last column (row) lies
    past the 64-pixel regions that level 1's tiles cover, and its gradients
    are still written (the box-mean launch covers all of level 0).  The flow
    matches the oracle over the whole image and over the bands along the
    right and lower borders, where the patches flush with the border read
    the last column's and row's gradients; FP16 storage too (the 8-byte
    staging loads of half levels)."""
    v = (1.7, 0.9)
    prm, s = make_stream(eb, W, H, storage=storage)
    S0 = _texture(W, H).astype(np.float32)
    S1 = _texture(W, H, v).astype(np.float32)
    flow = torch.full((2, H, W), float("nan"), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_surface(s, dev(S0), flow) == eb.EBOF_NO_PREVIOUS
    assert eb.ebof_process_surface(s, dev(S1), flow) == eb.EBOF_OK
    torch.cuda.synchronize()
    F = flow.cpu().numpy()
    assert np.isfinite(F).all()
    U = oracle_flow(prm, 255.0 * S0.astype(np.float64), 255.0 * S1.astype(np.float64))
    e = epe(F, U)
    print("%dx%d storage %d: mean EPE %.5f, right band %.5f, lower band %.5f"
          % (W, H, storage, e.mean(), e[:, -prm.patch:].mean(), e[-prm.patch:, :].mean()))
    tol = EPE_TOL if storage == 0 else FP16_EPE_TOL
    assert e.mean() <= tol
    assert e[:, -prm.patch:].mean() <= tol
    assert e[-prm.patch:, :].mean() <= tol
    inner = (slice(None), slice(16, -16), slice(16, -16))
    assert epe(F[inner], np.array(v)[:, None, None]).mean() <= 0.05  # not a trivial flow
    s.close()


def test_many_sor_sweeps_take_the_half_sweep_kernels(eb):
    """More SOR sweeps than a 64-px region's halo allows (13 sweeps need a
    25-px halo) run the variational refinement as one launch per half sweep;
    the same gates against the oracle, with the same number of sweeps."""
    W, H = 160, 120
    v = (1.7, 0.9)
    prm, s = make_stream(eb, W, H, var_sor=13)
    S0 = _texture(W, H).astype(np.float32)
    S1 = _texture(W, H, v).astype(np.float32)
    flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_surface(s, dev(S0), flow) == eb.EBOF_NO_PREVIOUS
    assert eb.ebof_process_surface(s, dev(S1), flow) == eb.EBOF_OK
    torch.cuda.synchronize()
    F = flow.cpu().numpy()
    U = oracle_flow(prm, 255.0 * S0.astype(np.float64), 255.0 * S1.astype(np.float64))
    assert epe(F, U).mean() <= EPE_TOL
    inner = (slice(None), slice(16, -16), slice(16, -16))
    assert epe(F[inner], np.array(v)[:, None, None]).mean() <= 0.05
    s.close()


def test_flat_and_zero_motion_surfaces(eb):
    W, H = 96, 64
    prm, s = make_stream(eb, W, H)
    flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    S = dev(_texture(W, H).astype(np.float32))
    eb.ebof_process_surface(s, S, flow)
    eb.check(eb.ebof_process_surface(s, S, flow))
    torch.cuda.synchronize()
    assert torch.count_nonzero(flow).item() == 0
    F = dev(np.full((H, W), 0.7, np.float32))
    eb.ebof_process_surface(s, F, flow)
    eb.check(eb.ebof_process_surface(s, dev(np.full((H, W), 0.6, np.float32)), flow))
    torch.cuda.synchronize()
    f = flow.cpu().numpy()
    assert not np.isnan(f).any() and np.all(f == 0.0)
    s.close()


# ---------------------------------------------------------------- API
def test_batched_equals_sequential(eb):
    s_ = synth.translating_segments(n_windows=5, seed=3)
    W, H = s_.width, s_.height
    prm, seq = make_stream(eb, W, H)
    outs = [run_k(eb, seq, s_, k) for k in range(5)]
    _, bat = make_stream(eb, W, H, max_batch=4)
    # first window alone, then windows 1..4 in one call
    run_k(eb, bat, s_, 0)
    a, b = int(s_.offsets[1]), int(s_.offsets[5])
    flow = torch.empty((4, 2, H, W), dtype=torch.float32, device="cuda:0")
    edge = torch.empty((4, H, W), dtype=torch.uint8, device="cuda:0")
    edt = torch.empty((4, H, W), dtype=torch.int32, device="cuda:0")
    st = eb.ebof_process_windows(bat, 4, dev(s_.x[a:b]), dev(s_.y[a:b]), dev(s_.t[a:b]), None,
                                 int(s_.t_begin[1]), s_.dt, flow, edge, edt)
    assert st == eb.EBOF_OK
    sst, stats = eb.ebof_stream_sync(bat, 4)
    eb.check(sst)
    for k in range(4):
        o = outs[k + 1]
        assert np.array_equal(edge[k].cpu().numpy(), o["edge"])
        assert np.array_equal(edt[k].cpu().numpy(), o["edt"])
        assert np.array_equal(flow[k].cpu().numpy(), o["flow"])
        assert stats[k].in_window == o["stats"].in_window
        assert stats[k].edge_px == o["stats"].edge_px
    # a batch that starts a stream: window 0 gets zero flow
    _, b2 = make_stream(eb, W, H, max_batch=3)
    a, b = int(s_.offsets[0]), int(s_.offsets[3])
    flow3 = torch.empty((3, 2, H, W), dtype=torch.float32, device="cuda:0")
    st = eb.ebof_process_windows(b2, 3, dev(s_.x[a:b]), dev(s_.y[a:b]), dev(s_.t[a:b]), None,
                                 int(s_.t_begin[0]), s_.dt, flow3)
    assert st == eb.EBOF_NO_PREVIOUS
    torch.cuda.synchronize()
    assert torch.count_nonzero(flow3[0]).item() == 0
    assert np.array_equal(flow3[1].cpu().numpy(), outs[1]["flow"])
    assert np.array_equal(flow3[2].cpu().numpy(), outs[2]["flow"])
    for h in (seq, bat, b2):
        h.close()


def test_reset_interleave_host_and_errors(eb):
    s_ = synth.translating_segments(n_windows=3, seed=5)
    W, H = s_.width, s_.height
    prm, a = make_stream(eb, W, H)
    _, b = make_stream(eb, W, H)
    ra = [run_k(eb, a, s_, k) for k in range(3)]
    # b interleaved with a second pass over a after reset
    assert eb.ebof_stream_reset(a) == eb.EBOF_OK
    rb, ra2 = [], []
    for k in range(3):
        rb.append(run_k(eb, b, s_, k))
        ra2.append(run_k(eb, a, s_, k))
    for k in range(3):
        assert np.array_equal(ra[k]["flow"], rb[k]["flow"])
        assert np.array_equal(ra[k]["flow"], ra2[k]["flow"])
    assert ra2[0]["status"] == eb.EBOF_NO_PREVIOUS
    # host-buffer variant gives the same flow
    _, c = make_stream(eb, W, H)
    for k in range(3):
        x, y, t, p, tb, te = s_.window(k)
        hf = np.empty((2, H, W), np.float32)
        st = eb.ebof_process_window_host(c, np.ascontiguousarray(x), np.ascontiguousarray(y),
                                         np.ascontiguousarray(t), tb, te, hf)
        assert st == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        assert np.array_equal(hf, ra[k]["flow"])
    # page-locked host buffers: from the second window on the kernels read the
    # events and write the flow in place; the same flow

    def pinned(a):
        buf = torch.empty(max(a.nbytes, 1), dtype=torch.uint8).pin_memory()
        v = buf.numpy()[:a.nbytes].view(a.dtype)
        v[:] = a
        return v, buf

    _, d = make_stream(eb, W, H)
    hfp, hfp_buf = pinned(np.zeros((2 * H * W,), np.float32))
    for k in range(3):
        x, y, t, p, tb, te = s_.window(k)
        (xp, xb), (yp, yb), (tp, tbuf) = pinned(x), pinned(y), pinned(t)
        hfp[:] = np.nan
        st = eb.ebof_process_window_host(d, xp, yp, tp, tb, te, hfp)
        assert st == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        assert np.array_equal(hfp.reshape(2, H, W), ra[k]["flow"]), k
    # the asynchronous variant: every window enqueued before one sync, each
    # into its own page-locked flow buffer (events in and flows out on the
    # stream's copy streams, through alternating staging slots); the same flows
    _, e = make_stream(eb, W, H)
    keep, outs = [], []
    for k in range(3):
        x, y, t, p, tb, te = s_.window(k)
        (xp, xb), (yp, yb), (tp, tbuf) = pinned(x), pinned(y), pinned(t)
        hf_k, hf_buf = pinned(np.full((2 * H * W,), np.nan, np.float32))
        keep.append((xb, yb, tbuf, hf_buf))
        st = eb.ebof_process_window_host_async(e, xp, yp, tp, tb, te, hf_k)
        assert st == (eb.EBOF_NO_PREVIOUS if k == 0 else eb.EBOF_OK)
        outs.append(hf_k)
    assert eb.ebof_stream_sync(e, 1)[0] == eb.EBOF_OK
    for k in range(3):
        assert np.array_equal(outs[k].reshape(2, H, W), ra[k]["flow"]), k
    # pageable buffers take the synchronous staged call
    x, y, t, p, tb, te = s_.window(1)
    hf = np.empty((2, H, W), np.float32)
    assert eb.ebof_process_window_host_async(e, np.ascontiguousarray(x), np.ascontiguousarray(y),
                                             np.ascontiguousarray(t), tb, te, hf) == eb.EBOF_OK
    assert np.isfinite(hf).all()
    e.close()
    # argument errors enqueue nothing
    x, y, t, p, tb, te = s_.window(0)
    lib = eb.load()
    assert lib.ebof_process_window(a.handle, None, None, None, None, 5, tb, te, None, None, None,
                                   None, None) == eb.EBOF_ERR_INVALID_ARG
    flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_window(a, dev(x), dev(y), dev(t), None, te, tb, flow) == \
        eb.EBOF_ERR_INVALID_ARG
    flow2 = torch.empty((2, 2, H, W), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_windows(a, 2, dev(x), dev(y), dev(t), None, tb, 100, flow2) == \
        eb.EBOF_ERR_INVALID_ARG  # max_batch is 1
    # an empty window is legal: no edge pixel, D = INT32_MAX, S = 1
    g = run_window(eb, a, x[:0], y[:0], t[:0], tb, te)
    assert g["stats"].edge_px == 0 and np.all(g["edt"] == 2147483647) and np.all(g["surf"] == 1.0)
    for h in (a, b, c, d):
        h.close()


def test_graph_replay_equals_eager_launches(eb):
    # without optional outputs, steady-state single windows replay a CUDA
    # graph; with them, every stage is launched step by step
    s_ = synth.translating_segments(n_windows=5, seed=13)
    W, H = s_.width, s_.height
    _, a = make_stream(eb, W, H)
    _, b = make_stream(eb, W, H)
    for k in range(5):
        x, y, t, p, tb, te = s_.window(k)
        fa = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
        fb = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
        edge = torch.empty((H, W), dtype=torch.uint8, device="cuda:0")
        ra = eb.ebof_process_window(a, dev(x), dev(y), dev(t), None, tb, te, fa)
        rb = eb.ebof_process_window(b, dev(x), dev(y), dev(t), None, tb, te, fb, edge)
        assert ra == rb
        torch.cuda.synchronize()
        assert torch.equal(fa, fb), k
        sa, st_a = eb.ebof_stream_sync(a, 1)
        sb, st_b = eb.ebof_stream_sync(b, 1)
        assert sa == sb == eb.EBOF_OK
        assert (st_a[0].in_window, st_a[0].edge_px) == (st_b[0].in_window, st_b[0].edge_px)
    a.close()
    b.close()
