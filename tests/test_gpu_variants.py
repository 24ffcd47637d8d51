"""The paper's variants on the GPU, against the FP64 oracle (needs a GB300).

* The ablation surfaces of §IV-D (DS_L, DS_LB, DS_Log) in place of Eq. 1:
  EDT bit-exact, surface within 1e-5 relative, flow within 0.05 px mean
  endpoint error (FP32 storage) or 0.15 px (FP16 storage).
* The 4-neighbour denoising/filling settings of §IV-A, {N_d=1, N_f=4} at low
  resolution and {N_d=2, N_f=3} at high resolution: edge images bit-exact,
  flow within 0.05 px.
"""
import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPE_TOL = 0.05
EPE_TOL_FP16 = 0.15


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def gpu_pair(eb, prm, ev):
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    W, H = prm.width, prm.height
    out = []
    for k in range(2):
        x, y, t, _, tb, te = ev.window(k)
        flow = torch.full((2, H, W), float("nan"), device="cuda:0")
        edge = torch.empty((H, W), dtype=torch.uint8, device="cuda:0")
        edt = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
        surf = torch.empty((H, W), dtype=torch.float32, device="cuda:0")
        eb.check(eb.ebof_process_window(s, dev(x), dev(y), dev(t), None, tb, te, flow, edge,
                                        edt, surf))
        eb.check(eb.ebof_stream_sync(s, 0)[0])
        out.append(dict(flow=flow.cpu().numpy(), edge=edge.cpu().numpy(),
                        edt=edt.cpu().numpy(), surf=surf.cpu().numpy()))
    s.close()
    return out


def oracle_pair(prm, ev):
    w0 = ev.window(0)
    w1 = ev.window(1)
    return oracle.process_pair(
        prm.width, prm.height, (w0[0], w0[1], w0[2], w0[4], w0[5]),
        (w1[0], w1[1], w1[2], w1[4], w1[5]), connectivity=prm.connectivity, n_d=prm.n_d,
        n_f=prm.n_f, alpha=float(prm.alpha), surface=prm.surface, d_sat=float(prm.d_sat),
        levels=prm.levels, patch=prm.patch, stride=prm.stride, gn_iters=prm.gn_iters,
        gn_damping=float(prm.gn_damping), var_outer=prm.var_outer, var_sor=prm.var_sor,
        var_delta=float(prm.var_delta), var_gamma=float(prm.var_gamma),
        var_alpha=float(prm.var_alpha), sor_omega=float(prm.sor_omega))


def compare(g, o, fp16=False):
    s0, s1, U = o
    for gk, ok in zip(g, (s0, s1)):
        assert np.array_equal(gk["edge"], ok["Edf"])
        assert np.array_equal(gk["edt"], ok["D"])
        err = np.abs(gk["surf"].astype(np.float64) - ok["S"]) / np.maximum(1.0, np.abs(ok["S"]))
        assert err.max() <= 1e-5, err.max()
    e = np.hypot(g[1]["flow"][0] - U[0], g[1]["flow"][1] - U[1])
    assert np.isfinite(g[1]["flow"]).all()
    assert e.mean() <= (EPE_TOL_FP16 if fp16 else EPE_TOL), e.mean()
    assert np.all(g[0]["flow"] == 0.0)
    return float(e.mean())


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_ablation_surface_346x260(eb, mode):
    ev = synth.workload_346x260()
    prm = eb.ebof_default_params(ev.width, ev.height)
    prm.surface = mode
    compare(gpu_pair(eb, prm, ev), oracle_pair(prm, ev))


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_ablation_surface_1280x720(eb, mode):
    """DS_L and DS_Log are unbounded: far from the edges the surface is a
    smooth cone field where the flow is poorly determined, and the oracle's
    own flow moves by 0.02 px mean EPE when only its inputs are rounded to
    FP32 (Eq. 1: 0.006).  The bar for those two is derived from that
    sensitivity, measured here: 10 times it (at least 0.05 px) over the image
    and 0.1 px on the edge pixels; DS_LB keeps the fixed 0.05 px bar."""
    ev = synth.workload_1280x720(n_windows=2)
    prm = eb.ebof_default_params(ev.width, ev.height)
    prm.surface = mode
    g = gpu_pair(eb, prm, ev)
    o = oracle_pair(prm, ev)
    if mode == eb.EBOF_SURFACE_BOUNDED:
        compare(g, o)
        return
    s0, s1, U = o
    for gk, ok in zip(g, (s0, s1)):
        assert np.array_equal(gk["edt"], ok["D"])
    gain = oracle.intensity_gain(mode, float(prm.d_sat))
    kw = dict(levels=prm.levels, patch=prm.patch, stride=prm.stride)
    r32 = lambda a: (gain * a).astype(np.float32).astype(np.float64)
    U32 = oracle.flow(r32(s0["S"]), r32(s1["S"]), **kw)
    sens = np.hypot(U[0] - U32[0], U[1] - U32[1]).mean()
    e = np.hypot(g[1]["flow"][0] - U[0], g[1]["flow"][1] - U[1])
    edge = s1["Edf"].astype(bool)
    print("mode %d: GPU vs oracle %.4f (edges %.4f), oracle FP32-input sensitivity %.4f"
          % (mode, e.mean(), e[edge].mean(), sens))
    assert np.isfinite(g[1]["flow"]).all()
    assert e.mean() <= max(EPE_TOL, 10.0 * sens), (e.mean(), sens)
    assert e[edge].mean() <= 0.1, e[edge].mean()


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_ablation_surface_fp16(eb, mode):
    ev = synth.workload_346x260()
    prm = eb.ebof_default_params(ev.width, ev.height)
    prm.surface = mode
    prm.storage = eb.EBOF_STORAGE_FP16
    g = gpu_pair(eb, prm, ev)
    o = oracle_pair(prm, ev)
    compare(g, o, fp16=True)


def test_ablation_surface_through_process_surface(eb):
    """A surface exported by one stream and fed to another stream of the same
    kind gives the same flow, bit for bit (same intensity scale)."""
    ev = synth.workload_346x260()
    prm = eb.ebof_default_params(ev.width, ev.height)
    prm.surface = eb.EBOF_SURFACE_LOG
    g = gpu_pair(eb, prm, ev)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    flow = torch.empty((2, prm.height, prm.width), device="cuda:0")
    eb.ebof_process_surface(s, dev(g[0]["surf"]), flow)
    eb.check(eb.ebof_process_surface(s, dev(g[1]["surf"]), flow))
    torch.cuda.synchronize()
    assert np.array_equal(flow.cpu().numpy(), g[1]["flow"])
    s.close()


def test_ablation_surface_empty_window_is_flat(eb):
    """A window without events: every ablation surface is one constant, the
    flow from and to it stays finite."""
    W, H = 96, 64
    for mode in (1, 2, 3):
        for storage in (0, 1):
            prm = eb.ebof_default_params(W, H)
            prm.surface = mode
            prm.storage = storage
            st, s = eb.ebof_stream_create(prm, 0)
            eb.check(st)
            e16 = torch.empty(0, dtype=torch.uint16, device="cuda:0")
            e64 = torch.empty(0, dtype=torch.int64, device="cuda:0")
            flow = torch.empty((2, H, W), device="cuda:0")
            surf = torch.empty((H, W), device="cuda:0")
            eb.ebof_process_window(s, e16, e16, e64, None, 0, 10, flow, None, None, surf)
            eb.check(eb.ebof_process_window(s, e16, e16, e64, None, 10, 20, flow, None, None,
                                            surf))
            torch.cuda.synchronize()
            sv = surf.cpu().numpy()
            want = oracle.surface_mode(np.array([oracle.INF_D], np.int32), mode)[0]
            assert np.all(sv == sv[0, 0]) and abs(sv[0, 0] - want) <= 1e-5 * want
            f = flow.cpu().numpy()
            assert np.isfinite(f).all() and np.all(f == 0.0)
            s.close()


@pytest.mark.parametrize("which", ["lr", "hr"])
def test_paper_four_neighbour_settings(eb, which):
    if which == "lr":
        ev = synth.workload_346x260()
        n_d, n_f = 1, 4
    else:
        ev = synth.workload_1280x720(n_windows=2)
        n_d, n_f = 2, 3
    prm = eb.ebof_default_params(ev.width, ev.height)
    prm.connectivity, prm.n_d, prm.n_f = 4, n_d, n_f
    g = gpu_pair(eb, prm, ev)
    o = oracle_pair(prm, ev)
    compare(g, o)
    # denoising and filling both act with these settings
    for gk, ok in zip(g, o[:2]):
        assert not np.array_equal(ok["E"], ok["Edf"])


# ---------------------------------------------------------------- §IV-C FWL
def _fwl_case(eb, ev, k, flow_np):
    x, y, t, p, tb, te = ev.window(k)
    W, H = ev.width, ev.height
    fl = dev(flow_np.astype(np.float32))
    st, out = eb.ebof_fwl(dev(x), dev(y), dev(t), dev(p), tb, te, fl, W, H)
    eb.check(st)
    torch.cuda.synchronize()
    g = out.cpu().numpy()
    o = oracle.fwl(W, H, x, y, t, p, tb, te, flow_np.astype(np.float32).astype(np.float64))
    return g, np.array(o)


@pytest.mark.parametrize("which", ["346x260", "1280x720"])
def test_fwl_matches_oracle_on_computed_flow(eb, which):
    ev = synth.workload_346x260() if which == "346x260" else synth.workload_1280x720(n_windows=2)
    prm = eb.ebof_default_params(ev.width, ev.height)
    g = gpu_pair(eb, prm, ev)
    fg, fo = _fwl_case(eb, ev, 1, g[1]["flow"])
    rel = np.abs(fg - fo) / np.abs(fo)
    assert rel.max() <= 1e-5, (fg, fo)
    if which == "346x260":
        assert fg[0] > 1.0  # the flow of the translating scene sharpens its events


def test_fwl_zero_flow_and_edge_cases(eb):
    ev = synth.workload_346x260()
    W, H = ev.width, ev.height
    fg, fo = _fwl_case(eb, ev, 0, np.zeros((2, H, W)))
    assert fg[0] == 1.0 and fg[1] == fg[2] and abs(fg[2] - fo[2]) <= 1e-9 * fo[2]
    # without polarity, no events, window with every event outside
    x, y, t, p, tb, te = ev.window(1)
    U = np.zeros((2, H, W), np.float32)
    U[0], U[1] = 3.0, -1.5
    st, out = eb.ebof_fwl(dev(x), dev(y), dev(t), None, tb, te, dev(U), W, H)
    eb.check(st)
    torch.cuda.synchronize()
    o = oracle.fwl(W, H, x, y, t, None, tb, te, U.astype(np.float64))
    assert abs(out[0].item() - o[0]) <= 1e-5 * o[0]
    e16 = torch.empty(0, dtype=torch.uint16, device="cuda:0")
    st, out = eb.ebof_fwl(e16, e16, torch.empty(0, dtype=torch.int64, device="cuda:0"), None,
                          0, 10, dev(U), W, H)
    eb.check(st)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [1.0, 0.0, 0.0]
    st, out = eb.ebof_fwl(dev(x), dev(y), dev(t), dev(p), te + 10, te + 20, dev(U), W, H)
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [1.0, 0.0, 0.0]
    assert eb.load().ebof_fwl(None, None, None, None, 5, 0, 10, None, W, H, None, None,
                              None) == eb.EBOF_ERR_INVALID_ARG
