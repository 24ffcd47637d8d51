"""GPU path vs the FP64 oracle away from the default parameters and inputs.

* Patch sizes and strides other than the defaults: odd sizes (per-lane column
  and row counts that do not divide the patch), the largest patch (16), a
  stride equal to the patch (one covering patch per axis) and strides whose
  covering-patch count takes the densification's runtime loop, and a patch
  count that takes the search's wide layout with a small patch.
* A window without events between two windows with events (its edge image
  is empty, its surface flat).
* The 640x480 resolution of the served workload.
Gates as in the main parity tests: edge image and squared EDT bit-exact,
flow within 0.05 px mean endpoint error of the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

EPE_TOL = 0.05


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _run(eb, prm, wins):
    """wins: (x, y, t, t_begin, t_end) numpy windows; returns per window
    (status, flow, edge, edt, stats)."""
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    W, H = prm.width, prm.height
    out = []
    for x, y, t, tb, te in wins:
        flow = torch.full((2, H, W), float("nan"), dtype=torch.float32, device="cuda:0")
        edge = torch.empty((H, W), dtype=torch.uint8, device="cuda:0")
        edt = torch.empty((H, W), dtype=torch.int32, device="cuda:0")
        r = eb.ebof_process_window(s, _dev(x), _dev(y), _dev(t), None, tb, te, flow, edge, edt)
        eb.check(r)
        sst, stats = eb.ebof_stream_sync(s, 1)
        eb.check(sst)
        out.append((r, flow.cpu().numpy(), edge.cpu().numpy(), edt.cpu().numpy(), stats[0]))
    s.close()
    return out


def _oracle(prm, wins):
    W, H = prm.width, prm.height
    surf = [oracle.surface_from_events(W, H, x, y, t, tb, te, connectivity=prm.connectivity,
                                       n_d=prm.n_d, n_f=prm.n_f, alpha=float(prm.alpha))
            for x, y, t, tb, te in wins]
    flows = [None]
    for k in range(1, len(wins)):
        flows.append(oracle.flow(255.0 * surf[k - 1]["S"], 255.0 * surf[k]["S"],
                                 levels=prm.levels, patch=prm.patch, stride=prm.stride,
                                 gn_iters=prm.gn_iters, gn_damping=float(prm.gn_damping),
                                 var_outer=prm.var_outer, var_sor=prm.var_sor,
                                 var_delta=float(prm.var_delta),
                                 var_gamma=float(prm.var_gamma),
                                 var_alpha=float(prm.var_alpha),
                                 sor_omega=float(prm.sor_omega)))
    return surf, flows


def _windows(ev, n):
    return [tuple(ev.window(k)[i] for i in (0, 1, 2, 4, 5)) for k in range(n)]


@pytest.mark.parametrize("W,H,ps,stride,levels", [
    (96, 72, 4, 1, 2),      # smallest patch, every pixel a patch origin
    (160, 120, 7, 3, 3),    # odd patch
    (173, 130, 9, 5, 3),    # odd patch and stride, odd level sizes
    (200, 150, 16, 3, 2),   # largest patch; six covering patches per axis (runtime loop)
    (128, 96, 16, 16, 1),   # stride = patch: one covering patch per axis
    (346, 260, 5, 2, 3),    # 22 188 patches at level 0: the wide layout with a 5x5 patch
])
def test_patch_sizes_and_strides(eb, W, H, ps, stride, levels):
    ev = synth.translating_segments(width=W, height=H, n_windows=2, seed=W + ps,
                                    events_per_window=max(2000, W * H // 5))
    prm = eb.ebof_default_params(W, H)
    prm.patch, prm.stride, prm.levels = ps, stride, levels
    wins = _windows(ev, 2)
    g = _run(eb, prm, wins)
    surf, flows = _oracle(prm, wins)
    for (r, F, E, D, _), o in zip(g, surf):
        assert np.array_equal(E, o["Edf"]) and np.array_equal(D, o["D"])
    e = np.hypot(g[1][1][0] - flows[1][0], g[1][1][1] - flows[1][1])
    print("%dx%d ps %d stride %d levels %d: mean EPE vs oracle %.5f, p99 %.4f"
          % (W, H, ps, stride, levels, e.mean(), np.percentile(e, 99)))
    assert e.mean() <= EPE_TOL


def test_window_without_events(eb):
    ev = synth.translating_segments(n_windows=3, seed=12)
    W, H = ev.width, ev.height
    prm = eb.ebof_default_params(W, H)
    wins = _windows(ev, 3)
    x, y, t, tb, te = wins[1]
    wins[1] = (x[:0], y[:0], t[:0], tb, te)  # the middle window has no events
    g = _run(eb, prm, wins)
    surf, flows = _oracle(prm, wins)
    assert g[1][4].edge_px == 0 and g[1][4].events == 0
    assert np.all(g[1][3] == np.iinfo(np.int32).max)
    for k in (1, 2):
        assert np.array_equal(g[k][2], surf[k]["Edf"]) and np.array_equal(g[k][3], surf[k]["D"])
        assert np.isfinite(g[k][1]).all()
        e = np.hypot(g[k][1][0] - flows[k][0], g[k][1][1] - flows[k][1])
        print("empty window, frame %d: mean EPE vs oracle %.5f" % (k, e.mean()))
        assert e.mean() <= EPE_TOL


def test_640x480_served_resolution(eb):
    ev = synth.rigid_objects(width=640, height=480, n_windows=2, n_objects=8, n_edges=150,
                             radius=(25.0, 110.0), extra_length=(8.0, 80.0),
                             events=(60000, 120000), seed=33)
    prm = eb.ebof_default_params(640, 480)
    wins = _windows(ev, 2)
    g = _run(eb, prm, wins)
    surf, flows = _oracle(prm, wins)
    for (r, F, E, D, _), o in zip(g, surf):
        assert np.array_equal(E, o["Edf"]) and np.array_equal(D, o["D"])
    e = np.hypot(g[1][1][0] - flows[1][0], g[1][1][1] - flows[1][1])
    print("640x480: mean EPE vs oracle %.5f, p99 %.4f" % (e.mean(), np.percentile(e, 99)))
    assert e.mean() <= EPE_TOL
    assert np.percentile(e, 99) <= 1.0
