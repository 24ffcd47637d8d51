"""The multi-stream autotuner (config 3's parameter choice) on the GPU.

* Every method candidate the tuner may pick, at both workload resolutions,
  gives a GPU flow within 0.05 px mean endpoint error of the FP64 oracle run
  with the same parameters: the tuner only chooses among configurations whose
  parity with the oracle holds.
* A tuning run returns an accepted method candidate (no worse than the
  defaults by the Flow Warping Loss, §IV-C) and layouts whose flows are the
  default layout's bit for bit.
"""
import numpy as np
import pytest

import oracle
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


@pytest.mark.parametrize("res", ["346x260", "1280x720"])
def test_every_method_candidate_matches_the_oracle(eb, res):
    from paper_2112_10591_gb300 import autotune
    if res == "346x260":
        ev = synth.translating_segments(n_windows=2, seed=0)
    else:
        ev = synth.rigid_objects(n_windows=2, seed=31, events=(150000, 200000))
    W, H = ev.width, ev.height
    S = []
    for k in range(2):
        x, y, t, _, tb, te = ev.window(k)
        S.append(255.0 * oracle.surface_from_events(W, H, x, y, t, tb, te)["S"])
    for ps, st, lv in autotune.method_candidates(W, H):
        prm = eb.ebof_default_params(W, H)
        prm.patch, prm.stride, prm.levels = ps, st, lv
        rc, s = eb.ebof_stream_create(prm, 0)
        eb.check(rc)
        flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
        for k in range(2):
            x, y, t, _, tb, te = ev.window(k)
            eb.check(eb.ebof_process_window(s, _dev(x), _dev(y), _dev(t), None, tb, te, flow))
        eb.check(eb.ebof_stream_sync(s, 1)[0])
        s.close()
        U = oracle.flow(S[0], S[1], levels=lv, patch=ps, stride=st, gn_iters=prm.gn_iters,
                        gn_damping=float(prm.gn_damping))
        F = flow.cpu().numpy()
        e = np.hypot(F[0] - U[0], F[1] - U[1]).mean()
        print("%s candidate ps %d stride %d levels %d: mean EPE vs oracle %.4f"
              % (res, ps, st, lv, e))
        assert e <= 0.05, (ps, st, lv, e)


def test_tuning_run(eb):
    from paper_2112_10591_gb300 import autotune
    W, H = 346, 260
    calib = []
    keep = []
    for i in range(3):
        ev = synth.translating_segments(n_windows=2, seed=90 + i, velocity=(2.0, 1.0 + i))
        pair = []
        for k in range(2):
            x, y, t, _, tb, te = ev.window(k)
            pair.append((_dev(x), _dev(y), _dev(t), tb, te))
        calib.append(pair)
        keep.append(ev)
    prm, table = autotune.tune(W, H, calib, repeats=3)
    chosen = [r for r in table["method"]
              if (r["patch"], r["stride"], r["levels"]) == (prm.patch, prm.stride, prm.levels)]
    assert chosen and chosen[0]["accepted"]
    assert table["method"][0]["accepted"]  # the defaults are the reference
    timed = [r for r in table["layout"] if r.get("ms_per_step") is not None]
    assert len(timed) >= 1 + sum(len(v) - 1 for v in autotune.LAYOUT_CANDIDATES.values())
    assert all(r["identical"] for r in timed)
    for knob in autotune.LAYOUT_CANDIDATES:
        assert getattr(prm, knob) == table["layout_chosen"][knob]
    rc, s = eb.ebof_stream_create(prm, 0)
    eb.check(rc)
    s.close()
