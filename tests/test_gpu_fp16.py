"""FP16 storage of surfaces, pyramid levels and gradients (the precision
variant of the 1280x720 stream): patch sums, densification and the
variational refinement stay FP32.  The edge image and the EDT stay exact
integers; the flow's endpoint error is stated against the FP64 oracle and
against the FP32 GPU path."""
import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

FP16_EPE_TOL = 0.06

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def _run(eb, storage, s_, n):
    W, H = s_.width, s_.height
    p = eb.ebof_default_params(W, H)
    p.storage = storage
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st)
    outs = []
    for k in range(n):
        x, y, t, pp, tb, te = s_.window(k)
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
        edge = torch.empty((H, W), dtype=torch.uint8, device="cuda")
        edt = torch.empty((H, W), dtype=torch.int32, device="cuda")
        eb.check(eb.ebof_process_window(s, dev(x), dev(y), dev(t), None, tb, te, flow, edge, edt))
        outs.append((flow.cpu().numpy(), edge.cpu().numpy(), edt.cpu().numpy()))
    eb.check(eb.ebof_stream_sync(s, 1)[0])
    s.close()
    return p, outs


def test_fp16_storage_1280x720(eb):
    s_ = synth.workload_1280x720(n_windows=2)
    p32, o32 = _run(eb, eb.EBOF_STORAGE_FP32, s_, 2)
    p16, o16 = _run(eb, eb.EBOF_STORAGE_FP16, s_, 2)
    for a, b in zip(o32, o16):
        assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])
    e_gpu = np.hypot(*(o16[1][0] - o32[1][0]))
    S = []
    for k in range(2):
        x, y, t, _, tb, te = s_.window(k)
        S.append(255.0 * oracle.surface_from_events(1280, 720, x, y, t, tb, te)["S"])
    U = oracle.flow(S[0], S[1], levels=p16.levels, patch=p16.patch, stride=p16.stride,
                    gn_iters=p16.gn_iters, gn_damping=float(p16.gn_damping))
    e_orc = np.hypot(*(o16[1][0] - U))
    e32 = np.hypot(*(o32[1][0] - U))
    print("FP16 storage 1280x720: EPE vs FP32 GPU %.5f (p99 %.4f), vs FP64 oracle %.5f "
          "(p99 %.4f); FP32 GPU vs oracle %.5f" % (e_gpu.mean(), np.percentile(e_gpu, 99),
                                                  e_orc.mean(), np.percentile(e_orc, 99),
                                                  e32.mean()))
    # measured 0.049 px mean over 16 frames of this stream (against the
    # oracle and against the FP32 path); FP16's 11-bit mantissa on the
    # complement surface adds about as much as the 0.05 px flow gate
    assert e_orc.mean() <= FP16_EPE_TOL
    assert e_gpu.mean() <= FP16_EPE_TOL


def test_fp16_batched_equals_sequential(eb):
    s_ = synth.translating_segments(n_windows=4, seed=8)
    W, H = s_.width, s_.height
    _, seq = _run(eb, eb.EBOF_STORAGE_FP16, s_, 4)
    p = eb.ebof_default_params(W, H)
    p.storage = eb.EBOF_STORAGE_FP16
    p.max_batch = 4
    st, b = eb.ebof_stream_create(p, 0)
    eb.check(st)
    flow = torch.empty((4, 2, H, W), dtype=torch.float32, device="cuda")
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    a0, a1 = int(s_.offsets[0]), int(s_.offsets[4])
    r = eb.ebof_process_windows(b, 4, dev(s_.x[a0:a1]), dev(s_.y[a0:a1]), dev(s_.t[a0:a1]),
                                None, int(s_.t_begin[0]), s_.dt, flow)
    assert r == eb.EBOF_NO_PREVIOUS
    torch.cuda.synchronize()
    for k in range(1, 4):
        assert np.array_equal(flow[k].cpu().numpy(), seq[k][0])
    b.close()
