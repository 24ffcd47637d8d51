"""Error paths of the library, driven from the host without faulting a GPU.

* A copy-ahead SOR wait that runs out: the stream's wait bound is set to 0
  (ebof_stream_set_wait_limit), so the batched SOR kernel's first wait for
  its coefficient copy ends at once; the kernel latches EBOF_ERR_TIMEOUT and
  lets the copy in flight land under a second wait at the default bound.
  ebof_stream_sync reports the timeout; after a reset the stream gives the
  same flow as a fresh stream, and that flow matches the oracle.
* A device allocation that fails (ebof_debug_fail_allocation, an injected
  cudaMalloc failure): stream creation reports EBOF_ERR_OOM and frees what
  it had allocated; an existing stream whose host-buffer call meets the
  failure reports EBOF_ERR_OOM and stays usable; so does a first pipelined
  call whose buffers cannot all be allocated.
* Two host threads on one stream: the second call is refused with
  EBOF_ERR_BUSY and enqueues nothing.
"""
import threading
import time

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
    yield m
    m.ebof_debug_fail_allocation(-1)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


def _batch_events(ev, k0, n):
    a, b = int(ev.offsets[k0]), int(ev.offsets[k0 + n])
    return _dev(ev.x[a:b]), _dev(ev.y[a:b]), _dev(ev.t[a:b]), int(ev.t_begin[k0])


def _run_batches(eb, s, ev, n, flow):
    """Window 0 alone, then windows 1..n in one batched call."""
    x, y, t, p, tb, te = ev.window(0)
    f0 = torch.empty((2, ev.height, ev.width), dtype=torch.float32, device="cuda:0")
    assert eb.ebof_process_window(s, _dev(x), _dev(y), _dev(t), None, tb, te,
                                  f0) == eb.EBOF_NO_PREVIOUS
    bx, by, bt, btb = _batch_events(ev, 1, n)
    return eb.ebof_process_windows(s, n, bx, by, bt, None, btb, ev.dt, flow)


def test_sor_wait_timeout_is_reported_and_the_stream_recovers(eb):
    # 32 windows of 346x260 in one call: 48 SOR regions per frame at level 0,
    # 1536 in all, at least four per SM, so level 0 takes the copy-ahead kernel
    ev = synth.translating_segments(n_windows=33, seed=3)
    W, H, n = ev.width, ev.height, 32
    p = eb.ebof_default_params(W, H)
    p.max_batch = n
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st)
    st, ref = eb.ebof_stream_create(p, 0)
    eb.check(st)
    flow = torch.zeros((n, 2, H, W), dtype=torch.float32, device="cuda:0")
    flow_ref = torch.zeros_like(flow)
    assert eb.ebof_stream_set_wait_limit(s, 0) == eb.EBOF_OK
    assert _run_batches(eb, s, ev, n, flow) == eb.EBOF_OK
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is intact
    # the latched error is cleared by the sync that reported it
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    assert eb.ebof_stream_set_wait_limit(s, -1) == eb.EBOF_OK
    assert eb.ebof_stream_reset(s) == eb.EBOF_OK
    assert _run_batches(eb, s, ev, n, flow) == eb.EBOF_OK
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    assert _run_batches(eb, ref, ev, n, flow_ref) == eb.EBOF_OK
    assert eb.ebof_stream_sync(ref, 1)[0] == eb.EBOF_OK
    assert torch.equal(flow, flow_ref)
    # and the recovered flow of the first pair matches the oracle
    S = []
    for k in range(2):
        x, y, t, _, tb, te = ev.window(k)
        S.append(255.0 * oracle.surface_from_events(W, H, x, y, t, tb, te, connectivity=8,
                                                    n_d=1, n_f=9)["S"])
    U = oracle.flow(S[0], S[1], levels=p.levels, patch=p.patch, stride=p.stride,
                    gn_iters=p.gn_iters, gn_damping=float(p.gn_damping))
    F = flow[0].cpu().numpy()
    assert np.hypot(F[0] - U[0], F[1] - U[1]).mean() <= 0.05
    s.close()
    ref.close()


def test_allocation_failure_reports_oom_and_frees_everything(eb):
    p = eb.ebof_default_params(1280, 720)
    p.max_batch = 2
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    created = None
    try:
        for n in range(64):
            eb.ebof_debug_fail_allocation(n)
            st, s = eb.ebof_stream_create(p, 0)
            if st == eb.EBOF_OK:
                created = (n, s)
                break
            assert st == eb.EBOF_ERR_OOM, (n, st)
            assert s is None
            # every buffer allocated before the failure was freed (the
            # smallest large buffer of this stream is 1.8 MB)
            assert free0 - torch.cuda.mem_get_info()[0] < (1 << 20), n
    finally:
        eb.ebof_debug_fail_allocation(-1)
    assert created is not None and created[0] >= 10
    s = created[1]
    # an existing stream: its first host-buffer call with pageable buffers
    # needs a staging buffer, and that allocation fails
    ev = synth.rigid_objects(n_windows=3, seed=9, events=(150000, 200000))
    st, ref = eb.ebof_stream_create(p, 0)
    eb.check(st)

    def three_windows(strm):
        out = []
        for k in range(3):
            x, y, t, _, tb, te = ev.window(k)
            f = torch.empty((2, 720, 1280), dtype=torch.float32, device="cuda:0")
            eb.check(eb.ebof_process_window(strm, _dev(x), _dev(y), _dev(t), None, tb, te, f))
            out.append(f)
        return out

    three_windows(s)
    x, y, t, _, tb, te = ev.window(0)
    hflow = np.empty((2, 720, 1280), np.float32)
    eb.ebof_debug_fail_allocation(0)
    try:
        r = eb.ebof_process_window_host(s, np.ascontiguousarray(x), np.ascontiguousarray(y),
                                        np.ascontiguousarray(t), tb, te, hflow)
    finally:
        eb.ebof_debug_fail_allocation(-1)
    assert r == eb.EBOF_ERR_OOM
    assert eb.ebof_stream_reset(s) == eb.EBOF_OK
    got, want = three_windows(s), three_windows(ref)
    torch.cuda.synchronize()
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    s.close()
    ref.close()


def test_second_thread_on_a_busy_stream_is_refused(eb):
    ev = synth.rigid_objects(n_windows=9, seed=10, events=(150000, 200000))
    W, H, n = 1280, 720, 8
    p = eb.ebof_default_params(W, H)
    p.max_batch = n
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st)
    lib = eb.load()
    bx, by, bt, btb = _batch_events(ev, 1, n)
    x0, y0, t0, _, tb0, te0 = ev.window(0)
    x0, y0, t0 = _dev(x0), _dev(y0), _dev(t0)
    flow = torch.empty((n, 2, H, W), dtype=torch.float32, device="cuda:0")
    f1 = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    cs = torch.cuda.current_stream().cuda_stream
    seen = []
    for attempt in range(5):
        # about 25 ms of queued work, then thread A waits for it inside
        # ebof_stream_sync while thread B tries a call on the same stream
        for _ in range(8):
            eb.check(lib.ebof_process_windows(s.handle, n, bx.data_ptr(), by.data_ptr(),
                                              bt.data_ptr(), None, bx.numel(), btb, ev.dt,
                                              flow.data_ptr(), None, None, None, cs))
        entered = threading.Event()
        res = {}

        def a():
            entered.set()
            res["a"] = lib.ebof_stream_sync(s.handle, None, 0)

        def b():
            entered.wait()
            time.sleep(0.002)
            res["b"] = lib.ebof_process_window(s.handle, x0.data_ptr(), y0.data_ptr(),
                                               t0.data_ptr(), None, x0.numel(), tb0, te0,
                                               f1.data_ptr(), None, None, None, cs)
        ta, tb_ = threading.Thread(target=a), threading.Thread(target=b)
        ta.start()
        tb_.start()
        ta.join()
        tb_.join()
        assert res["a"] == eb.EBOF_OK
        assert res["b"] in (eb.EBOF_OK, eb.EBOF_ERR_BUSY)
        seen.append(res["b"])
        if res["b"] == eb.EBOF_ERR_BUSY:
            break
    assert eb.EBOF_ERR_BUSY in seen, seen
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    s.close()


def test_pipeline_allocation_failure_reports_oom_and_recovers(eb):
    """The pipelined call allocates its buffers (eight pyramid slots, three
    scratch sets) on first use.  A failure among them is reported as
    EBOF_ERR_OOM with nothing enqueued and everything made so far released;
    a later call allocates again and gives the flows of ordinary calls."""
    ev = synth.translating_segments(n_windows=4, seed=13)
    W, H = ev.width, ev.height
    p = eb.ebof_default_params(W, H)
    st, s = eb.ebof_stream_create(p, 0)
    eb.check(st)
    st, ref = eb.ebof_stream_create(p, 0)
    eb.check(st)
    wins = []
    for k in range(4):
        x, y, t, _, tb, te = ev.window(k)
        wins.append((_dev(x), _dev(y), _dev(t), tb, te))
    f = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
    free = []
    # the buffers are 14 allocations (slots, descriptor blocks, three sets
    # of four); fail the first, the fourth and the ninth
    for n in (0, 0, 3, 8):
        eb.ebof_debug_fail_allocation(n)
        try:
            x, y, t, tb, te = wins[0]
            assert eb.ebof_process_window_async(s, x, y, t, None, tb, te, f) == eb.EBOF_ERR_OOM
        finally:
            eb.ebof_debug_fail_allocation(-1)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    # nothing is kept from one failed attempt to the next (the first attempt
    # may leave the driver's own stream and event bookkeeping behind; the
    # slots alone are 12 MB here)
    assert max(free[1:]) - min(free[1:]) < (1 << 20), free
    got, want = [], []
    for x, y, t, tb, te in wins:
        a = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
        b = torch.empty((2, H, W), dtype=torch.float32, device="cuda:0")
        eb.check(eb.ebof_process_window_async(s, x, y, t, None, tb, te, a))
        eb.check(eb.ebof_process_window(ref, x, y, t, None, tb, te, b))
        got.append(a)
        want.append(b)
    assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
    torch.cuda.synchronize()
    for a, b in zip(got, want):
        assert torch.equal(a, b)
    s.close()
    ref.close()
