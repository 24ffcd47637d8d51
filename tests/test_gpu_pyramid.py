"""Pyramid parity (A5, reading F1 of the flow block of §III-D): every level's
box-mean image and its central differences, read back through
ebof_stream_get_pyramid, against the FP64 oracle's downsample() and
gradients() (themselves pinned by closed forms), element by element.

Tolerances follow from the arithmetic (M = 255, the largest intensity;
u = 2^-24, FP32's unit roundoff; h = 2^-11, FP16's):
  * FP32 storage: level 0 is 255 * S rounded once (u M); a box mean of four
    FP32 values is three rounded sums of at most 4 M and an exact * 0.25
    (at most 2.25 u M more per level); a central difference 0.5 (a - b) adds
    one rounding of at most u M / 2.  Level l: I within (1 + 2.25 l) u M,
    Ix and Iy within (1.5 + 2.25 l) u M.
  * FP16 storage (the complement 255 (1 - S) is stored): each stored level
    and gradient is rounded to half once more, h M per level and h M / 2 per
    gradient on top of the FP32 terms (with one more FP32 rounding of 1 - S).
"""
import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

M, U32, U16 = 255.0, 2.0 ** -24, 2.0 ** -11


@pytest.fixture(scope="module")
def eb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2112_10591_gb300 as m
    m.load()
    return m


def _surface(W, H, seed):
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    S = 0.5 + 0.3 * np.sin(xx / 7.3) * np.cos(yy / 5.1) + 0.1 * rng.standard_normal((H, W))
    return np.clip(S, 0.0, 1.0).astype(np.float32)


def _read(eb, s, W, H, level):
    w, h = W >> level, H >> level
    out = [torch.full((h, w), float("nan"), dtype=torch.float32, device="cuda")
           for _ in range(3)]
    eb.check(eb.ebof_stream_get_pyramid(s, level, *out))
    torch.cuda.synchronize()
    return [o.cpu().numpy().astype(np.float64) for o in out]


@pytest.mark.parametrize("W,H,storage", [(1280, 720, 0), (193, 129, 0), (346, 260, 1),
                                         (129, 97, 1)])
def test_pyramid_levels_and_gradients_match_oracle(eb, W, H, storage):
    prm = eb.ebof_default_params(W, H)
    prm.storage = storage
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    S = _surface(W, H, W + H + storage)
    flow = torch.empty((2, H, W), dtype=torch.float32, device="cuda")
    assert eb.ebof_process_surface(s, torch.from_numpy(S).cuda(), flow) == eb.EBOF_NO_PREVIOUS
    L = oracle.levels_used(W, H, prm.levels, prm.patch)
    assert L >= 2
    S64 = S.astype(np.float64)
    I = 255.0 * S64 if storage == 0 else 255.0 * (1.0 - S64)
    for l in range(L):
        if l > 0:
            I = oracle.downsample(I)
        Ix, Iy = oracle.gradients(I)
        gI, gIx, gIy = _read(eb, s, W, H, l)
        assert gI.shape == I.shape
        if storage == 0:
            tol_i = (1.0 + 2.25 * l) * U32 * M
            tol_g = (1.5 + 2.25 * l) * U32 * M
        else:
            tol_i = (l + 1) * U16 * M + (2.0 + 2.25 * l) * U32 * M
            tol_g = tol_i + 0.5 * U16 * M + 0.5 * U32 * M
        di = np.abs(gI - I).max()
        dx, dy = np.abs(gIx - Ix).max(), np.abs(gIy - Iy).max()
        print("%dx%d storage %d level %d: |dI| %.3g (bound %.3g), |dIx| %.3g, |dIy| %.3g "
              "(bound %.3g)" % (W, H, storage, l, di, tol_i, dx, dy, tol_g))
        assert di <= tol_i and dx <= tol_g and dy <= tol_g, l
    # errors: levels outside the pyramid
    for bad in (-1, L):
        assert eb.ebof_stream_get_pyramid(s, bad, None, None, None) == eb.EBOF_ERR_INVALID_ARG
    s.close()


def test_pyramid_before_the_first_window(eb):
    prm = eb.ebof_default_params(160, 120)
    st, s = eb.ebof_stream_create(prm, 0)
    eb.check(st)
    I = torch.zeros((120, 160), dtype=torch.float32, device="cuda")
    assert eb.ebof_stream_get_pyramid(s, 0, I, None, None) == eb.EBOF_NO_PREVIOUS
    s.close()


def _windows(ev, n):
    out = []
    for k in range(n):
        x, y, t, _, tb, te = ev.window(k)
        out.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (x, y, t))
                   + (tb, te))
    return out


def test_pyramid_after_pipelined_calls_equals_ordinary(eb):
    """The newest window's pyramid read after pipelined calls (handed back
    from the pipeline's own slots) equals the one after ordinary calls, bit
    for bit, at every level; reading it in between changes no later flow."""
    n = 6
    ev = synth.rigid_objects(n_windows=n, seed=46, events=(40000, 90000), width=640,
                             height=360, n_edges=120)
    wins = _windows(ev, n)
    prm = eb.ebof_default_params(640, 360)
    L = oracle.levels_used(640, 360, prm.levels, prm.patch)
    res = []
    for kind in ("o", "a"):
        st, s = eb.ebof_stream_create(prm, 0)
        eb.check(st)
        flows = []
        for k, (x, y, t, tb, te) in enumerate(wins):
            f = torch.empty((2, 360, 640), dtype=torch.float32, device="cuda")
            call = eb.ebof_process_window if kind == "o" else eb.ebof_process_window_async
            eb.check(call(s, x, y, t, None, tb, te, f))
            flows.append(f)
            if k == 3:  # a read between calls
                _read(eb, s, 640, 360, 1)
        assert eb.ebof_stream_sync(s, 1)[0] == eb.EBOF_OK
        res.append(([_read(eb, s, 640, 360, l) for l in range(L)],
                    [f.cpu().numpy() for f in flows]))
        s.close()
    (pa, fa), (pb, fb) = res
    for l in range(L):
        for a, b in zip(pa[l], pb[l]):
            assert np.array_equal(a, b), l
    for k in range(n):
        assert np.array_equal(fa[k], fb[k]), k
