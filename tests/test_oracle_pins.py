"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test ties one oracle function to something it does not compute itself:
hand-worked cases of Alg. 1/2, the distance definition by brute force,
scipy's exact EDT, closed forms of Eq. 1-3, closed-form translations of
analytic images, exact symmetries.  ``test_planted_mistakes_are_caught``
plants mistakes in the oracle one at a time and checks that some pin fails.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2112_10591_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- Alg. 1/2
def _parse_cases(path):
    cases, cur, block = [], None, None
    for raw in open(path):
        line = raw.rstrip("\n")
        if not line.strip() or line.startswith("# ") or line == "#":
            continue
        tok = line.split()
        if tok[0] == "case":
            cur = {"name": tok[1], "E": [], "Ed": [], "Edf": []}
            block = None
        elif tok[0] in ("conn", "n_d", "n_f"):
            cur[tok[0]] = int(tok[1])
        elif tok[0] in ("E", "Ed", "Edf"):
            block = tok[0]
        elif tok[0] == "end":
            for k in ("E", "Ed", "Edf"):
                cur[k] = np.array([[c == "#" for c in r] for r in cur[k]], np.uint8)
            cases.append(cur)
            cur = None
        else:
            cur[block].append(line.strip())
    return cases


def _hand_cases(golden_dir):
    return _parse_cases(os.path.join(golden_dir, "denoise_fill_cases.txt"))


def test_denoise_fill_hand_cases(golden_dir):
    cases = _hand_cases(golden_dir)
    assert len(cases) >= 9
    for c in cases:
        Ed = oracle.denoise(c["E"], c["conn"], c["n_d"])
        Edf = oracle.fill(Ed, c["conn"], c["n_f"])
        assert np.array_equal(Ed, c["Ed"]), c["name"]
        assert np.array_equal(Edf, c["Edf"]), c["name"]


def test_disable_switches():
    # §III-B: N_d = 0 disables denoising, N_f above the neighbourhood size
    # disables filling; both then return their input unchanged.
    rng = np.random.default_rng(3)
    for conn, nf_off in ((4, 5), (8, 9)):
        for dens in (0.05, 0.3, 0.7):
            E = (rng.random((23, 31)) < dens).astype(np.uint8)
            assert np.array_equal(oracle.denoise(E, conn, 0), E)
            assert np.array_equal(oracle.fill(E, conn, nf_off), E)


def test_denoise_monotone_in_threshold():
    # raising N_d can only remove more pixels; raising N_f only fills fewer
    rng = np.random.default_rng(4)
    E = (rng.random((40, 40)) < 0.3).astype(np.uint8)
    for conn in (4, 8):
        prev = E
        for nd in range(0, conn + 2):
            cur = oracle.denoise(E, conn, nd)
            assert np.all(cur <= prev)
            prev = cur
        prev = None
        for nf in range(0, conn + 2):
            cur = oracle.fill(E, conn, nf)
            if prev is not None:
                assert np.all(cur <= prev)
            prev = cur


# ---------------------------------------------------------------- §III-A
def test_edge_image_window_and_bounds():
    x = np.array([0, 5, 5, 9, 10, 2, 3], np.uint16)
    y = np.array([0, 1, 1, 3, 0, 4, 2], np.uint16)
    t = np.array([100, 100, 150, 199, 120, 99, 200], np.int64)
    E, st = oracle.edge_image(10, 4, x, y, t, 100, 200)
    want = np.zeros((4, 10), np.uint8)
    want[0, 0] = want[1, 5] = want[3, 9] = 1
    assert np.array_equal(E, want)
    # given, in window, outside window (t=99, t=200), in window off-image (x=10)
    assert list(st) == [7, 5, 2, 1]


# ---------------------------------------------------------------- §III-C EDT
def test_edt_matches_brute_force_small():
    rng = np.random.default_rng(5)
    for H in range(1, 13):
        for W in range(1, 13):
            for dens in (0.0, 0.05, 0.5, 1.0):
                E = (rng.random((H, W)) < dens).astype(np.uint8)
                if dens > 0 and E.sum() == 0:
                    E[rng.integers(H), rng.integers(W)] = 1
                assert np.array_equal(oracle.edt(E), oracle.edt_brute(E)), (H, W, dens)


def test_edt_matches_scipy_exact_edt():
    ndi = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(6)
    for H, W, dens in ((64, 64, 0.01), (37, 53, 0.2), (50, 90, 0.002)):
        E = (rng.random((H, W)) < dens).astype(np.uint8)
        E[rng.integers(H), rng.integers(W)] = 1
        d = ndi.distance_transform_edt(E == 0)
        want = np.rint(d * d).astype(np.int64)
        assert np.array_equal(oracle.edt(E).astype(np.int64), want)


def test_edt_single_site_closed_form_and_empty():
    E = np.zeros((17, 29), np.uint8)
    E[5, 20] = 1
    yy, xx = np.mgrid[0:17, 0:29]
    assert np.array_equal(oracle.edt(E), (xx - 20) ** 2 + (yy - 5) ** 2)
    D = oracle.edt(np.zeros((7, 9), np.uint8))
    assert np.all(D == oracle.INF_D)


# ---------------------------------------------------------------- Eq. 1-3
def test_surface_closed_forms():
    # Eq. 3 quotes alpha ~= d_sat / 5.541, i.e. ln(255) = 5.5413
    assert abs(6.0 / oracle.alpha_from_dsat(6.0) - 5.541) < 1e-3
    # §IV-A: alpha = 1.08 for d_sat = 6 px is the rounding of 6 / ln 255
    assert round(oracle.alpha_from_dsat(6.0), 2) == 1.08
    a = oracle.alpha_from_dsat(6.0)
    S = oracle.surface(np.array([0, 36, oracle.INF_D], np.int32), a)
    assert S[0] == 0.0                                 # 0 on edge pixels
    assert abs(S[1] - (1.0 - 1.0 / 255.0)) < 1e-12      # saturation at d_sat
    assert S[2] == 1.0                                  # no edge at all
    D = np.arange(0, 2000, dtype=np.int32)
    S = oracle.surface(D, 1.08)
    assert np.all(np.diff(S) >= 0)                      # monotone in distance
    assert abs(S[4] - (1 - math.exp(-2.0 / 1.08))) < 1e-15
    assert abs(S[1] - (1 - math.exp(-1.0 / 1.08))) < 1e-15


# ---------------------------------------------------------------- §IV-D ablation surfaces
def test_ablation_surfaces_closed_forms():
    D = np.array([0, 1, 4, 36, 49, 50, oracle.INF_D], np.int32)
    lin = oracle.surface_mode(D, oracle.SURFACE_LINEAR)
    lb = oracle.surface_mode(D, oracle.SURFACE_BOUNDED, d_sat=6.0)
    lg = oracle.surface_mode(D, oracle.SURFACE_LOG)
    assert lin[:6].tolist() == [0.0, 1.0, 2.0, 6.0, 7.0, 7.0710678118654755]
    assert lb[:6].tolist() == [0.0, 1.0, 2.0, 6.0, 6.0, 6.0]          # the 6 px bound
    assert abs(lg[1] - 0.6931471805599453) < 1e-15                    # ln 2
    assert abs(lg[3] - 1.9459101490553132) < 1e-15                    # ln 7
    assert abs(lg[4] - 2.0794415416798357) < 1e-15                    # ln 8
    assert lg[0] == 0.0
    # no edge pixel: a constant (finite) image for every surface
    assert lin[6] == math.sqrt(2147483647.0) and lb[6] == 6.0 and np.isfinite(lg[6])
    # mode 0 is Eq. 1 itself
    Dd = np.arange(0, 400, dtype=np.int32)
    assert np.array_equal(oracle.surface_mode(Dd, oracle.SURFACE_EXP, 1.08), oracle.surface(Dd))
    # shapes of the plotted variants: DS_LB = min(DS_L, 6) <= DS_L, DS_Log <= DS_L
    L = oracle.surface_mode(Dd, oracle.SURFACE_LINEAR)
    B = oracle.surface_mode(Dd, oracle.SURFACE_BOUNDED)
    G = oracle.surface_mode(Dd, oracle.SURFACE_LOG)
    assert np.all(B <= L) and np.all(G <= L) and np.all(np.diff(G) > 0)
    assert np.array_equal(B, np.minimum(L, 6.0))


def test_ablation_intensity_scale():
    # reading S2: every surface puts 255 at d_sat = 6 px, except Eq. 1 whose
    # value there is 1 - 1/255 with alpha = 6 / ln 255 (Eq. 3), i.e. 254
    a = oracle.alpha_from_dsat(6.0)
    D = np.array([36], np.int32)
    for mode in (oracle.SURFACE_LINEAR, oracle.SURFACE_BOUNDED, oracle.SURFACE_LOG):
        v = oracle.intensity_gain(mode, 6.0) * oracle.surface_mode(D, mode, a, 6.0)[0]
        assert abs(v - 255.0) < 1e-12, mode
    v = oracle.intensity_gain(oracle.SURFACE_EXP) * oracle.surface_mode(D, 0, a)[0]
    assert abs(v - 254.0) < 1e-9


@pytest.mark.parametrize("mode", [1, 2, 3])
def test_ablation_surface_flow_recovers_shift(mode):
    # the flow block on each ablation surface recovers an integer shift of an
    # edge image on the edge pixels (the same scene as the Eq. 1 pin below)
    rng = np.random.default_rng(11)
    H, W = 120, 160
    E = np.zeros((H, W), np.uint8)
    for _ in range(300):
        x, y = rng.integers(0, W - 2), rng.integers(0, H - 2)
        E[y:y + 2, x:x + 2] = 1
    E2 = np.zeros_like(E)
    E2[0:H - 1, 3:W] = E[1:H, 0:W - 3]
    g = oracle.intensity_gain(mode)
    U = oracle.flow(g * oracle.surface_mode(oracle.edt(E), mode),
                    g * oracle.surface_mode(oracle.edt(E2), mode))
    m = E2.astype(bool)
    m[:16] = m[-16:] = False
    m[:, :16] = m[:, -16:] = False
    e = np.hypot(U[0] - 3.0, U[1] + 1.0)[m]
    assert e.mean() <= 0.1, e.mean()


# ---------------------------------------------------------------- §IV-C FWL
def _point_track():
    # one point moving 4 px per window along x, seen at tau = 0, 1/4, 1/2, 3/4
    # of a 100 us window: events at x = 2, 3, 4, 5 on row 5 of a 10 x 10 image
    x = np.array([2, 3, 4, 5], np.uint16)
    y = np.full(4, 5, np.uint16)
    t = np.array([1000, 1025, 1050, 1075], np.int64)
    return x, y, t


def test_fwl_zero_flow_is_one():
    x, y, t = _point_track()
    U = np.zeros((2, 10, 10))
    f, vc, vu = oracle.fwl(10, 10, x, y, t, None, 1000, 1100, U)
    assert f == 1.0 and vc == vu


def test_fwl_point_track_closed_form():
    x, y, t = _point_track()
    U = np.zeros((2, 10, 10))
    U[0] = 4.0
    img = oracle.iwe(10, 10, x, y, t, None, 1000, 1100, U)
    assert img[5, 2] == 4.0 and img.sum() == 4.0        # all four land on x = 2
    f, vc, vu = oracle.fwl(10, 10, x, y, t, None, 1000, 1100, U)
    # 100 pixels: var_u = 4/100 - (4/100)^2, var_c = 16/100 - (4/100)^2
    assert abs(vu - 0.0384) < 1e-15 and abs(vc - 0.1584) < 1e-15
    assert abs(f - 4.125) < 1e-12


def test_fwl_bilinear_split_polarity_and_bounds():
    # an event half way through the window with flow (1, 0) lands between two
    # pixels; a negative event votes -1; events outside the window or image,
    # and votes moved outside the image, do not count
    x = np.array([3, 6, 7, 0, 9], np.uint16)
    y = np.array([2, 2, 2, 0, 12], np.uint16)
    t = np.array([50, 0, 100, 50, 10], np.int64)
    p = np.array([1, -1, 1, 1, 1], np.int8)
    U = np.zeros((2, 10, 10))
    U[0] = 1.0
    img = oracle.iwe(10, 10, x, y, t, p, 0, 100, U)
    want = np.zeros((10, 10))
    want[2, 2] = want[2, 3] = 0.5      # x = 3 - 0.5
    want[2, 6] = -1.0                  # tau = 0: not moved, polarity -1
    want[0, 0] = 0.5                   # x = 0 - 0.5: the vote at x = -1 is dropped
    assert np.array_equal(img, want)   # t = 100 is outside [0, 100); y = 12 outside


def test_fwl_prefers_the_true_flow():
    ev = synth.translating_segments(n_windows=1, seed=5, velocity=(3.0, -1.5), noise_frac=0.0)
    x, y, t, p, tb, te = ev.window(0)
    U = np.zeros((2, ev.height, ev.width))
    U[0], U[1] = 3.0, -1.5
    good = oracle.fwl(ev.width, ev.height, x, y, t, p, tb, te, U)[0]
    bad = oracle.fwl(ev.width, ev.height, x, y, t, p, tb, te, -U)[0]
    assert good > 1.0 > bad


# ---------------------------------------------------------------- §IV-C AEE vs ground truth
def _aee(U, G, m):
    e = np.hypot(U[0] - G[0], U[1] - G[1])[m]
    mag = np.hypot(G[0], G[1])[m]
    return e.mean(), ((e > 3.0) & (e > 0.05 * mag)).mean()


def test_flow_recovers_generator_motion_on_translating_scene():
    # the whole path on the 346x260 workload against the generator's own
    # motion at the previous window's event pixels: AEE (§IV-C) well below
    # the zero flow's and no outliers (error > 3 px and > 5 % of the motion)
    ev = synth.translating_segments(keep_truth=True)
    w0, w1 = ev.window(0), ev.window(1)
    _, _, U = oracle.process_pair(ev.width, ev.height, (w0[0], w0[1], w0[2], w0[4], w0[5]),
                                  (w1[0], w1[1], w1[2], w1[4], w1[5]))
    G, m = ev.true_flow(1)
    assert np.allclose(G[0][m], 3.0) and np.allclose(G[1][m], -1.5)
    aee, out = _aee(U, G, m)
    zero, _ = _aee(np.zeros_like(U), G, m)
    assert aee <= 0.6 and out == 0.0 and zero > 3.0, (aee, out, zero)


# ---------------------------------------------------------------- pyramid
def test_downsample_and_gradients_closed_forms():
    I = np.arange(30, dtype=np.float64).reshape(5, 6)
    D = oracle.downsample(I)
    assert D.shape == (2, 3)
    # 2x2 means of rows 0-1 and 2-3 (last row of the odd height is dropped)
    assert np.allclose(D, [[3.5, 5.5, 7.5], [15.5, 17.5, 19.5]])
    yy, xx = np.mgrid[0:9, 0:11].astype(np.float64)
    Ix, Iy = oracle.gradients(2.5 * xx - 1.25 * yy + 7)
    assert np.allclose(Ix[:, 1:-1], 2.5) and np.allclose(Iy[1:-1, :], -1.25)
    assert np.allclose(Ix[:, 0], 1.25) and np.allclose(Ix[:, -1], 1.25)
    assert np.allclose(Iy[0, :], -0.625) and np.allclose(Iy[-1, :], -0.625)


def test_patch_grid_and_levels():
    o = oracle.patch_origins(346, 8, 4)
    assert len(o) == 86 and o[0] == 0 and o[-1] == 338 and o[-2] == 336
    assert len(oracle.patch_origins(260, 8, 4)) == 64
    assert len(oracle.patch_origins(1280, 12, 4)) == 318
    assert len(oracle.patch_origins(720, 12, 4)) == 178
    assert len(oracle.patch_origins(7, 8, 4)) == 0
    assert oracle.levels_used(346, 260, 3, 8) == 3
    assert oracle.levels_used(1280, 720, 5, 12) == 5
    assert oracle.levels_used(40, 40, 5, 12) == 2
    assert oracle.levels_used(7, 40, 3, 8) == 0


# ---------------------------------------------------------------- flow
def _texture(W, H, v=(0.0, 0.0)):
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    xx = xx - v[0]
    yy = yy - v[1]
    return 127.5 + 60.0 * np.sin(2 * np.pi * xx / 23.0) * np.cos(2 * np.pi * yy / 17.0)


@pytest.mark.parametrize("v", [(0.3, -0.2), (1.7, 0.9), (3.0, -1.5)])
def test_flow_recovers_closed_form_translation(v):
    I0, I1 = _texture(128, 96), _texture(128, 96, v)
    U = oracle.flow(I0, I1)
    e = np.hypot(U[0] - v[0], U[1] - v[1])[16:-16, 16:-16]
    assert e.mean() <= 0.02, e.mean()


def test_patch_search_recovers_translation():
    v = (1.25, -0.6)
    I0, I1 = _texture(96, 80), _texture(96, 80, v)
    Ix, Iy = oracle.gradients(I0)
    up, fl = oracle.patch_search(I0, Ix, Iy, I1, None, 8, 4, 12)
    inner = (slice(3, -3), slice(3, -3))
    assert np.all(fl[inner] == 0)
    e = np.hypot(up[0][inner] - v[0], up[1][inner] - v[1])
    assert e.mean() < 0.05


def test_zero_motion_gives_zero_flow():
    I0 = _texture(64, 48)
    assert np.array_equal(oracle.flow(I0, I0), np.zeros((2, 48, 64)))


def test_flat_images_give_zero_flow_without_nan():
    F = np.full((48, 64), 200.0)
    U = oracle.flow(F, np.full((48, 64), 180.0))
    assert not np.isnan(U).any() and np.all(U == 0)
    Ix, Iy = oracle.gradients(F)
    up, fl = oracle.patch_search(F, Ix, Iy, F, None, 8, 4, 12)
    assert np.all(fl == 1)


def test_patch_start_from_coarser_level():
    # F3: on a flat image every patch keeps its start value, 2 * U_{l+1}
    # at coarse pixel round-half-down(centre / 2).  Worked by hand for
    # ps = 8, stride 4: origins 0, 4, 8 -> centres 3.5, 7.5, 11.5 -> coarse
    # indices 2, 4, 6 (= round-half-down of 1.75, 3.75, 5.75).
    W = H = 20
    Wc = Hc = 10
    Uc = np.zeros((2, Hc, Wc))
    Uc[0] = np.arange(Wc)[None, :] + 100.0 * np.arange(Hc)[:, None]
    Uc[1] = -Uc[0]
    F = np.full((H, W), 50.0)
    Ix, Iy = oracle.gradients(F)
    up, fl = oracle.patch_search(F, Ix, Iy, F, Uc, 8, 4, 12)
    assert up.shape == (2, 4, 4)        # origins 0, 4, 8, 12
    idx = [2, 4, 6, 8]
    for j in range(4):
        for i in range(4):
            assert up[0, j, i] == 2.0 * (idx[i] + 100.0 * idx[j])
            assert up[1, j, i] == -up[0, j, i]


def test_reset_rule_on_unrelated_images():
    rng = np.random.default_rng(9)
    I0 = rng.random((48, 48)) * 255.0
    I1 = rng.random((48, 48)) * 255.0
    Ix, Iy = oracle.gradients(I0)
    up, fl = oracle.patch_search(I0, Ix, Iy, I1, None, 8, 4, 12)
    reset = fl == 2
    assert np.all(np.hypot(up[0], up[1])[~reset] <= 8.0 + 1e-12)
    assert np.all(up[:, reset] == 0.0)


def test_densify_constant_flow_and_flat_weights():
    # equal patch flows give that flow everywhere; with flat images every
    # weight is equal, so U is the plain mean of the covering patch flows
    I0 = _texture(30, 22)
    up = np.zeros((2, 5, 7))
    up[0] = 1.5
    up[1] = -0.25
    U = oracle.densify(I0, I0, up, 8, 4)
    assert np.allclose(U[0], 1.5) and np.allclose(U[1], -0.25)
    F0, F1 = np.full((22, 30), 10.0), np.full((22, 30), 13.0)
    rng = np.random.default_rng(2)
    up = rng.standard_normal((2, 5, 7))
    U = oracle.densify(F0, F1, up, 8, 4)
    ox, oy = oracle.patch_origins(30, 8, 4), oracle.patch_origins(22, 8, 4)
    for y, x in ((0, 0), (5, 9), (21, 29), (10, 24)):
        cov = [(j, i) for j in range(len(oy)) for i in range(len(ox))
               if oy[j] <= y < oy[j] + 8 and ox[i] <= x < ox[i] + 8]
        want = np.mean([up[0, j, i] for j, i in cov])
        assert abs(U[0, y, x] - want) < 1e-12


def test_densify_weights_closed_form():
    # I0 = I1 = 4x: a patch flow (1, 0) leaves the residual 4 (weight 1/4),
    # a flow (0, 0) the residual 0 (weight 1).  Even patch columns carry
    # (1, 0), odd ones (0, 0); an inner pixel lies in two patch columns, one
    # of each, and two patch rows, so U = (2 * 1/4) / (2 * 1/4 + 2) = 0.2.
    W, H = 40, 24
    I = 4.0 * np.mgrid[0:H, 0:W][1].astype(np.float64)
    npx = len(oracle.patch_origins(W, 8, 4))
    npy = len(oracle.patch_origins(H, 8, 4))
    up = np.zeros((2, npy, npx))
    up[0, :, 0::2] = 1.0
    U = oracle.densify(I, I, up, 8, 4)
    assert np.allclose(U[0, 4:20, 4:30], 0.2, atol=1e-12)
    assert np.all(U[1] == 0.0)


def test_variational_smooths_without_data():
    # flat images carry no data term, so only the smoothness term acts and
    # an isolated spike in the flow is flattened out
    F = np.full((20, 24), 100.0)
    Ix, Iy = oracle.gradients(F)
    U = np.zeros((2, 20, 24))
    U[0, 10, 12] = 1.0
    U[1, 5, 5] = -2.0
    R = oracle.variational(F, Ix, Iy, F, U)
    assert np.ptp(R[0]) < 0.1 * np.ptp(U[0])
    assert np.ptp(R[1]) < 0.1 * np.ptp(U[1])


def test_variational_keeps_exact_solution():
    # an exact integer translation warps exactly, so the true constant flow
    # has zero data and gradient residuals and zero smoothness: dU = 0
    I = _texture(60, 50)
    I1 = np.zeros_like(I)
    I1[:, 2:] = I[:, :-2]
    I1[:, :2] = I[:, :2]
    Ix, Iy = oracle.gradients(I)
    U = np.zeros((2, 50, 60))
    U[0] = 2.0
    R = oracle.variational(I, Ix, Iy, I1, U)
    # the two rightmost columns warp off the image; their effect decays
    # within a few tens of pixels
    assert np.abs(R - U)[:, :, :30].max() < 1e-8


def _var_sor_case(golden_dir):
    """The hand-worked sweep of tests/golden/var_sor_sweep.txt."""
    from fractions import Fraction
    rows = {}
    with open(os.path.join(golden_dir, "var_sor_sweep.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *vals = line.split()
            rows[k] = [float(Fraction(v)) for v in vals]
    W, H = int(rows["grid"][0]), int(rows["grid"][1])
    pl = {k: np.array(rows[k]).reshape(H, W) for k in oracle.VAR_PLANES}
    U = np.stack([np.array(rows["u"]), np.array(rows["v"])]).reshape(2, H, W)
    dU0 = np.stack([np.array(rows["du_start"]), np.array(rows["dv_start"])]).reshape(2, H, W)
    want = np.stack([np.array(rows["du"]), np.array(rows["dv"])]).reshape(2, H, W)
    return pl, U, dU0, int(rows["sweeps"][0]), rows["omega"][0], want


def test_var_sor_hand_worked_sweep(golden_dir):
    # one red-black sweep of the Euler-Lagrange system, worked by hand on a
    # 2x2 grid with a gradient-constancy cross term, unequal smoothness
    # weights and a relaxation factor that acts on a non-zero start value
    pl, U, dU0, sweeps, omega, want = _var_sor_case(golden_dir)
    got = oracle.var_sor(pl, U, dU0, sweeps, omega)
    assert np.abs(got - want).max() <= 1e-14, (got, want)


def _var_energy(pl, U, dU):
    """The linearised energy whose Euler-Lagrange equations the SOR solves:
    squared data and gradient-constancy residuals of the increment plus the
    smoothness of U + dU over 4-neighbour pairs, with the frozen weights."""
    du, dv = dU
    e = pl["ad"] * (pl["Ix"] * du + pl["Iy"] * dv + pl["Iz"]) ** 2
    e = e + pl["ag"] * ((pl["Ixx"] * du + pl["Ixy"] * dv + pl["Ixz"]) ** 2
                        + (pl["Ixy"] * du + pl["Iyy"] * dv + pl["Iyz"]) ** 2)
    total = e.sum()
    a = pl["as"]
    for c in range(2):
        f = U[c] + dU[c]
        wx = 0.5 * (a[:, 1:] + a[:, :-1])
        wy = 0.5 * (a[1:, :] + a[:-1, :])
        total += (wx * (f[:, 1:] - f[:, :-1]) ** 2).sum()
        total += (wy * (f[1:, :] - f[:-1, :]) ** 2).sum()
    return total


def _energy_gradient(pl, U, dU, h=1e-3):
    # the energy is quadratic in dU, so central differences are exact up to
    # rounding
    g = np.zeros_like(dU)
    for idx in np.ndindex(*dU.shape):
        d = dU.copy()
        d[idx] += h
        ep = _var_energy(pl, U, d)
        d[idx] -= 2 * h
        em = _var_energy(pl, U, d)
        g[idx] = (ep - em) / (2 * h)
    return g


def _warped_pair(W, H):
    """A textured image and a non-translational copy (a slight rotation and
    scaling about the centre), so the mixed derivative Ixy is not zero."""
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    cx, cy = (W - 1) / 2, (H - 1) / 2
    th, sc = 0.08, 1.05
    xs = cx + sc * (np.cos(th) * (xx - cx) - np.sin(th) * (yy - cy))
    ys = cy + sc * (np.sin(th) * (xx - cx) + np.cos(th) * (yy - cy))

    def tex(x, y):
        return (127.5 + 60 * np.sin(2 * np.pi * x / 9.0) * np.cos(2 * np.pi * y / 7.0)
                + 25 * np.sin(x * y / 11.0))
    return tex(xx, yy), tex(xs, ys)


def test_var_sor_converges_to_the_energy_minimum():
    # Many sweeps of the SOR solve the linear system; its solution must be the
    # stationary point of the linearised energy, whose gradient is taken here
    # by differentiating the energy itself, not from the equations.  A wrong
    # or missing coefficient (e.g. the gradient-constancy coupling in a12)
    # moves the solution off the minimum.
    W, H = 13, 11
    I0, I1 = _warped_pair(W, H)
    I0x, I0y = oracle.gradients(I0)
    rng = np.random.default_rng(5)
    U = 0.6 * rng.standard_normal((2, H, W))
    pl = oracle.var_linearise(I0, I0x, I0y, I1, U)
    assert np.abs(pl["Ixy"]).max() > 1.0 and pl["ag"].max() > 0
    g0 = _energy_gradient(pl, U, np.zeros((2, H, W)))
    dU = oracle.var_sor(pl, U, np.zeros((2, H, W)), 6000, 1.6)
    g = _energy_gradient(pl, U, dU)
    assert np.abs(g).max() <= 1e-7 * np.abs(g0).max(), (np.abs(g).max(), np.abs(g0).max())
    # and it is a minimum: any perturbation raises the energy
    e = _var_energy(pl, U, dU)
    for _ in range(5):
        assert _var_energy(pl, U, dU + 1e-2 * rng.standard_normal(dU.shape)) > e


def test_var_linearise_planes_closed_forms():
    # On a quadratic image central differences are exact away from the
    # border, so the warped image's derivative planes have closed forms; an
    # integer flow warps exactly.  Where the warp leaves the image the data
    # and gradient terms are dropped, and a constant flow has the smoothness
    # weight Psi'(0) alpha = alpha / (2 eps).
    W, H = 16, 12
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)

    def quad(x, y):
        return 100 + 3 * x + 2 * y + 0.5 * x * x + 0.25 * x * y - 0.3 * y * y
    I1 = quad(xx, yy)
    I0 = I1 - 7.0
    I0x = np.zeros_like(I1)
    I0y = np.full_like(I1, 2.0)
    U = np.zeros((2, H, W))
    U[0] = 1.0
    pl = oracle.var_linearise(I0, I0x, I0y, I1, U, delta=5.0, gamma=10.0, alpha=20.0)
    i = (slice(2, H - 2), slice(2, W - 3))   # x + 1 stays two pixels inside
    X, Y = xx[i] + 1.0, yy[i]
    assert np.allclose(pl["Ix"][i], 3 + X + 0.25 * Y, atol=1e-9)
    assert np.allclose(pl["Iy"][i], 2 + 0.25 * X - 0.6 * Y, atol=1e-9)
    assert np.allclose(pl["Ixx"][i], 1.0, atol=1e-9)
    assert np.allclose(pl["Ixy"][i], 0.25, atol=1e-9)
    assert np.allclose(pl["Iyy"][i], -0.6, atol=1e-9)
    assert np.allclose(pl["Iz"][i], quad(X, Y) - I0[i], atol=1e-9)
    assert np.allclose(pl["Ixz"][i], 3 + X + 0.25 * Y, atol=1e-9)
    assert np.allclose(pl["Iyz"][i], 0.25 * X - 0.6 * Y, atol=1e-9)
    assert np.all(pl["ad"][:, :W - 1] > 0) and np.all(pl["ag"][:, :W - 1] > 0)
    assert np.all(pl["ad"][:, W - 1] == 0) and np.all(pl["ag"][:, W - 1] == 0)
    assert np.allclose(pl["as"], 20.0 / (2 * 1e-3), rtol=1e-12)


def test_event_surface_integer_shift():
    # an edge image shifted by (3, -1) gives exactly shifted D and S, and the
    # flow on the shifted edge pixels recovers (3, -1)
    rng = np.random.default_rng(11)
    H, W = 120, 160
    E = np.zeros((H, W), np.uint8)
    for _ in range(300):
        x, y = rng.integers(0, W - 2), rng.integers(0, H - 2)
        E[y:y + 2, x:x + 2] = 1
    E2 = np.zeros_like(E)
    E2[0:H - 1, 3:W] = E[1:H, 0:W - 3]
    D, D2 = oracle.edt(E), oracle.edt(E2)
    inner = (slice(20, H - 20), slice(20, W - 20))
    assert np.array_equal(D2[20:H - 20, 20:W - 20], D[21:H - 19, 17:W - 23])
    U = oracle.flow(255 * oracle.surface(D), 255 * oracle.surface(D2))
    m = E2.astype(bool)
    m[:16] = m[-16:] = False
    m[:, :16] = m[:, -16:] = False
    e = np.hypot(U[0] - 3.0, U[1] + 1.0)[m]
    assert e.mean() <= 0.1, e.mean()
    del inner


def test_flow_is_well_conditioned():
    # Rounding the input surfaces to FP32 must move the flow only a little:
    # the damped Gauss-Newton step keeps edge-like (aperture) patches from
    # drifting and flipping the reset rule.  With the undamped step this
    # scene moves by 0.032 px on average; damped, by 0.007 px.
    from paper_2112_10591_gb300 import synth
    W, H = 640, 360
    s = synth.rigid_objects(width=W, height=H, n_windows=2, events=(60000, 100000), seed=4)
    S = []
    for k in range(2):
        x, y, t, _, tb, te = s.window(k)
        S.append(255.0 * oracle.surface_from_events(W, H, x, y, t, tb, te)["S"])
    S32 = [a.astype(np.float32).astype(np.float64) for a in S]
    U = oracle.flow(S[0], S[1], levels=4, patch=12)
    U32 = oracle.flow(S32[0], S32[1], levels=4, patch=12)
    assert np.hypot(*(U - U32)).mean() <= 0.015


def test_transpose_symmetry():
    I0, I1 = _texture(96, 96), _texture(96, 96, (1.7, 0.9))
    U = oracle.flow(I0, I1)
    Ut = oracle.flow(I0.T.copy(), I1.T.copy())
    assert np.abs(U[0] - Ut[1].T).max() <= 1e-3
    assert np.abs(U[1] - Ut[0].T).max() <= 1e-3


def test_complement_invariance():
    # 1 - d_exp is 1 on edges; the flow is invariant to I -> 255 - I
    I0, I1 = _texture(80, 64), _texture(80, 64, (2.2, -0.7))
    U = oracle.flow(I0, I1)
    Uc = oracle.flow(255.0 - I0, 255.0 - I1)
    assert np.abs(U - Uc).max() <= 1e-6


# ---------------------------------------------------------------- mutations
def _pins_fail():
    """Run a fast subset of the pins; return True if any of them fails."""
    import tests.test_oracle_pins as me
    checks = [
        lambda: me.test_denoise_fill_hand_cases(os.path.join(os.path.dirname(__file__), "golden")),
        me.test_edt_single_site_closed_form_and_empty,
        me.test_surface_closed_forms,
        me.test_ablation_surfaces_closed_forms,
        me.test_fwl_point_track_closed_form,
        me.test_downsample_and_gradients_closed_forms,
        lambda: me.test_flow_recovers_closed_form_translation((1.7, 0.9)),
        me.test_patch_search_recovers_translation,
        me.test_densify_constant_flow_and_flat_weights,
        me.test_densify_weights_closed_form,
        me.test_variational_keeps_exact_solution,
        me.test_variational_smooths_without_data,
        me.test_event_surface_integer_shift,
        lambda: me.test_var_sor_hand_worked_sweep(os.path.join(os.path.dirname(__file__), "golden")),
        me.test_var_sor_converges_to_the_energy_minimum,
        me.test_var_linearise_planes_closed_forms,
    ]
    for c in checks:
        try:
            c()
        except AssertionError:
            return True
    return False


@pytest.mark.parametrize("k", range(1, 14))
def test_planted_mistakes_are_caught(k):
    try:
        oracle.set_mutation(k)
        assert _pins_fail(), "mistake %d went unnoticed" % k
    finally:
        oracle.set_mutation(0)
    assert not _pins_fail()
