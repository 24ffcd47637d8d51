"""FP64 CPU oracle of the event-to-flow path (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (the CUDA library and its
Python binding) never does, and shares no code with it.

The arithmetic lives in ``ebof_oracle.c`` (plain C, double precision); this
module only builds that file with gcc, loads it with ctypes and marshals
numpy arrays.  Each wrapper names the passage of the paper it follows; the
C source states the readings taken where the paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ebof_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF_D = 2147483647


def build(force: bool = False) -> str:
    """Compile ebof_oracle.c into oracle/_build/liboracle.so with gcc."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp,
                    _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _declare(L):
    vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    L.orc_edge_image.argtypes = [i32, i32, i64, vp, vp, vp, i64, i64, vp, vp]
    L.orc_denoise.argtypes = [i32, i32, vp, i32, i32, vp]
    L.orc_fill.argtypes = [i32, i32, vp, i32, i32, vp]
    L.orc_edt_brute.argtypes = [i32, i32, vp, vp]
    L.orc_edt_separable.argtypes = [i32, i32, vp, vp]
    L.orc_surface.argtypes = [i32, vp, f64, vp]
    L.orc_surface_mode.argtypes = [i32, vp, i32, f64, f64, vp]
    L.orc_iwe.argtypes = [i32, i32, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int64,
                          ctypes.c_int64, vp, vp]
    L.orc_fwl.argtypes = [i32, i32, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int64,
                          ctypes.c_int64, vp, vp]
    L.orc_alpha_from_dsat.argtypes = [f64, f64]
    L.orc_alpha_from_dsat.restype = f64
    L.orc_downsample.argtypes = [i32, i32, vp, vp]
    L.orc_gradients.argtypes = [i32, i32, vp, vp, vp]
    L.orc_patch_origins.argtypes = [i32, i32, i32, vp]
    L.orc_patch_origins.restype = i32
    L.orc_levels_used.argtypes = [i32, i32, i32, i32]
    L.orc_levels_used.restype = i32
    L.orc_patch_search.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, i32, i32,
                                   i32, i32, f64, vp, vp]
    L.orc_densify.argtypes = [i32, i32, vp, vp, i32, i32, vp, vp]
    L.orc_variational.argtypes = [i32, i32, vp, vp, vp, vp, vp, i32, i32, f64,
                                  f64, f64, f64]
    L.orc_var_linearise.argtypes = [i32, i32, vp, vp, vp, vp, vp, f64, f64, f64, vp]
    L.orc_var_sor.argtypes = [i32, i32, vp, vp, i32, f64, vp]
    L.orc_flow.argtypes = [i32, i32, vp, vp, i32, i32, i32, i32, f64, i32, i32, f64,
                           f64, f64, f64, vp]
    L.orc_flow.restype = i32


def set_mutation(k: int) -> None:
    """Plant deliberate mistake number k (0 removes it); tests only."""
    ctypes.c_int.in_dll(lib(), "orc_mutation").value = int(k)


# Default flow parameters (readings F1-F6; see ebof_oracle.c).
FLOW_DEFAULTS = dict(levels=3, patch=8, stride=4, gn_iters=12, gn_damping=0.1, var_outer=5,
                     var_sor=5, var_delta=5.0, var_gamma=10.0, var_alpha=20.0,
                     sor_omega=1.6)


def edge_image(width, height, x, y, t, t_begin, t_end):
    """§III-A: binary edge image of one window, plus event counts
    (given, in window, outside window, in window but outside the image)."""
    x = np.ascontiguousarray(x, np.uint16)
    y = np.ascontiguousarray(y, np.uint16)
    t = np.ascontiguousarray(t, np.int64)
    E = np.zeros((height, width), np.uint8)
    st = np.zeros(4, np.int64)
    lib().orc_edge_image(width, height, len(x), _p(x), _p(y), _p(t),
                         int(t_begin), int(t_end), _p(E), _p(st))
    return E, st


def denoise(E, connectivity=4, n_d=1):
    """Alg. 1."""
    E = np.ascontiguousarray(E, np.uint8)
    out = np.empty_like(E)
    lib().orc_denoise(E.shape[1], E.shape[0], _p(E), connectivity, n_d, _p(out))
    return out


def fill(Ed, connectivity=4, n_f=5):
    """Alg. 2 (on the denoised image)."""
    Ed = np.ascontiguousarray(Ed, np.uint8)
    out = np.empty_like(Ed)
    lib().orc_fill(Ed.shape[1], Ed.shape[0], _p(Ed), connectivity, n_f, _p(out))
    return out


def edt_brute(E):
    """§III-C distance definition, squared, by brute force."""
    E = np.ascontiguousarray(E, np.uint8)
    D = np.empty(E.shape, np.int32)
    lib().orc_edt_brute(E.shape[1], E.shape[0], _p(E), _p(D))
    return D


def edt(E):
    """§III-C exact squared EDT in separable form."""
    E = np.ascontiguousarray(E, np.uint8)
    D = np.empty(E.shape, np.int32)
    lib().orc_edt_separable(E.shape[1], E.shape[0], _p(E), _p(D))
    return D


def surface(D, alpha=1.08):
    """Eq. 1 on squared distances D."""
    D = np.ascontiguousarray(D, np.int32)
    S = np.empty(D.shape, np.float64)
    lib().orc_surface(D.size, _p(D), float(alpha), _p(S))
    return S


SURFACE_EXP, SURFACE_LINEAR, SURFACE_BOUNDED, SURFACE_LOG = 0, 1, 2, 3


def surface_mode(D, mode=SURFACE_EXP, alpha=1.08, d_sat=6.0):
    """Eq. 1 (mode 0) or one of the ablation surfaces of §IV-D: DS_L (1),
    DS_LB (2, bounded at d_sat), DS_Log (3)."""
    D = np.ascontiguousarray(D, np.int32)
    Y = np.empty(D.shape, np.float64)
    lib().orc_surface_mode(D.size, _p(D), int(mode), float(alpha), float(d_sat), _p(Y))
    return Y


def intensity_gain(mode=SURFACE_EXP, d_sat=6.0):
    """Scale from a surface to the flow block's intensity (reading S2): Eq. 1
    on the 8-bit scale, 255 d_exp (reading F0); each ablation surface scaled
    so that its value at d_sat, the distance where Eq. 1 reaches 254 of 255
    with alpha = d_sat / ln 255 (Eq. 3), maps to 255."""
    if mode == SURFACE_EXP:
        return 255.0
    if mode in (SURFACE_LINEAR, SURFACE_BOUNDED):
        return 255.0 / d_sat
    return 255.0 / np.log(d_sat + 1.0)


def _events(x, y, t, p):
    x = np.ascontiguousarray(x, np.uint16)
    y = np.ascontiguousarray(y, np.uint16)
    t = np.ascontiguousarray(t, np.int64)
    p = None if p is None else np.ascontiguousarray(p, np.int8)
    return x, y, t, p


def iwe(width, height, x, y, t, p, t_begin, t_end, U=None):
    """§IV-C image of events moved back along the flow U (None: not moved),
    readings W1-W3 of the C source."""
    x, y, t, p = _events(x, y, t, p)
    Ud = None if U is None else np.ascontiguousarray(U, np.float64)
    img = np.empty((height, width), np.float64)
    lib().orc_iwe(width, height, x.size, _p(x), _p(y), _p(t), None if p is None else _p(p),
                  int(t_begin), int(t_end), None if Ud is None else _p(Ud), _p(img))
    return img


def fwl(width, height, x, y, t, p, t_begin, t_end, U):
    """§IV-C Flow Warping Loss of flow U [2][H][W] on one window's events.
    Returns (FWL, var(I_comp), var(I_uncomp))."""
    x, y, t, p = _events(x, y, t, p)
    Ud = np.ascontiguousarray(U, np.float64)
    out = np.empty(3, np.float64)
    lib().orc_fwl(width, height, x.size, _p(x), _p(y), _p(t), None if p is None else _p(p),
                  int(t_begin), int(t_end), _p(Ud), _p(out))
    return float(out[0]), float(out[1]), float(out[2])


def alpha_from_dsat(d_sat, eps=1.0 / 255.0):
    """Eq. 2 (Eq. 3 at the default eps)."""
    return lib().orc_alpha_from_dsat(float(d_sat), float(eps))


def downsample(I):
    I = np.ascontiguousarray(I, np.float64)
    out = np.empty((I.shape[0] // 2, I.shape[1] // 2), np.float64)
    lib().orc_downsample(I.shape[1], I.shape[0], _p(I), _p(out))
    return out


def gradients(I):
    I = np.ascontiguousarray(I, np.float64)
    Ix = np.empty_like(I)
    Iy = np.empty_like(I)
    lib().orc_gradients(I.shape[1], I.shape[0], _p(I), _p(Ix), _p(Iy))
    return Ix, Iy


def patch_origins(n, ps, stride):
    buf = np.zeros(n + 2, np.int32)
    c = lib().orc_patch_origins(n, ps, stride, _p(buf))
    return buf[:c].copy()


def levels_used(width, height, levels, ps):
    return lib().orc_levels_used(width, height, levels, ps)


def patch_search(I0, I0x, I0y, I1, Uc, ps, stride, iters, kappa=0.1):
    """Readings F3-F4 at one level; returns patch flows [2][npy][npx] and flags."""
    H, W = I0.shape
    a = [np.ascontiguousarray(v, np.float64) for v in (I0, I0x, I0y, I1)]
    npx = len(patch_origins(W, ps, stride))
    npy = len(patch_origins(H, ps, stride))
    up = np.zeros((2, npy, npx), np.float64)
    fl = np.zeros((npy, npx), np.uint8)
    if Uc is None:
        ucp, Wc, Hc = None, 0, 0
    else:
        Uc = np.ascontiguousarray(Uc, np.float64)
        ucp, Wc, Hc = _p(Uc), Uc.shape[2], Uc.shape[1]
    lib().orc_patch_search(W, H, _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), ucp,
                           Wc, Hc, ps, stride, iters, float(kappa), _p(up), _p(fl))
    return up, fl


def densify(I0, I1, up, ps, stride):
    """Reading F5."""
    H, W = I0.shape
    I0 = np.ascontiguousarray(I0, np.float64)
    I1 = np.ascontiguousarray(I1, np.float64)
    up = np.ascontiguousarray(up, np.float64)
    U = np.zeros((2, H, W), np.float64)
    lib().orc_densify(W, H, _p(I0), _p(I1), ps, stride, _p(up), _p(U))
    return U


def variational(I0, I0x, I0y, I1, U, outer=5, sor=5, delta=5.0, gamma=10.0,
                alpha=20.0, omega=1.6):
    """Reading F6; returns the refined copy of U."""
    H, W = I0.shape
    a = [np.ascontiguousarray(v, np.float64) for v in (I0, I0x, I0y, I1)]
    U = np.array(U, np.float64, copy=True, order="C")
    lib().orc_variational(W, H, _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), _p(U),
                          outer, sor, delta, gamma, alpha, omega)
    return U


# Planes of the linearised variational system (orc_var_linearise's order).
VAR_PLANES = ("Ix", "Iy", "Ixx", "Ixy", "Iyy", "Iz", "Ixz", "Iyz", "ad", "ag", "as")


def var_linearise(I0, I0x, I0y, I1, U, delta=5.0, gamma=10.0, alpha=20.0):
    """Reading F6, first half of one outer iteration: the derivative and
    residual planes of the image warped by U and the frozen robust weights.
    Returns a dict of the VAR_PLANES, each [H][W]."""
    H, W = I0.shape
    a = [np.ascontiguousarray(v, np.float64) for v in (I0, I0x, I0y, I1)]
    U = np.ascontiguousarray(U, np.float64)
    Q = np.zeros((len(VAR_PLANES), H, W), np.float64)
    lib().orc_var_linearise(W, H, _p(a[0]), _p(a[1]), _p(a[2]), _p(a[3]), _p(U),
                            delta, gamma, alpha, _p(Q))
    return {k: Q[i] for i, k in enumerate(VAR_PLANES)}


def var_sor(planes, U, dU, sweeps, omega=1.6):
    """Reading F6, second half: `sweeps` red-black SOR sweeps on the
    linearised system given by ``planes`` (a dict of VAR_PLANES) at flow U,
    starting from dU; returns the new dU [2][H][W]."""
    Q = np.ascontiguousarray(np.stack([planes[k] for k in VAR_PLANES]), np.float64)
    H, W = Q.shape[1:]
    U = np.ascontiguousarray(U, np.float64)
    dU = np.array(dU, np.float64, copy=True, order="C")
    lib().orc_var_sor(W, H, _p(Q), _p(U), int(sweeps), float(omega), _p(dU))
    return dU


def flow(I0, I1, levels=3, patch=8, stride=4, gn_iters=12, gn_damping=0.1, var_outer=5,
         var_sor=5, var_delta=5.0, var_gamma=10.0, var_alpha=20.0,
         sor_omega=1.6):
    """§III-D flow block on two level-0 intensity images (255 * d_exp).
    Returns the planar flow [2][H][W] (pixels per window, previous to
    current)."""
    I0 = np.ascontiguousarray(I0, np.float64)
    I1 = np.ascontiguousarray(I1, np.float64)
    H, W = I0.shape
    U = np.zeros((2, H, W), np.float64)
    lib().orc_flow(W, H, _p(I0), _p(I1), levels, patch, stride, gn_iters,
                   float(gn_damping), var_outer, var_sor, var_delta, var_gamma, var_alpha,
                   sor_omega, _p(U))
    return U


def surface_from_events(width, height, x, y, t, t_begin, t_end,
                        connectivity=8, n_d=1, n_f=9, alpha=1.08, surface=SURFACE_EXP,
                        d_sat=6.0):
    """§III-A to §III-C for one window: edge image, Alg. 1, Alg. 2, exact
    EDT and Eq. 1 (or an ablation surface of §IV-D).  Returns dict with E,
    Edf, D, S (the surface) and the event counts."""
    E, st = edge_image(width, height, x, y, t, t_begin, t_end)
    Ed = denoise(E, connectivity, n_d)
    Edf = fill(Ed, connectivity, n_f)
    D = edt(Edf)
    S = surface_mode(D, surface, alpha, d_sat)
    return dict(E=E, Edf=Edf, D=D, S=S, stats=st)


def process_pair(width, height, win0, win1, connectivity=8, n_d=1, n_f=9,
                 alpha=1.08, surface=SURFACE_EXP, d_sat=6.0, **flow_kw):
    """Whole path for two consecutive windows ``(x, y, t, t_begin, t_end)``:
    surfaces of both, then the flow from the first to the second on the
    intensity scale of readings F0 and S2."""
    s0 = surface_from_events(width, height, *win0, connectivity=connectivity,
                             n_d=n_d, n_f=n_f, alpha=alpha, surface=surface, d_sat=d_sat)
    s1 = surface_from_events(width, height, *win1, connectivity=connectivity,
                             n_d=n_d, n_f=n_f, alpha=alpha, surface=surface, d_sat=d_sat)
    kw = dict(FLOW_DEFAULTS)
    kw.update(flow_kw)
    g = intensity_gain(surface, d_sat)
    U = flow(g * s0["S"], g * s1["S"], **kw)
    return s0, s1, U
