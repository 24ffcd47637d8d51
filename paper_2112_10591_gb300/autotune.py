"""Per-resolution choice of the patch grid and pyramid depth for
multi-stream groups.

For one sensor resolution the tuner times a group step for a few candidate
(patch size, stride, levels) triples on calibration windows and keeps the
fastest candidate whose flow stays within ``tol_px`` mean endpoint error of
the flow computed with the library's default parameters on the same windows.
Every measurement goes through the C ABI (ebof_group_*); the tuner itself
only orchestrates and compares.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as eb


def _copy_params(p):
    q = eb.ebof_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
    return q


def tune(width, height, calib, storage=eb.EBOF_STORAGE_FP32, candidates=None, tol_px=0.25,
         repeats=4, device=0):
    """calib: list over streams of two consecutive windows, each a tuple
    (x, y, t, t_begin, t_end) of CUDA tensors and ints.  Returns (params,
    table) where table lists every candidate's step time and EPE."""
    import torch
    base = eb.ebof_default_params(width, height)
    base.storage = storage
    if candidates is None:
        L = base.levels
        candidates = [(base.patch, base.stride, L), (base.patch, base.stride + 2, L),
                      (base.patch, base.stride, L - 1), (8, 4, L), (8, 6, L), (12, 4, L),
                      (12, 6, L)]
    seen, cands = set(), []
    for c in candidates:
        c = tuple(c) if len(c) == 3 else (c[0], c[1], base.levels)
        if c not in seen and min(width, height) >= c[0] and c[2] >= 1:
            seen.add(c)
            cands.append(c)
    n = len(calib)
    ref_flow = None
    table = []
    for ps, st, lv in cands:
        prm = _copy_params(base)
        prm.patch, prm.stride, prm.levels = ps, st, lv
        rc, g = eb.ebof_group_create(prm, n, device)
        if rc < 0:
            table.append({"patch": ps, "stride": st, "levels": lv,
                          "status": eb.ebof_status_string(rc)})
            continue
        flow = torch.empty((n, 2, height, width), dtype=torch.float32, device="cuda")
        w0 = [c[0] for c in calib]
        w1 = [c[1] for c in calib]
        eb.check(eb.ebof_group_process(g, w0))
        eb.check(eb.ebof_group_process(g, w1, flow))
        torch.cuda.synchronize()
        f = flow.cpu().numpy()
        if ref_flow is None:
            ref_flow = f
        epe = float(np.hypot(f[:, 0] - ref_flow[:, 0], f[:, 1] - ref_flow[:, 1]).mean())
        # steady-state step time (graph replays), alternating the two windows
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(repeats):
            eb.check(eb.ebof_group_process(g, w0 if r % 2 == 0 else w1))
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / repeats
        table.append({"patch": ps, "stride": st, "levels": lv, "ms_per_step": ms,
                      "epe_vs_default_px": epe})
        g.close()
    ok = [r for r in table if "ms_per_step" in r and r["epe_vs_default_px"] <= tol_px]
    best = min(ok, key=lambda r: r["ms_per_step"]) if ok else table[0]
    out = _copy_params(base)
    out.patch, out.stride, out.levels = best["patch"], best["stride"], best["levels"]
    return out, table
