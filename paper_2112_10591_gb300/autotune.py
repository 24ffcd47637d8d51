"""Per-resolution choice of the method's patch grid and pyramid depth, and of
the variational kernels' layouts, for multi-stream groups.

Two passes over calibration windows (two consecutive windows per stream);
every measurement goes through the C ABI (ebof_group_*, ebof_fwl) and the
tuner itself only orchestrates and compares.

1. Method candidates (patch size, stride, levels) change the flow.  A
   candidate is accepted when its flow is not worse than the flow of the
   library's default parameters by the paper's own measure without ground
   truth, the Flow Warping Loss of §IV-C: it must keep at least ``keep`` of
   the default's FWL gain over the zero flow (FWL - 1) on the calibration
   windows (or, where the default does not beat the zero flow, reach the
   default's FWL).  The fastest accepted candidate wins.  Whether the GPU
   path of a candidate configuration matches the FP64 oracle is a property
   of the library, covered by its tests; the tuner runs in the product path,
   which never touches the oracle.
2. Layout candidates (the coefficient kernel's form and the height of its
   column-walk strips, the SOR kernels' forms: the persistent copy-ahead
   kernel, regions of one-row strips; the cluster-resident refinement of
   small levels) never change the flow.  The tuner checks that each one gives the flow of
   the default layout bit for bit and keeps the fastest, one knob at a time
   from the default, then the combination of the winners.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import binding as eb

# Layout knobs of ebof_params (every value gives the same flow bit for bit)
# and the values tried besides the default.
NEVER = 1 << 20
LAYOUT_CANDIDATES = {
    "coeff_cw_min_width": (640, NEVER),
    "sor_tma_min_per_sm": (2, 4, NEVER),
    "sor_row_waves": (0, 2),
    "var_cluster_max": (8, 16),
    "coeff_cw_rows": (4, 16),
}


def _copy_params(p):
    q = eb.ebof_params()
    ctypes.memmove(ctypes.byref(q), ctypes.byref(p), ctypes.sizeof(q))
    return q


def _run(prm, calib, width, height, device, repeats, want_fwl):
    """Flows of the calibration pair, their mean FWL (optional) and the
    steady-state group step time (graph replays, the two windows alternating)."""
    import torch
    n = len(calib)
    rc, g = eb.ebof_group_create(prm, n, device)
    if rc < 0:
        return None, eb.ebof_status_string(rc)
    try:
        flow = torch.empty((n, 2, height, width), dtype=torch.float32, device="cuda")
        w0 = [c[0] for c in calib]
        w1 = [c[1] for c in calib]
        eb.check(eb.ebof_group_process(g, w0))
        eb.check(eb.ebof_group_process(g, w1, flow))
        torch.cuda.synchronize()
        fwl = None
        if want_fwl:
            scr = torch.empty(eb.ebof_fwl_scratch_bytes(width, height), dtype=torch.uint8,
                              device="cuda")
            out = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
            for k, (x, y, t, tb, te) in enumerate(w1):
                rc, _ = eb.ebof_fwl(x, y, t, None, tb, te, flow[k], width, height, scr, out[k])
                eb.check(rc, "ebof_fwl")
            torch.cuda.synchronize()
            fwl = float(out[:, 0].mean().item())
        for r in range(2):  # warm the graphs of both parities
            eb.check(eb.ebof_group_process(g, w0 if r % 2 == 0 else w1))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for r in range(repeats):
            eb.check(eb.ebof_group_process(g, w0 if r % 2 == 0 else w1))
        e1.record()
        torch.cuda.synchronize()
        return (flow.cpu().numpy(), fwl, e0.elapsed_time(e1) / repeats), None
    finally:
        g.close()


def _accept(fwl, fwl_default, keep):
    if fwl is None or fwl_default is None:
        return False
    if fwl_default > 1.0:
        return fwl - 1.0 >= keep * (fwl_default - 1.0)
    return fwl >= fwl_default


def method_candidates(width, height, candidates=None):
    """(patch, stride, levels) triples the tuner tries for a resolution, the
    library's defaults first: a wider stride, one level fewer, and 8x8 and
    12x12 patches at strides 4 and 6."""
    base = eb.ebof_default_params(width, height)
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
    return cands


def tune(width, height, calib, storage=eb.EBOF_STORAGE_FP32, candidates=None, keep=0.9,
         repeats=6, device=0, layouts=True):
    """calib: list over streams of two consecutive windows, each a tuple
    (x, y, t, t_begin, t_end) of CUDA tensors and ints.  Returns (params,
    table): table["method"] lists every method candidate's step time, FWL
    and acceptance, table["layout"] every layout candidate's step time."""
    base = eb.ebof_default_params(width, height)
    base.storage = storage
    cands = method_candidates(width, height, candidates)
    method = []
    fwl_default = None
    for i, (ps, st, lv) in enumerate(cands):
        prm = _copy_params(base)
        prm.patch, prm.stride, prm.levels = ps, st, lv
        res, err = _run(prm, calib, width, height, device, repeats, True)
        row = {"patch": ps, "stride": st, "levels": lv}
        if res is None:
            row["status"] = err
            method.append(row)
            continue
        _, fwl, ms = res
        if i == 0:
            fwl_default = fwl
        row.update({"ms_per_step": ms, "fwl": fwl,
                    "accepted": i == 0 or _accept(fwl, fwl_default, keep)})
        method.append(row)
    ok = [r for r in method if r.get("accepted")]
    best = min(ok, key=lambda r: r["ms_per_step"]) if ok else None
    out = _copy_params(base)
    if best is not None:
        out.patch, out.stride, out.levels = best["patch"], best["stride"], best["levels"]
    table = {"method": method, "method_rule": "fastest candidate keeping >= %.0f%% of the "
             "default's FWL gain over zero flow (§IV-C)" % (100 * keep), "layout": []}
    if not layouts:
        return out, table
    # layouts: the default first (its flow is the reference), one knob at a time
    ref, err = _run(out, calib, width, height, device, repeats, False)
    if ref is None:
        return out, table
    ref_flow, _, ref_ms = ref
    table["layout"].append({"knob": "default", "ms_per_step": ref_ms, "identical": True})
    chosen = {}
    for knob, values in LAYOUT_CANDIDATES.items():
        best_v, best_ms = getattr(out, knob), ref_ms
        for v in values:
            if v == getattr(out, knob):
                continue  # the default, timed above
            prm = _copy_params(out)
            setattr(prm, knob, v)
            res, err = _run(prm, calib, width, height, device, repeats, False)
            if res is None:
                table["layout"].append({"knob": knob, "value": v, "status": err})
                continue
            f, _, ms = res
            same = bool(np.array_equal(f, ref_flow))
            table["layout"].append({"knob": knob, "value": v, "ms_per_step": ms,
                                    "identical": same})
            if same and ms < best_ms:
                best_v, best_ms = v, ms
        chosen[knob] = best_v
    final = _copy_params(out)
    for knob, v in chosen.items():
        setattr(final, knob, v)
    if any(getattr(final, k) != getattr(out, k) for k in chosen):
        res, err = _run(final, calib, width, height, device, repeats, False)
        if res is not None and np.array_equal(res[0], ref_flow) and res[2] < ref_ms:
            table["layout"].append({"knob": "combined", "values": dict(chosen),
                                    "ms_per_step": res[2], "identical": True})
            out = final
        else:
            table["layout"].append({"knob": "combined", "values": dict(chosen),
                                    "ms_per_step": None if res is None else res[2],
                                    "identical": res is not None and
                                    bool(np.array_equal(res[0], ref_flow)),
                                    "kept_default": True})
    table["layout_chosen"] = {k: getattr(out, k) for k in LAYOUT_CANDIDATES}
    return out, table
