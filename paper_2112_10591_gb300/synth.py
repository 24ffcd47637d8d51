"""Seeded synthetic event streams shaped like the paper's driving sequences.

The paper evaluates on recorded event streams (MVSEC at 346x260, Prophesee
1 Mp recordings at 1280x720; §IV-B, Table I).  None of those recordings is
available here, so every input of the tests and the benchmark comes from
this module instead: events (x, y, t, p) drawn from rigidly moving line
segments plus uniform noise, with the sizes, counts and motions of the two
resolutions the paper targets.

This module holds none of the method's arithmetic: it only draws events.
It is the one module shared by the CUDA path's tests and benchmark and by
the CPU oracle's tests, so both sides always see the same inputs.

Recipe (one line per knob):
  * timestamps are int64 microseconds, uniform over each 10 ms window;
  * an edge event picks a segment with probability proportional to its
    length and a point s ~ U[0, 1) along it; its position is that point
    carried by its object's motion up to the event's normalised time
    tau = k + (t - t_k) / dt, rounded with floor(v + 0.5); events that land
    off the image are drawn again;
  * noise events are uniform over the image and the window;
  * polarity: every edge has a contrast sign (alternating over the scene's
    segments) that 90 % of its events carry; noise events are +1 or -1 with
    equal odds (the method ignores polarity; the FWL metric uses it);
  * events of one window are sorted by timestamp, as a sensor emits them.

With ``keep_truth`` a stream also keeps, per event, the segment and the
point on it that produced the event, from which ``true_flow`` gives the
ground-truth displacement of every edge pixel between two windows.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

WINDOW_US = 10_000


@dataclasses.dataclass
class EventStream:
    """Events of consecutive fixed-length windows, concatenated.

    Window k holds events ``offsets[k]:offsets[k+1]`` and covers the
    half-open time range ``[t_begin[k], t_begin[k] + dt)``.
    """

    width: int
    height: int
    x: np.ndarray          # uint16 [N]
    y: np.ndarray          # uint16 [N]
    t: np.ndarray          # int64  [N], microseconds
    p: np.ndarray          # int8   [N], +1 / -1
    offsets: np.ndarray    # int64  [n_windows + 1]
    t_begin: np.ndarray    # int64  [n_windows]
    dt: int
    seg: np.ndarray = None     # int32 [N] producing segment, -1 for noise (keep_truth)
    frac: np.ndarray = None    # float64 [N] point on the segment (keep_truth)
    scene: "_Scene" = None     # the moving scene (keep_truth)

    @property
    def n_windows(self) -> int:
        return len(self.t_begin)

    def window(self, k: int):
        a, b = int(self.offsets[k]), int(self.offsets[k + 1])
        tb = int(self.t_begin[k])
        return (self.x[a:b], self.y[a:b], self.t[a:b], self.p[a:b],
                tb, tb + self.dt)

    def true_flow(self, k: int):
        """Ground truth of the flow from window k - 1 to window k (k >= 1):
        at every pixel where window k - 1 has an edge event, the mean over
        those events of how far the scene point that produced the event
        moves in one window (its position at the same phase of window k
        minus its position at the event).  Returns (flow [2][H][W] float64,
        mask [H][W] bool); flow is 0 where mask is False.  Needs a stream
        made with keep_truth."""
        if self.seg is None or k < 1:
            raise ValueError("true_flow needs keep_truth and k >= 1")
        a, b = int(self.offsets[k - 1]), int(self.offsets[k])
        seg = self.seg[a:b]
        m = seg >= 0
        seg = seg[m].astype(np.int64)
        frac = self.frac[a:b][m]
        f = (self.t[a:b][m] - self.t_begin[k - 1]) / self.dt
        x0, y0 = _place(self.scene, seg, frac, k - 1, f)
        x1, y1 = _place(self.scene, seg, frac, k, f)
        W, H = self.width, self.height
        pix = self.y[a:b][m].astype(np.int64) * W + self.x[a:b][m].astype(np.int64)
        cnt = np.bincount(pix, minlength=W * H)
        u = np.bincount(pix, weights=x1 - x0, minlength=W * H)
        v = np.bincount(pix, weights=y1 - y0, minlength=W * H)
        mask = cnt > 0
        flow = np.zeros((2, W * H))
        flow[0, mask] = u[mask] / cnt[mask]
        flow[1, mask] = v[mask] / cnt[mask]
        return flow.reshape(2, H, W), mask.reshape(H, W)


@dataclasses.dataclass
class _Scene:
    p0: np.ndarray         # float64 [S, 2]  segment start (x, y) at tau = 0
    p1: np.ndarray         # float64 [S, 2]  segment end
    obj: np.ndarray        # int64 [S]       owning object
    centre: np.ndarray     # float64 [O, 2]  rotation centre per object
    theta: np.ndarray      # float64 [K+1, O] rotation at window boundaries
    shift: np.ndarray      # float64 [K+1, O, 2] translation at boundaries


def _place(scene: _Scene, seg: np.ndarray, s: np.ndarray, k: int,
           f: np.ndarray):
    """Position of point ``s`` of segment ``seg`` at normalised time k + f."""
    k = min(max(k, 0), scene.theta.shape[0] - 2)
    o = scene.obj[seg]
    th0, th1 = scene.theta[k], scene.theta[k + 1]
    sh0, sh1 = scene.shift[k], scene.shift[k + 1]
    th = th0[o] + f * (th1 - th0)[o]
    shx = sh0[:, 0][o] + f * (sh1[:, 0] - sh0[:, 0])[o]
    shy = sh0[:, 1][o] + f * (sh1[:, 1] - sh0[:, 1])[o]
    d = scene.p1 - scene.p0
    relx = (scene.p0[:, 0] - scene.centre[scene.obj, 0])[seg] + s * d[:, 0][seg]
    rely = (scene.p0[:, 1] - scene.centre[scene.obj, 1])[seg] + s * d[:, 1][seg]
    c, sn = np.cos(th), np.sin(th)
    cx, cy = scene.centre[:, 0][o], scene.centre[:, 1][o]
    return (cx + (c * relx - sn * rely) + shx,
            cy + (sn * relx + c * rely) + shy)


def _draw_window(rng, scene: _Scene, W: int, H: int, k: int, n_events: int,
                 noise_frac: float, t0: int, dt: int):
    n_noise = int(round(noise_frac * n_events))
    n_edge = n_events - n_noise
    length = np.hypot(*(scene.p1 - scene.p0).T)
    cdf = np.cumsum(length / length.sum())
    cdf[-1] = 1.0
    xs, ys, ts, ss, fs = [], [], [], [], []
    need = n_edge
    while need > 0:
        m = int(need * 1.3) + 64
        seg = np.minimum(np.searchsorted(cdf, rng.random(m), side="right"),
                         len(cdf) - 1)
        s = rng.random(m)
        t = rng.integers(t0, t0 + dt, size=m, dtype=np.int64)
        px, py = _place(scene, seg, s, k, (t - t0) / dt)
        ix = np.floor(px + 0.5)
        iy = np.floor(py + 0.5)
        ok = (ix >= 0) & (ix < W) & (iy >= 0) & (iy < H)
        ix, iy, t = ix[ok][:need], iy[ok][:need], t[ok][:need]
        xs.append(ix.astype(np.uint16))
        ys.append(iy.astype(np.uint16))
        ts.append(t)
        ss.append(seg[ok][:need])
        fs.append(s[ok][:need])
        need -= len(t)
    xs.append(rng.integers(0, W, size=n_noise).astype(np.uint16))
    ys.append(rng.integers(0, H, size=n_noise).astype(np.uint16))
    ts.append(rng.integers(t0, t0 + dt, size=n_noise, dtype=np.int64))
    ss.append(np.full(n_noise, -1))
    fs.append(np.zeros(n_noise))
    x = np.concatenate(xs)
    y = np.concatenate(ys)
    t = np.concatenate(ts)
    seg = np.concatenate(ss)[:n_events]
    frac = np.concatenate(fs)[:n_events]
    order = np.argsort((t - t0).astype(np.uint32), kind="stable")
    # polarity: every edge has a contrast sign (alternating over the scene's
    # segments) that 90 % of its events carry; noise events are +1 or -1
    # with equal odds
    u = rng.random(n_events)[np.argsort(order, kind="stable")]
    sign = np.where(seg % 2 == 0, 1, -1)
    p = np.where(seg < 0, np.where(u < 0.5, 1, -1), np.where(u < 0.9, sign, -sign))
    return (x[order], y[order], t[order], p[order].astype(np.int8), seg[order].astype(np.int32),
            frac[order])


def _assemble(rng, scene, W, H, counts, noise_frac, dt, t_start=0, keep_truth=False):
    xs, ys, ts, ps, ss, fs = [], [], [], [], [], []
    offsets = [0]
    t_begin = []
    for k, n in enumerate(counts):
        t0 = t_start + k * dt
        x, y, t, p, sg, fr = _draw_window(rng, scene, W, H, k, int(n), noise_frac, t0, dt)
        xs.append(x); ys.append(y); ts.append(t); ps.append(p)
        if keep_truth:
            ss.append(sg); fs.append(fr)
        offsets.append(offsets[-1] + len(x))
        t_begin.append(t0)
    ev = EventStream(W, H, np.concatenate(xs), np.concatenate(ys),
                     np.concatenate(ts), np.concatenate(ps),
                     np.asarray(offsets, np.int64),
                     np.asarray(t_begin, np.int64), dt)
    if keep_truth:
        ev.seg = np.concatenate(ss)
        ev.frac = np.concatenate(fs)
        ev.scene = scene
    return ev


def translating_segments(width=346, height=260, n_windows=2, n_segments=40,
                         length=(10.0, 60.0), velocity=(3.0, -1.5),
                         events_per_window=20_000, noise_frac=0.05, seed=0,
                         dt=WINDOW_US, keep_truth=False) -> EventStream:
    """Low-resolution stream: line segments translating at one velocity.

    Default arguments give the 346x260 single-window workload: two windows of
    20 000 events, 40 segments of length U[10, 60] px at random angles with
    start points uniform in the image, all moving at (3.0, -1.5) px per
    window, plus 5 % uniform noise events; seed 0.
    """
    rng = np.random.default_rng(seed)
    start = rng.random((n_segments, 2)) * [width, height]
    ln = rng.uniform(length[0], length[1], n_segments)
    ang = rng.uniform(0.0, 2.0 * math.pi, n_segments)
    end = start + np.stack([ln * np.cos(ang), ln * np.sin(ang)], 1)
    K = n_windows
    theta = np.zeros((K + 1, 1))
    shift = np.arange(K + 1, dtype=np.float64)[:, None, None] * np.asarray(velocity)[None, None, :]
    scene = _Scene(start, end, np.zeros(n_segments, np.int64),
                   np.zeros((1, 2)), theta, shift)
    return _assemble(rng, scene, width, height, [events_per_window] * K,
                     noise_frac, dt, keep_truth=keep_truth)


def rigid_objects(width=1280, height=720, n_windows=201, n_objects=12,
                  n_edges=300, radius=(40.0, 200.0), extra_length=(10.0, 120.0),
                  max_rot_deg=2.0, max_shift=20.0, events=(150_000, 400_000),
                  noise_frac=0.03, seed=1, dt=WINDOW_US,
                  lognormal_counts=False, keep_truth=False,
                  constant_velocity=False) -> EventStream:
    """High-resolution stream: rigid objects with their own affine motion.

    Default arguments give the 1280x720 stream workload: 201 windows (200
    flow frames) of U{150k..400k} events; 12 objects, each a random polygon
    (4 to 8 vertices, radius 40 to 200 px) plus extra segments of length
    U[10, 120] px, 300 edges in all; every window each object turns by
    U[-2, 2] degrees about its centre and moves by a translation with
    components U[-20, 20] px (norm capped at 20 px), reflected when the
    centre would leave the image; the background is static and produces
    no events; 3 % uniform noise; seed 1.  With ``lognormal_counts`` the
    per-window counts are lognormal, clipped to ``events``.  With
    ``constant_velocity`` each object's turn and translation are drawn once
    and kept for every window (a reflected component stays reflected), so
    that consecutive windows smear the edges along the same displacement.
    """
    rng = np.random.default_rng(seed)
    centres = rng.random((n_objects, 2)) * [width, height]
    p0, p1, obj = [], [], []
    for o in range(n_objects):
        nv = int(rng.integers(4, 9))
        r = rng.uniform(radius[0], radius[1])
        a = np.sort(rng.uniform(0.0, 2.0 * math.pi, nv))
        rr = r * rng.uniform(0.6, 1.0, nv)
        v = centres[o] + np.stack([rr * np.cos(a), rr * np.sin(a)], 1)
        for i in range(nv):
            p0.append(v[i]); p1.append(v[(i + 1) % nv]); obj.append(o)
    while len(p0) < n_edges:
        o = int(rng.integers(0, n_objects))
        r = rng.uniform(radius[0], radius[1])
        rho = r * math.sqrt(rng.random())
        phi = rng.uniform(0.0, 2.0 * math.pi)
        s = centres[o] + rho * np.array([math.cos(phi), math.sin(phi)])
        ln = rng.uniform(extra_length[0], extra_length[1])
        ang = rng.uniform(0.0, 2.0 * math.pi)
        p0.append(s); p1.append(s + ln * np.array([math.cos(ang), math.sin(ang)])); obj.append(o)
    p0 = np.asarray(p0[:n_edges]); p1 = np.asarray(p1[:n_edges])
    obj = np.asarray(obj[:n_edges], np.int64)

    K = n_windows
    theta = np.zeros((K + 1, n_objects))
    shift = np.zeros((K + 1, n_objects, 2))
    dth = d = None
    for k in range(K):
        if not constant_velocity or k == 0:
            dth = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg, n_objects))
            d = rng.uniform(-max_shift, max_shift, (n_objects, 2))
            nrm = np.linalg.norm(d, axis=1, keepdims=True)
            d = np.where(nrm > max_shift, d * (max_shift / np.maximum(nrm, 1e-12)), d)
        pos = centres + shift[k] + d
        out_x = (pos[:, 0] < 0) | (pos[:, 0] >= width)
        out_y = (pos[:, 1] < 0) | (pos[:, 1] >= height)
        d[out_x, 0] *= -1.0
        d[out_y, 1] *= -1.0
        theta[k + 1] = theta[k] + dth
        shift[k + 1] = shift[k] + d
    scene = _Scene(p0, p1, obj, centres, theta, shift)
    if lognormal_counts:
        lo, hi = events
        mu = 0.5 * (math.log(lo) + math.log(hi))
        sig = (math.log(hi) - math.log(lo)) / 4.0
        counts = np.clip(np.round(rng.lognormal(mu, sig, K)), lo, hi).astype(np.int64)
    else:
        counts = rng.integers(events[0], events[1] + 1, size=K)
    return _assemble(rng, scene, width, height, counts, noise_frac, dt, keep_truth=keep_truth)


def workload_346x260(seed=0) -> EventStream:
    """346x260, two windows of 20 000 events: one flow frame."""
    return translating_segments(seed=seed)


def workload_1280x720(seed=1, n_windows=201, keep_truth=False) -> EventStream:
    """1280x720, 201 windows of 150k-400k events: 200 flow frames."""
    return rigid_objects(seed=seed, n_windows=n_windows, keep_truth=keep_truth)


def random_edge_events(rng, width, height, n, t_begin=0, dt=WINDOW_US,
                       out_of_range=0.0):
    """Uniform random events for edge-case tests.

    A fraction ``out_of_range`` of the events get coordinates beyond the
    image or timestamps outside the window, to exercise dropping.
    """
    x = rng.integers(0, width, size=n).astype(np.int64)
    y = rng.integers(0, height, size=n).astype(np.int64)
    t = rng.integers(t_begin, t_begin + dt, size=n, dtype=np.int64)
    if out_of_range > 0 and n > 0:
        m = rng.random(n) < out_of_range
        kind = rng.integers(0, 4, size=n)
        x = np.where(m & (kind == 0), width + rng.integers(0, 50, size=n), x)
        y = np.where(m & (kind == 1), height + rng.integers(0, 50, size=n), y)
        t = np.where(m & (kind == 2), t_begin - 1 - rng.integers(0, 1000, size=n), t)
        t = np.where(m & (kind == 3), t_begin + dt + rng.integers(0, 1000, size=n), t)
    x = np.minimum(x, 65535).astype(np.uint16)
    y = np.minimum(y, 65535).astype(np.uint16)
    p = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    return x, y, t, p
