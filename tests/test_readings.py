"""Identities the CUDA path relies on, checked in exact arithmetic (CPU).

The patch search (inverse search of Kroeger et al., the flow block of
§III-D) warps a patch by one displacement (u, v), so every sample of the
patch has the same fractional offsets and the warped patch is one
(ps+1) x (ps+1) window of texels with fixed weights.  Where the window
leaves the level the kernel clamps the window's row and column indices;
the oracle's reading is a bilinear sample with the sample *position*
clamped to the level.  The two are the same function: outside the level
both taps of a lerp are the same edge texel.  Checked here with rational
arithmetic on random images, displacements inside, across and far outside
the level, and positions exactly on the last row and column.
"""
import math
import random
from fractions import Fraction as Q


def position_clamped(I, w, h, x, y):
    """Bilinear sample with the position clamped to [0, w-1] x [0, h-1]."""
    x = min(max(x, Q(0)), Q(w - 1))
    y = min(max(y, Q(0)), Q(h - 1))
    x0, y0 = math.floor(x), math.floor(y)
    fx, fy = x - x0, y - y0
    x1, y1 = min(x0 + 1, w - 1), min(y0 + 1, h - 1)
    top = (1 - fx) * I[y0][x0] + fx * I[y0][x1]
    bot = (1 - fx) * I[y1][x0] + fx * I[y1][x1]
    return (1 - fy) * top + fy * bot


def window_clamped(I, w, h, px, py, i, j, u, v):
    """Sample (i, j) of the patch at origin (px, py) displaced by (u, v):
    the fixed-weight window from (px + floor(u), py + floor(v)) with its
    column and row indices clamped, horizontal lerps first (the kernel's
    order), the displacement first clamped to +-(w + h) as the kernel does."""
    lim = Q(w + h)
    u = min(max(u, -lim), lim)
    v = min(max(v, -lim), lim)
    sx0, sy0 = px + math.floor(u), py + math.floor(v)
    ax, ay = u - math.floor(u), v - math.floor(v)
    cx = lambda c: min(max(c, 0), w - 1)
    ry = lambda r: min(max(r, 0), h - 1)

    def row(r):
        s0, s1 = I[ry(r)][cx(sx0 + i)], I[ry(r)][cx(sx0 + i + 1)]
        return s0 + ax * (s1 - s0)

    h0, h1 = row(sy0 + j), row(sy0 + j + 1)
    return h0 + ay * (h1 - h0)


def _rand_q(rng, lo, hi, den=64):
    return Q(rng.randrange(lo * den, hi * den), den)


def test_window_clamp_equals_position_clamp():
    rng = random.Random(7)
    for trial in range(40):
        w, h = rng.randrange(13, 40), rng.randrange(13, 30)
        ps = 12
        I = [[rng.randrange(0, 256) for _ in range(w)] for _ in range(h)]
        px, py = rng.randrange(0, w - ps + 1), rng.randrange(0, h - ps + 1)
        big = 3 * (w + h)
        if trial % 4 == 0:      # far outside, beyond the kernel's clamp of (u, v)
            u, v = _rand_q(rng, -big, big), _rand_q(rng, -big, big)
        elif trial % 4 == 1:    # onto the last column and row exactly
            u, v = Q(w - ps - px), Q(h - ps - py)
        else:                   # around the level's borders
            u, v = _rand_q(rng, -px - 3, w - px + 3), _rand_q(rng, -py - 3, h - py + 3)
        for j in range(ps):
            for i in range(ps):
                a = position_clamped(I, w, h, px + i + u, py + j + v)
                b = window_clamped(I, w, h, px, py, i, j, u, v)
                assert a == b, (trial, i, j, u, v)


def test_window_inside_the_level_needs_no_clamp():
    """Where the whole window lies inside the level the clamps do nothing, so
    a warp may take either form without changing a value."""
    rng = random.Random(8)
    w, h, ps = 50, 40, 12
    I = [[rng.randrange(0, 256) for _ in range(w)] for _ in range(h)]
    for _ in range(30):
        px, py = rng.randrange(4, w - ps - 4), rng.randrange(4, h - ps - 4)
        u, v = _rand_q(rng, -3, 3), _rand_q(rng, -3, 3)
        sx0, sy0 = px + math.floor(u), py + math.floor(v)
        assert 0 <= sx0 and sx0 + ps <= w - 1 and 0 <= sy0 and sy0 + ps <= h - 1
        ax, ay = u - math.floor(u), v - math.floor(v)
        for j in range(ps):
            for i in range(ps):
                r0, r1 = I[sy0 + j], I[sy0 + j + 1]
                h0 = r0[sx0 + i] + ax * (r0[sx0 + i + 1] - r0[sx0 + i])
                h1 = r1[sx0 + i] + ax * (r1[sx0 + i + 1] - r1[sx0 + i])
                assert h0 + ay * (h1 - h0) == window_clamped(I, w, h, px, py, i, j, u, v)
