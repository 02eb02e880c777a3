"""Independent brute-force re-derivations used to pin the oracle (test helper; imports neither the oracle nor
the CUDA library).

* characteristic offsets re-derived from the written layout rules;
* segment lengths by clipping the line against every cell box (Liang-Barsky), not by sorting crossings;
* band-cell areas by polygon clipping (shoelace), the exact area the paper's A = l w approximates;
* the transport ODE dI/ds + kappa~ I = Q integrated by classical RK4 with the segment average by Simpson's
  rule, instead of the exponential solution and alpha of Eq. (12)-(13).
"""
from __future__ import annotations

import math

import numpy as np


def unit(c, s):
    n = math.hypot(c, s)
    return c / n, s / n


def corners(x0, y0, lx, ly):
    return [(x0, y0), (x0 + lx, y0), (x0, y0 + ly), (x0 + lx, y0 + ly)]


def uniform_offsets(lx, ly, c, s, spacing, x0=0.0, y0=0.0):
    t = [-s * x + c * y for x, y in corners(x0, y0, lx, ly)]
    tmin, tmax = min(t), max(t)
    n = max(1, math.ceil((tmax - tmin) / spacing - 1e-9))
    w = (tmax - tmin) / n
    return [tmin + (k + 0.5) * w for k in range(n)], [w] * n


def paper_offsets(nx, ny, lx, ly, c, s, spacing, x0=0.0, y0=0.0):
    hx, hy = lx / nx, ly / ny
    v = sorted(-s * (x0 + a * hx) + c * (y0 + b * hy) for a in range(nx + 1) for b in range(ny + 1))
    merge = 1e-13 * (v[-1] - v[0])
    u = []
    for x in v:
        if not u or x - u[-1] > merge:
            u.append(x)
    ts, ws = [], []
    for a, b in zip(u[:-1], u[1:]):
        pieces = 1
        while (b - a) / pieces > spacing:
            pieces *= 2
        w = (b - a) / pieces
        for p in range(pieces):
            ts.append(a + (p + 0.5) * w)
            ws.append(w)
    return ts, ws


def clip_line_box(t, c, s, xa, xb, ya, yb):
    """Parameter interval [u0, u1] of the line p(u) = t n + u d (n = (-s, c), d = (c, s)) inside the box."""
    bx, by = -t * s, t * c
    u0, u1 = -math.inf, math.inf
    for p0, d, lo, hi in ((bx, c, xa, xb), (by, s, ya, yb)):
        if d == 0.0:
            if p0 < lo or p0 > hi:
                return None
            continue
        a, b = (lo - p0) / d, (hi - p0) / d
        if a > b:
            a, b = b, a
        u0, u1 = max(u0, a), min(u1, b)
    if u1 <= u0:
        return None
    return u0, u1


def ray_segments(nx, ny, lx, ly, c, s, t, x0=0.0, y0=0.0):
    """[(cell, length, u_start)] in traversal order, plus the entry edge (0 L, 1 R, 2 B, 3 T)."""
    hx, hy = lx / nx, ly / ny
    eps = 1e-12 * min(hx, hy)
    segs = []
    for iy in range(ny):
        for ix in range(nx):
            r = clip_line_box(t, c, s, x0 + ix * hx, x0 + (ix + 1) * hx, y0 + iy * hy, y0 + (iy + 1) * hy)
            if r is not None and r[1] - r[0] > eps:
                segs.append((iy * nx + ix, r[1] - r[0], r[0]))
    segs.sort(key=lambda q: q[2])
    dom = clip_line_box(t, c, s, x0, x0 + lx, y0, y0 + ly)
    u_in = dom[0]
    px, py = -t * s + u_in * c, t * c + u_in * s
    tol = 1e-9 * max(lx, ly)
    on_x = abs(px - x0) < tol or abs(px - (x0 + lx)) < tol
    if on_x:
        edge = 0 if c > 0 else 1
    else:
        edge = 2 if s > 0 else 3
    return segs, edge


def polygon_area(poly):
    a = 0.0
    for (x1, y1), (x2, y2) in zip(poly, poly[1:] + poly[:1]):
        a += x1 * y2 - x2 * y1
    return 0.5 * abs(a)


def clip_halfplane(poly, nxv, nyv, off, keep_ge):
    """Clip a convex polygon to {p : p.n >= off} (keep_ge) or {p : p.n <= off}."""
    out = []
    f = (lambda p: p[0] * nxv + p[1] * nyv - off) if keep_ge else (lambda p: off - (p[0] * nxv + p[1] * nyv))
    n = len(poly)
    for i in range(n):
        P, Qp = poly[i], poly[(i + 1) % n]
        fp, fq = f(P), f(Qp)
        if fp >= 0:
            out.append(P)
        if (fp >= 0) != (fq >= 0):
            r = fp / (fp - fq)
            out.append((P[0] + r * (Qp[0] - P[0]), P[1] + r * (Qp[1] - P[1])))
    return out


def band_cell_area(t, w, c, s, xa, xb, ya, yb):
    """Exact area of {t - w/2 <= p.n <= t + w/2} intersected with the cell box."""
    poly = [(xa, ya), (xb, ya), (xb, yb), (xa, yb)]
    poly = clip_halfplane(poly, -s, c, t - 0.5 * w, True)
    if len(poly) < 3:
        return 0.0
    poly = clip_halfplane(poly, -s, c, t + 0.5 * w, False)
    if len(poly) < 3:
        return 0.0
    return polygon_area(poly)


def rk4_segment(I0, Q, kt, L, n=2000):
    """Integrate dI/ds = Q - kt I over s in [0, L] by RK4 (n steps); return (I(L), mean of I by Simpson)."""
    h = L / n
    I = I0
    vals = [I]
    f = lambda y: Q - kt * y
    for _ in range(n):
        k1 = f(I)
        k2 = f(I + 0.5 * h * k1)
        k3 = f(I + 0.5 * h * k2)
        k4 = f(I + h * k3)
        I = I + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        vals.append(I)
    v = np.array(vals)
    simpson = (v[0] + v[-1] + 4 * v[1:-1:2].sum() + 2 * v[2:-1:2].sum()) * h / 3.0
    return I, simpson / L
