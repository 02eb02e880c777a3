"""Seeded synthetic inputs for the MOLC sweep: material fields, group Planck sources, opacities,
boundary intensities and the angular quadrature.

This module produces *inputs only*.  It holds none of the sweep's arithmetic (no ray tracing, no
attenuation, no moments); both the CUDA library and the CPU oracle consume the arrays it returns.

The workloads stand in for the Fleck-Cummings supersonic-wave problem of Sec. 4 of Coale & Anistratov
(6x6 cm slab, opacity 27/nu^3 (1 - exp(-nu/T)), 1 keV incoming radiation on the left edge, vacuum elsewhere,
17 groups).  The paper's angular set (Abu-Shumays q461214) is not available, so a Gauss-Legendre x Chebyshev
product set is used instead.

Units: lengths in cm, time in shakes (1 sh = 1e-8 s), temperature and photon energy in keV, intensity in
jerk cm^-2 sh^-1 sr^-1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Physical constants (the paper gives none; standard values in the units above).
C_LIGHT = 29.98          # cm / sh
A_RAD = 0.01372          # jerk cm^-3 keV^-4
DT_DEFAULT = 2.0e-3      # sh  (0.02 ns, the time step of Sec. 4)
T_HOT = 1.0              # keV, incoming radiation temperature on the left edge (Sec. 4)
T_COLD = 1.0e-3          # keV, initial material temperature (1 eV, Sec. 4)

EDGE_LEFT, EDGE_RIGHT, EDGE_BOTTOM, EDGE_TOP = 0, 1, 2, 3

_PI4_15 = math.pi ** 4 / 15.0


# ----------------------------------------------------------------------------------------------------------
# Planck integral.  B_g(T) = (a c / 4 pi) T^4 (15/pi^4) * int_{x_lo}^{x_hi} x^3/(e^x - 1) dx, x = nu/T.
# ----------------------------------------------------------------------------------------------------------
# Bernoulli numbers B_2k for the small-x series of int_0^x t^3/(e^t-1) dt.
_BERNOULLI_2K = [1.0 / 6, -1.0 / 30, 1.0 / 42, -1.0 / 30, 5.0 / 66, -691.0 / 2730, 7.0 / 6, -3617.0 / 510,
                 43867.0 / 798, -174611.0 / 330, 854513.0 / 138, -236364091.0 / 2730]


def _planck_head(x: np.ndarray) -> np.ndarray:
    """int_0^x t^3/(e^t - 1) dt for 0 <= x <= 1 by the Bernoulli series
    t^3/(e^t-1) = sum_n B_n t^{n+2}/n!  (B_1 = -1/2, odd B_n = 0 otherwise)."""
    x = np.asarray(x, dtype=np.float64)
    s = x ** 3 / 3.0 - x ** 4 / 8.0
    fact = 1.0
    for k, b in enumerate(_BERNOULLI_2K, start=1):
        n = 2 * k
        fact *= (n - 1) * n
        s = s + b * x ** (n + 3) / ((n + 3) * fact)
    return s


def _planck_tail(x: np.ndarray, nterms: int = 60) -> np.ndarray:
    """int_x^inf t^3/(e^t - 1) dt for x >= 1 by expanding 1/(e^t-1) = sum_n e^{-nt}:
    each term integrates to e^{-nx} (x^3/n + 3x^2/n^2 + 6x/n^3 + 6/n^4)."""
    x = np.asarray(x, dtype=np.float64)
    s = np.zeros_like(x)
    for n in range(nterms, 0, -1):
        e = np.exp(-n * x)
        s = s + e * (x ** 3 / n + 3 * x ** 2 / n ** 2 + 6 * x / n ** 3 + 6.0 / n ** 4)
    return s


def planck_fraction_between(x_lo: np.ndarray, x_hi: np.ndarray) -> np.ndarray:
    """int_{x_lo}^{x_hi} t^3/(e^t-1) dt, evaluated without cancellation in each regime."""
    x_lo = np.asarray(x_lo, dtype=np.float64)
    x_hi = np.asarray(x_hi, dtype=np.float64)
    x_lo, x_hi = np.broadcast_arrays(x_lo, x_hi)
    out = np.empty(x_lo.shape)
    X = 1.0
    both_small = x_hi <= X
    both_large = x_lo >= X
    mixed = ~(both_small | both_large)
    if both_small.any():
        out[both_small] = _planck_head(x_hi[both_small]) - _planck_head(x_lo[both_small])
    if both_large.any():
        inf_hi = np.isinf(x_hi[both_large])
        hi_tail = np.where(inf_hi, 0.0, _planck_tail(np.where(inf_hi, X, x_hi[both_large])))
        out[both_large] = _planck_tail(x_lo[both_large]) - hi_tail
    if mixed.any():
        inf_hi = np.isinf(x_hi[mixed])
        hi_tail = np.where(inf_hi, 0.0, _planck_tail(np.where(inf_hi, X, x_hi[mixed])))
        head = _planck_head(np.full(x_lo[mixed].shape, X)) - _planck_head(x_lo[mixed])
        out[mixed] = head + (_planck_tail(np.full(x_lo[mixed].shape, X)) - hi_tail)
    return np.maximum(out, 0.0)


def planck_group(T: np.ndarray, e_lo: float, e_hi: float) -> np.ndarray:
    """Group-integrated Planck intensity B_g(T) in jerk cm^-2 sh^-1 sr^-1 (summing over [0, inf) gives
    a c T^4 / 4 pi)."""
    T = np.asarray(T, dtype=np.float64)
    with np.errstate(divide="ignore", over="ignore"):
        x_lo = e_lo / T
        x_hi = e_hi / T if np.isfinite(e_hi) else np.full(T.shape, np.inf)
    frac = planck_fraction_between(x_lo, x_hi) / _PI4_15
    return (A_RAD * C_LIGHT / (4.0 * math.pi)) * T ** 4 * frac


def group_edges(G: int, e_min: float, e_max: float) -> np.ndarray:
    """G+1 log-spaced group edges in keV."""
    return np.exp(np.linspace(math.log(e_min), math.log(e_max), G + 1))


def group_centres(edges: np.ndarray) -> np.ndarray:
    """Geometric centre of each group."""
    return np.sqrt(edges[:-1] * edges[1:])


def opacity(T: np.ndarray, nu: float) -> np.ndarray:
    """Fleck-Cummings opacity kappa_nu = 27/nu^3 (1 - exp(-nu/T)) in cm^-1 (Sec. 4)."""
    T = np.asarray(T, dtype=np.float64)
    return 27.0 / nu ** 3 * (-np.expm1(-nu / T))


def material(T: np.ndarray, edges: np.ndarray):
    """kappa[g][cell] and B[g][cell] for a cell temperature field T (any shape, flattened)."""
    Tf = np.asarray(T, dtype=np.float64).ravel()
    nu = group_centres(edges)
    G = len(nu)
    kappa = np.empty((G, Tf.size))
    B = np.empty((G, Tf.size))
    for g in range(G):
        kappa[g] = opacity(Tf, nu[g])
        B[g] = planck_group(Tf, edges[g], edges[g + 1])
    return kappa, B


# ----------------------------------------------------------------------------------------------------------
# Angular quadrature: Gauss-Legendre on mu in (0,1) x Chebyshev azimuths, upper hemisphere only.
# ----------------------------------------------------------------------------------------------------------
@dataclass
class Quadrature:
    mu: np.ndarray        # cos(zeta), (0, 1]
    cos_phi: np.ndarray   # in-plane unit direction
    sin_phi: np.ndarray
    w: np.ndarray         # weights, sum = 4 pi (each direction also stands for its z-mirror)
    n_polar: int
    n_azim: int

    @property
    def n(self) -> int:
        return self.mu.size


def product_quadrature(n_polar: int, n_azim: int) -> Quadrature:
    """mu_p: Gauss-Legendre nodes mapped to (0,1) (weights summing to 1); phi_j = (j - 1/2) 2 pi / n_azim
    with equal weights; omega = 4 pi w_p / n_azim.  Direction order m = p * n_azim + j.

    cos/sin of the azimuths are evaluated once in the first octant and reflected by exact swaps and sign
    flips, so the set maps exactly onto itself under phi -> phi + pi, pi - phi, -phi and phi + pi/2."""
    if n_polar < 1 or n_azim < 4 or n_azim % 4:
        raise ValueError("need n_polar >= 1 and n_azim a positive multiple of 4")
    x, W = np.polynomial.legendre.leggauss(n_polar)
    mu_p = 0.5 * (x + 1.0)
    w_p = 0.5 * W
    Q = n_azim // 4
    # First quadrant from its lower octant, reflected about phi = pi/4 (x <-> y), so that the whole set is
    # invariant under exact 90-degree rotation as well as under the reflections.
    c1 = np.empty(Q)
    s1 = np.empty(Q)
    for j in range((Q + 1) // 2):
        phi = (j + 0.5) * 2.0 * math.pi / n_azim
        c1[j], s1[j] = math.cos(phi), math.sin(phi)
        c1[Q - 1 - j], s1[Q - 1 - j] = s1[j], c1[j]
    if Q % 2:
        c1[Q // 2] = s1[Q // 2] = math.sqrt(0.5)
    c = np.empty(n_azim)
    s = np.empty(n_azim)
    for j in range(n_azim):          # j is 0-based here, phi = (j + 1/2) 2 pi / n_azim
        if j < Q:
            c[j], s[j] = c1[j], s1[j]
        elif j < 2 * Q:              # pi - phi_{2Q-1-j}
            r = 2 * Q - 1 - j
            c[j], s[j] = -c1[r], s1[r]
        elif j < 3 * Q:              # pi + phi_{j-2Q}
            r = j - 2 * Q
            c[j], s[j] = -c1[r], -s1[r]
        else:                        # 2 pi - phi_{4Q-1-j}
            r = 4 * Q - 1 - j
            c[j], s[j] = c1[r], -s1[r]
    mu = np.repeat(mu_p, n_azim)
    w = np.repeat(4.0 * math.pi * w_p / n_azim, n_azim)
    return Quadrature(mu=mu, cos_phi=np.tile(c, n_polar), sin_phi=np.tile(s, n_polar), w=w,
                      n_polar=n_polar, n_azim=n_azim)


# ----------------------------------------------------------------------------------------------------------
# Temperature fields.
# ----------------------------------------------------------------------------------------------------------
class _Uniform:
    """Portable uniform draws: numpy's PCG64 stream through Generator.random(), which is stable across
    numpy versions and platforms; every other distribution is built from these draws."""

    def __init__(self, seed: int):
        self._rng = np.random.Generator(np.random.PCG64(seed))

    def u(self, lo: float = 0.0, hi: float = 1.0) -> float:
        return lo + (hi - lo) * float(self._rng.random())

    def int_below(self, n: int) -> int:
        return min(int(self.u() * n), n - 1)


def cell_centres(nx: int, ny: int, lx: float, ly: float, x0: float = 0.0, y0: float = 0.0):
    xc = x0 + (np.arange(nx) + 0.5) * (lx / nx)
    yc = y0 + (np.arange(ny) + 0.5) * (ly / ny)
    X, Y = np.meshgrid(xc, yc)          # [iy][ix], cell index = iy*nx + ix
    return X, Y


def smooth_noise(X: np.ndarray, Y: np.ndarray, L: float, rnd: _Uniform, n_modes: int = 4) -> np.ndarray:
    """eta = sum_k a_k sin(2 pi (p_k x + q_k y)/L + theta_k), rescaled so max|eta| = 1 over the cells."""
    eta = np.zeros_like(X)
    for _ in range(n_modes):
        while True:
            p = rnd.int_below(4)
            q = rnd.int_below(4)
            if p or q:
                break
        a = rnd.u(0.5, 1.0)
        th = rnd.u(0.0, 2.0 * math.pi)
        eta += a * np.sin(2.0 * math.pi * (p * X + q * Y) / L + th)
    m = np.max(np.abs(eta))
    return eta / m if m > 0 else eta


def temperature_front(nx: int, ny: int, L: float, seed: int, delta: float = 0.25, noise: float = 0.05,
                      n_fronts: int = 1) -> np.ndarray:
    """Cell temperatures [iy][ix] in keV: T = [T_c + (T_h - T_c) f] (1 + noise * eta).

    n_fronts == 1: f = (1 - tanh((x - x0)/delta))/2, x0 ~ U[1, 3] cm (hot behind the front on the left).
    n_fronts > 1: fronts with unit normals at angles ~ U[0, 2 pi) through points ~ U[1,5]^2, each hot on the
    side away from the domain centre; f = max over fronts of (1 - tanh(d/delta))/2, d the distance to the
    front (positive on the centre side)."""
    rnd = _Uniform(seed)
    X, Y = cell_centres(nx, ny, L, L)
    if n_fronts == 1:
        x0 = rnd.u(1.0, 3.0)
        f = 0.5 * (1.0 - np.tanh((X - x0) / delta))
    else:
        f = np.zeros_like(X)
        for _ in range(n_fronts):
            th = rnd.u(0.0, 2.0 * math.pi)
            px, py = rnd.u(1.0, 5.0), rnd.u(1.0, 5.0)
            d = (X - px) * math.cos(th) + (Y - py) * math.sin(th)
            if (0.5 * L - px) * math.cos(th) + (0.5 * L - py) * math.sin(th) < 0.0:
                d = -d                     # the hot side is the side away from the domain centre
            f = np.maximum(f, 0.5 * (1.0 - np.tanh(d / delta)))
    eta = smooth_noise(X, Y, L, rnd)
    return (T_COLD + (T_HOT - T_COLD) * f) * (1.0 + noise * eta)


def boundary_left_hot(edges: np.ndarray, T_in: float = T_HOT) -> np.ndarray:
    """bnd[4][G]: isotropic incoming intensity per edge (left, right, bottom, top); left = B_g(T_in), rest vacuum."""
    G = len(edges) - 1
    bnd = np.zeros((4, G))
    for g in range(G):
        bnd[EDGE_LEFT, g] = planck_group(np.array([T_in]), edges[g], edges[g + 1])[0]
    return bnd


# ----------------------------------------------------------------------------------------------------------
# Named workloads.
# ----------------------------------------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    L: float
    G: int
    e_min: float
    e_max: float
    n_polar: int
    n_azim: int
    spacing_div: int          # ray spacing = h / spacing_div
    steps: int
    n_fronts: int = 1
    cold_start: bool = False  # T = T_COLD everywhere
    c: float = C_LIGHT
    dt: float = DT_DEFAULT
    extra: dict = field(default_factory=dict)

    @property
    def h(self) -> float:
        return self.L / self.nx

    @property
    def spacing(self) -> float:
        return self.h / self.spacing_div

    @property
    def ncell(self) -> int:
        return self.nx * self.ny

    def edges(self) -> np.ndarray:
        return group_edges(self.G, self.e_min, self.e_max)

    def quadrature(self) -> Quadrature:
        return product_quadrature(self.n_polar, self.n_azim)

    def temperature(self, seed: int = 0) -> np.ndarray:
        if self.cold_start:
            return np.full((self.ny, self.nx), T_COLD)
        return temperature_front(self.nx, self.ny, self.L, seed, n_fronts=self.n_fronts)

    def inputs(self, seed: int = 0) -> dict:
        """Everything one sweep needs, as float64 numpy arrays (kappa, B: [G][ncell]; bnd: [4][G])."""
        edges = self.edges()
        T = self.temperature(seed)
        kappa, B = material(T, edges)
        return dict(T=T, edges=edges, kappa=kappa, B=B, bnd=boundary_left_hot(edges), quad=self.quadrature(),
                    c=self.c, dt=self.dt)


# Fleck-Cummings-shaped stand-ins (6x6 cm, left edge at 1 keV, vacuum elsewhere).
WORKLOADS = {
    # small parity case: 16x16 cells, 4 groups 0.01-10 keV, 2 polar x 16 azimuths, spacing h/2, one step
    "fc16_g4_d32": Workload("fc16_g4_d32", 16, 16, 6.0, 4, 0.01, 10.0, 2, 16, 2, 1),
    # ten carried steps: 64x64, 17 groups 0.001-100 keV, 4 x 32 directions, spacing h/4
    "fc64_g17_d128": Workload("fc64_g17_d128", 64, 64, 6.0, 17, 0.001, 100.0, 4, 32, 4, 10),
    # production size (roofline point): 512x512, 17 groups, 4 x 32 directions, spacing h/2, three fronts
    "fc512_g17_d128": Workload("fc512_g17_d128", 512, 512, 6.0, 17, 0.001, 100.0, 4, 32, 2, 1, n_fronts=3),
    # profiling size of the production workload (same generators; 3.3 GB FP32 state, accumulators > L2)
    "fc384_g17_d128": Workload("fc384_g17_d128", 384, 384, 6.0, 17, 0.001, 100.0, 4, 32, 2, 1, n_fronts=3),
    # profiling sizes of the batched pattern's smaller polar counts: 256x256, 17 groups, spacing h/2, one front,
    # 3 polar x 48 azimuths and 2 polar x 64 azimuths
    "fc256_g17_p3x48": Workload("fc256_g17_p3x48", 256, 256, 6.0, 17, 0.001, 100.0, 3, 48, 2, 1),
    "fc256_g17_p2x64": Workload("fc256_g17_p2x64", 256, 256, 6.0, 17, 0.001, 100.0, 2, 64, 2, 1),
    # refinement stress base grid: 128x128, 17 groups, 8 x 64 directions, cold start (spacing set per run)
    "fc128_g17_d512": Workload("fc128_g17_d512", 128, 128, 6.0, 17, 0.001, 100.0, 8, 64, 2, 50,
                               cold_start=True),
}


def batch_instances(n: int = 64, seed: int = 0) -> list[Workload]:
    """Uneven independent instances: cells per side in {32,64,128,256}, G in {8,17,32}, 2-4 polar x
    {16,...,64 step 8} azimuths, spacing h/2 or h/4 (20 steps each)."""
    rnd = _Uniform(10_000 + seed)
    out = []
    for i in range(n):
        N = (32, 64, 128, 256)[rnd.int_below(4)]
        G = (8, 17, 32)[rnd.int_below(3)]
        npol = 2 + rnd.int_below(3)
        naz = 16 + 8 * rnd.int_below(7)
        div = (2, 4)[rnd.int_below(2)]
        out.append(Workload(f"batch{i}_n{N}_g{G}_p{npol}_a{naz}_s{div}", N, N, 6.0, G, 0.001, 100.0, npol, naz,
                            div, 20, extra=dict(seed=seed * 1000 + i)))
    return out
