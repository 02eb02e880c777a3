"""Material energy balance between sweeps, on the host in FP64: the coupling of the multistep runs.

The paper closes the transport with the MLQD method (low-order equations iterated with the energy balance of
Eq. 3 / Eq. 6); that solver is not part of this library.  For multistep runs of the sweep alone, the material
temperature is advanced after each sweep by the backward-Euler energy balance of Eq. 3 with the sweep's E_g
held fixed (reading the 4 pi of Eq. 3 onto B_g, as in Eq. 6):

    c_v (T^n - T^{n-1}) / dt = sum_g kappa_g(T^n) (c E_g^n - 4 pi B_g(T^n)),

solved per cell by a safeguarded Newton iteration (bisection whenever a step leaves the bracket).  This is a
transport-only stand-in: it is not the paper's algorithm and converges nothing between the sweep and the
balance within a step.
"""
from __future__ import annotations

import math

import numpy as np

import synth

C_V = 0.5917 * synth.A_RAD      # jerk cm^-3 keV^-1: heat capacity 0.5917 a_R (1 keV)^3 per keV


def _x3_over_expm1(x):
    """x^3 / (e^x - 1) (0 at x = 0 and as x -> inf)."""
    with np.errstate(over="ignore", invalid="ignore", divide="ignore"):
        v = x ** 3 / np.expm1(x)
    return np.where(np.isfinite(x) & (x > 0), np.nan_to_num(v, nan=0.0, posinf=0.0), 0.0)


def _residual_and_slope(T, T_old, cE, edges, dt, cv):
    """r(T) = c_v (T - T_old)/dt - sum_g kappa_g(T) (c E_g - 4 pi B_g(T)) per cell and dr/dT (analytic:
    d kappa_g/dT from kappa = 27/nu^3 (1 - e^{-nu/T}); dB_g/dT = 4 B_g/T + (a c / 4 pi) T^3 (15/pi^4)
    (x_lo f(x_lo) - x_hi f(x_hi)), f(x) = x^3/(e^x - 1), x = nu/T)."""
    kappa, B = synth.material(T, edges)
    nu = synth.group_centres(edges)[:, None]
    lo, hi = edges[:-1, None], edges[1:, None]
    dkappa = -27.0 / nu ** 3 * np.exp(-nu / T) * nu / T ** 2
    xl, xh = lo / T, hi / T
    dB = 4.0 * B / T + (synth.A_RAD * synth.C_LIGHT / (4.0 * math.pi)) * T ** 3 * (15.0 / math.pi ** 4) * (
        xl * _x3_over_expm1(xl) - xh * _x3_over_expm1(xh))
    src = cE - 4.0 * math.pi * B
    r = cv * (T - T_old) / dt - np.sum(kappa * src, axis=0)
    d = cv / dt - np.sum(dkappa * src - 4.0 * math.pi * kappa * dB, axis=0)
    scale = cv * (T + T_old) / dt + np.sum(kappa * (np.abs(cE) + 4.0 * math.pi * B), axis=0)
    return r, d, scale


def advance(T_old, E, edges, c, dt, cv=C_V, t_min=1.0e-5, rtol=1.0e-13, max_iter=100):
    """T^n per cell from T^{n-1} ([ncell] keV) and the step's E_g ([G][ncell]); returns (T, iterations)."""
    T_old = np.asarray(T_old, dtype=np.float64).ravel()
    cE = c * np.asarray(E, dtype=np.float64)
    nu = synth.group_centres(edges)
    # bracket: r(t_min) < 0 (heating can only raise T above t_min when T_old > t_min), and at
    # T_hi = T_old + dt sum_g kappa_g^max max(c E_g, 0) / c_v the heating term bounds the sum from above
    kmax = 27.0 / nu[:, None] ** 3
    lo = np.full_like(T_old, t_min)
    hi = np.maximum(T_old, t_min) + dt * np.sum(kmax * np.maximum(cE, 0.0), axis=0) / cv + 1.0e-6
    T = np.clip(T_old, lo, hi)
    act = np.arange(T.size)          # cells still iterating
    for it in range(1, max_iter + 1):
        Ta = T[act]
        r, d, scale = _residual_and_slope(Ta, T_old[act], cE[:, act], edges, dt, cv)
        la = np.where(r < 0, Ta, lo[act])
        ha = np.where(r > 0, Ta, hi[act])
        with np.errstate(divide="ignore", invalid="ignore"):
            Tn = Ta - r / d
        # converged: the residual, the Newton step or the bracket is at the level of rounding
        conv = (np.abs(r) <= 1e-15 * scale) | (np.abs(Tn - Ta) <= rtol * np.abs(Ta)) | (ha - la <= rtol * ha)
        Tn = np.where(conv & np.isfinite(Tn), np.clip(Tn, la, ha), Tn)
        bad = ~conv & (~np.isfinite(Tn) | (Tn <= la) | (Tn >= ha))
        Tn = np.where(bad, 0.5 * (la + ha), Tn)
        T[act], lo[act], hi[act] = Tn, la, ha
        act = act[~conv]
        if act.size == 0:
            return T, it
    return T, max_iter
