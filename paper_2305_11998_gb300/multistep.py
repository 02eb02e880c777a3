"""Multistep runs with the material temperature advanced between sweeps (refinement stress).

One reference temperature sequence T_0, T_1, ... is produced by the FP64 sweep on a reference characteristic
grid, each step followed by the host energy balance (meb.advance).  Every other run (another ray spacing,
either precision) then steps through that same sequence: step n sweeps with kappa, B of T_{n-1}, carrying its
own intensity state, so FP32 and FP64 runs differ only by their arithmetic.
"""
from __future__ import annotations

import numpy as np
import torch

import synth

from . import meb


def _dev(a, device):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=device)


def temperature_sequence(plan, wl, T0, steps, device="cuda"):
    """[T_0 .. T_steps] (each [ncell], keV) from the FP64 sweep of `plan` + the energy balance."""
    edges = wl.edges()
    bnd = _dev(synth.boundary_left_hot(edges), device)
    Ts = [np.asarray(T0, dtype=np.float64).ravel()]
    kappa, B = synth.material(Ts[0], edges)
    I = plan.new_intensity("fp64", device)
    plan.intensity_init("fp64", I, _dev(B, device))
    out = plan.new_moments(device)
    for _ in range(steps):
        kappa, B = synth.material(Ts[-1], edges)
        plan.sweep("fp64", _dev(kappa, device), _dev(B, device), wl.c, wl.dt, I, bnd, out=out)
        T, _ = meb.advance(Ts[-1], out["E"].cpu().numpy(), edges, wl.c, wl.dt)
        Ts.append(T)
    return Ts


def run_sequence(plan, wl, Ts, prec, device="cuda", on_step=None):
    """Sweep through a given temperature sequence in one precision; on_step(n, moments, ms) after each step
    (ms: CUDA-event time of the molc_sweep call).  Returns the list of per-step moments (host numpy)."""
    edges = wl.edges()
    bnd = _dev(synth.boundary_left_hot(edges), device)
    kappa, B = synth.material(Ts[0], edges)
    I = plan.new_intensity(prec, device)
    plan.intensity_init(prec, I, _dev(B, device))
    out = plan.new_moments(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    res = []
    for n in range(1, len(Ts)):
        kappa, B = synth.material(Ts[n - 1], edges)
        k_d, B_d = _dev(kappa, device), _dev(B, device)
        e0.record()
        plan.sweep(prec, k_d, B_d, wl.c, wl.dt, I, bnd, out=out)
        e1.record()
        torch.cuda.synchronize()
        m = {k: v.cpu().numpy() for k, v in out.items()}
        res.append(m)
        if on_step is not None:
            on_step(n, m, e0.elapsed_time(e1))
    del I
    return res


def precision_errors(m32, m64, c, tol=2e-5):
    """Errors of FP32 moments against FP64 ones: E relative (floor 1e-30 max|E|); F and N_xy both in the stated
    per-cell metric (relative to max(|x|, 1e-30 max|x|): the largest value and the fraction of cells within
    `tol`) and relative to c E; Eddington factors absolute where E is above the floor."""
    E = m64["E"]
    floor = 1e-30 * np.abs(E).max()
    den = np.maximum(np.abs(E), floor)
    cE = np.maximum(c * np.abs(E), c * floor)
    out = {"E": float(np.max(np.abs(m32["E"] - E) / den))}
    for k in ("Fx", "Fy", "Nxy"):
        out[k + "/cE"] = float(np.max(np.abs(m32[k] - m64[k]) / cE))
        dk = np.maximum(np.abs(m64[k]), 1e-30 * np.abs(m64[k]).max())
        lit = np.abs(m32[k] - m64[k]) / np.where(dk > 0, dk, 1e-300)
        out[k] = float(np.max(lit))
        out[k + "_literal_pass"] = float(np.mean(lit <= tol))
    ok = np.abs(E) > floor
    for k, n in (("fxx", "Nxx"), ("fxy", "Nxy"), ("fyy", "Nyy")):
        f32 = np.where(ok, m32[n] / (c * np.where(ok, m32["E"], 1.0)), 0.0)
        f64 = np.where(ok, m64[n] / (c * np.where(ok, E, 1.0)), 0.0)
        out[k] = float(np.max(np.abs(f32 - f64)))
    return out


def refinement_norms(ys, cell_volume):
    """Mesh-refinement norms in the paper's convention (Sec. 5): for solutions y_h on successively halved
    spacings (ys[0] coarsest), ||dy_h|| = ||y_h - y_{2h}||_{L2} (cell sums weighted by the cell volume) for every
    spacing after the first, and the estimated convergence rate rho_h = ||dy_{2h}|| / ||dy_h|| for every spacing
    after the second.  Returns [{"norm": ..., "rho": ...}] aligned with ys (None where undefined)."""
    out = [{"norm": None, "rho": None}]
    for i in range(1, len(ys)):
        d = np.asarray(ys[i], dtype=np.float64) - np.asarray(ys[i - 1], dtype=np.float64)
        out.append({"norm": float(np.sqrt(cell_volume * np.sum(d * d))), "rho": None})
    for i in range(2, len(ys)):
        if out[i]["norm"] > 0:
            out[i]["rho"] = out[i - 1]["norm"] / out[i]["norm"]
    return out
