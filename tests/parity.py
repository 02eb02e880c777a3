"""Parity metrics shared by the GPU tests (test helper).

The per-cell error of an output x is |x_gpu - x_ref| / max(|x_ref|, 1e-30 max|x_ref|), the metric the
accuracy targets are stated in.  E, N_xx, N_yy (positive sums) and f_xx, f_yy are held to it literally.

F_x, F_y and N_xy are sums of terms of both signs (they vanish by symmetry in equilibrium).  Their per-cell
relative error is bounded by the unit roundoff u times the sum's condition number sum|terms| / |sum|,
which is unbounded where the output crosses zero, so no arithmetic meets a fixed relative bound there.  For
these outputs the denominator also contains eta * x_abs, where x_abs = (1/V) sum omega |Omega..| A |Ibar - B|
is the magnitude of the deviation terms the GPU paths sum (computed by the oracle) and eta = C u / tol with
C = 64 for FP32 and C = 32 for FP64: cells whose output is at least eta x_abs are held to the literal relative
bound, the others to an absolute error of C u x_abs.  For FP32 the per-term error is not just a few u: tau is
formed from kappa~, l and 1/sin(zeta), each rounded to FP32, so e^-tau carries a relative error ~tau u, which
accumulates along a beam like a random walk over its segments (measured up to ~40 u of the deviation
magnitude on the 64^2 and 512^2 workloads).

When the reference is the double-precision oracle, which sums the literal intensities, its own error on a
signed moment is ~u_64 c E; the denominator then also contains 64 u_64 c E / tol.  N_xy also carries the Planck
part B geo_xy, added in FP64 from geometric moments (exactly 0 in the uniform layout, a tiny nonzero in the
paper layout): its denominator also contains 8 u_64 (1/V) sum omega A |Ox Oy| B / tol.  The FP32 path carries B
as two FP32 words (48 significant bits) and forms its deviations from B differences at every cell crossing, so
its signed moments also have an error floor ~2^-48 of their Planck magnitude (1/V) sum omega A |Omega..| B,
visible only where the deviations are tiny against B (cold cells): the denominator also contains
64 2^-48 (1/V) sum omega A |Omega..| B / tol.

The floor 1e-30 max|x| is taken over the whole output array (all groups); `floor_max` passes it when only some
groups are compared.  The literal pass fraction is reported alongside.

The Eddington factors f = N / (c E) are compared in the cells whose E is above that floor; below it E and N
are both unresolved and their ratio carries no information.
"""
import numpy as np

TOL = {"fp64": 1e-12, "fp32": 2e-5}
UNIT_ROUNDOFF = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}
TOL_F_ABS_FP32 = 1e-6          # absolute bound on the Eddington factors for the FP32 path
SIGNED = {"Fx": "absFx", "Fy": "absFy", "Nxy": "absNxy"}


ETA_C = {"fp64": 32.0, "fp32": 64.0}


def eta(prec: str, eta_c=None) -> float:
    return (ETA_C[prec] if eta_c is None else eta_c) * UNIT_ROUNDOFF[prec] / TOL[prec]


def rel_error(got, ref, absmag=None, eta_=0.0, floor_max=None, extra=None):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mx = np.max(np.abs(ref)) if floor_max is None else floor_max
    den = np.maximum(np.abs(ref), 1e-30 * mx)
    if absmag is not None:
        den = np.maximum(den, eta_ * np.asarray(absmag))
    if extra is not None:
        den = np.maximum(den, extra)
    den = np.where(den > 0, den, 1e-300)
    return np.abs(got - ref) / den


def _worst(err, got, ref, k, ak):
    g, i = np.unravel_index(np.argmax(err), np.shape(err))
    return dict(group=int(g), cell=int(i), got=float(got[k][g, i]), ref=float(ref[k][g, i]),
                abs=float(ref[ak][g, i]), E=float(ref["E"][g, i]))


def closure(m, c):
    cE = c * np.asarray(m["E"])
    safe = np.where(cE > 0, cE, 1.0)
    return {k: np.where(cE > 0, np.asarray(m[n]) / safe, 0.0) for k, n in (("fxx", "Nxx"), ("fxy", "Nxy"),
                                                                          ("fyy", "Nyy"))}


def compare(got: dict, ref: dict, prec: str, c: float, report=None, ref_precision="quad", floor_max=None,
            eta_c=None):
    """Assert the targets for one sweep's moments; return a dict of max errors (literal and gated).
    floor_max: {name: max|x| over the whole output} when `got`/`ref` hold a subset of the groups.
    eta_c: the constant C of the signed-moment gate when a case sums far more terms per cell than the
    workloads ETA_C was set on (recursive summation of n terms in any order errs by at most (n - 1) u sum|terms|,
    so C = n is a bound)."""
    tol = TOL[prec]
    e = eta(prec, eta_c)
    fm = floor_max or {}
    out = {}
    for k in ("E", "Nxx", "Nyy"):
        r = rel_error(got[k], ref[k], floor_max=fm.get(k))
        out[k] = float(r.max())
        assert out[k] <= tol, (k, out[k])
    ref_err = None
    if ref_precision == "double":
        ref_err = 64.0 * UNIT_ROUNDOFF["fp64"] / tol * c * np.asarray(ref["E"])
    for k, ak in SIGNED.items():
        lit = rel_error(got[k], ref[k], floor_max=fm.get(k))
        extra = ref_err
        bk = "absB" + k
        if bk in ref:
            # Planck parts: N_xy adds B geo_xy in FP64 from geometric moments (a tiny nonzero in the paper
            # layout), a few u_64 of its magnitude; the FP32 path forms its deviations from B differences at every
            # crossing with B carried as two FP32 words (a 48-bit significand), an error floor of ~2^-48 of the
            # Planck magnitude (1/V) sum omega A |Omega..| B that grows along the characteristics (C = 64)
            pb = (8.0 * UNIT_ROUNDOFF["fp64"] if k == "Nxy" else 0.0) + (64.0 * 2.0 ** -48 if prec == "fp32" else 0.0)
            if pb > 0:
                pb = pb / tol * np.asarray(ref[bk])
                extra = pb if extra is None else np.maximum(extra, pb)
        gated = rel_error(got[k], ref[k], ref[ak], e, floor_max=fm.get(k), extra=extra)
        out[k] = float(gated.max())
        out[k + "_literal_pass"] = float(np.mean(lit <= tol))
        assert out[k] <= tol, (k, out[k], _worst(gated, got, ref, k, ak))
    fg = closure(got, c)
    fr = closure(ref, c)
    cE = c * np.asarray(ref["E"])
    safe = np.where(cE > 0, cE, 1.0)
    resolved = np.asarray(ref["E"]) >= 1e-30 * (fm.get("E") or np.max(np.abs(ref["E"])))
    if prec == "fp32":
        for k in ("fxx", "fxy", "fyy"):
            err = np.where(resolved, np.abs(fg[k] - fr[k]), 0.0)
            out[k] = float(np.max(err))
            assert out[k] <= TOL_F_ABS_FP32, (k, out[k])
    else:
        for k in ("fxx", "fyy"):
            out[k] = float(np.where(resolved, rel_error(fg[k], fr[k]), 0.0).max())
            assert out[k] <= tol, (k, out[k])
        ex = None if ref_err is None else ref_err
        if "absBNxy" in ref:   # the FP64 Planck part of N_xy, as above
            pb = 8.0 * UNIT_ROUNDOFF["fp64"] / tol * np.asarray(ref["absBNxy"])
            ex = pb if ex is None else np.maximum(ex, pb)
        r = rel_error(fg["fxy"], fr["fxy"], np.where(cE > 0, ref["absNxy"] / safe, 0.0), e,
                      extra=None if ex is None else np.where(cE > 0, ex / safe, 0.0))
        out["fxy"] = float(np.where(resolved, r, 0.0).max())
        assert out["fxy"] <= tol, ("fxy", out["fxy"])
    if report is not None:
        report.append(out)
    return out
