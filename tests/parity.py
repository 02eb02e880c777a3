"""Parity gate shared by the GPU tests (test helper).

The reference is the binary128 oracle, run with the error model of the path under test (tests/error_model.py)
so that it also returns 'bound': a first-order bound, derived from that path's sequence of operations and
the stated accuracies of the functions it calls, of the error its arithmetic may make in each cell output.
Nothing in the gate comes from a measurement of the GPU path.

The targets are stated per cell and group as |x_gpu - x_ref| / max(|x_ref|, 1e-30 max|x_ref|): at most 1e-12
for the FP64 path; for the FP32 path at most 2e-5 on E and F and 1e-6 absolute on the Eddington factors.

* E, N_xx, N_yy are held to the literal metric.
* F_x, F_y, N_xy are sums of terms of both signs; where they cross zero their relative error in any finite
  arithmetic is unbounded (the condition number sum|terms| / |sum| grows without limit).  They are held to
  |x_gpu - x_ref| <= max(tol |x_ref|, tol 1e-30 max|x_ref|, bound_x): the literal metric in every cell the path's
  arithmetic resolves to the tolerance (bound_x <= tol |x_ref|), and the derived bound of that arithmetic in the
  others.  Reported beside it: the literal maximum and pass fraction, the fraction of cells the arithmetic
  cannot resolve to the tolerance, and the largest |x_gpu - x_ref| / bound_x (how much of the bound is used).
* The Eddington factors f = N / (c E) are compared where E is above the floor (below it E and N are both
  unresolved): FP32 to 1e-6 absolute; FP64 f_xx, f_yy literally and f_xy like the signed moments, with
  bound_f = (bound_N + |f| c bound_E) / (c E) + 2 u64 |f|.

The floor 1e-30 max|x| is taken over the whole output array (all groups); `floor_max` passes it when only some
groups are compared.
"""
import numpy as np

import error_model
import oracle

TOL = {"fp64": 1e-12, "fp32": 2e-5}
TOL_F_ABS_FP32 = 1e-6          # absolute bound on the Eddington factors for the FP32 path
U64 = 2.0 ** -53
SIGNED = ("Fx", "Fy", "Nxy")


def reference(geom, d, prec, n_polar, groups=None, I_prev=None, I_err=None, want_I=False, Bref=None, **kw):
    """The binary128 oracle on the inputs `d`, with the error model of path `prec` (its state carried as
    deviations from B; I_err the bound of the path's state entering this step)."""
    em = error_model.model(prec, n_polar, d["B"], d["bnd"], Bref=Bref)
    return oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=I_prev, groups=groups,
                        precision="quad", want_I=want_I or I_prev is not None, I_as_deviation=True,
                        I_prev_is_deviation=True, errmodel=em, I_err=I_err, **kw)


def rel_error(got, ref, floor_max=None, den_min=None):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    mx = np.max(np.abs(ref)) if floor_max is None else floor_max
    den = np.maximum(np.abs(ref), 1e-30 * mx)
    if den_min is not None:
        den = np.maximum(den, den_min)
    den = np.where(den > 0, den, 1e-300)
    return np.abs(got - ref) / den


def closure(m, c):
    cE = c * np.asarray(m["E"])
    safe = np.where(cE > 0, cE, 1.0)
    return {k: np.where(cE > 0, np.asarray(m[n]) / safe, 0.0) for k, n in (("fxx", "Nxx"), ("fxy", "Nxy"),
                                                                          ("fyy", "Nyy"))}


def _worst(err, got, ref, k):
    g, i = np.unravel_index(np.argmax(err), np.shape(err))
    return dict(group=int(g), cell=int(i), got=float(got[k][g, i]), ref=float(ref[k][g, i]),
                bound=float(ref["bound"][k][g, i]), E=float(ref["E"][g, i]))


def compare(got: dict, ref: dict, prec: str, c: float, report=None, floor_max=None):
    """Assert the targets for one sweep's moments against a `reference()` result; return the errors.
    floor_max: {name: max|x| over the whole output} when `got`/`ref` hold a subset of the groups."""
    assert "bound" in ref, "the reference must come from reference(): the binary128 oracle with an error model"
    tol = TOL[prec]
    fm = floor_max or {}
    out = {}
    for k in ("E", "Nxx", "Nyy"):
        r = rel_error(got[k], ref[k], floor_max=fm.get(k))
        out[k] = float(r.max())
        assert out[k] <= tol, (k, out[k])
    for k in SIGNED:
        bnd = np.asarray(ref["bound"][k])
        lit = rel_error(got[k], ref[k], floor_max=fm.get(k))
        gated = rel_error(got[k], ref[k], floor_max=fm.get(k), den_min=bnd / tol)
        diff = np.abs(np.asarray(got[k]) - np.asarray(ref[k]))
        out[k] = float(gated.max())
        out[k + "_literal"] = float(lit.max())
        out[k + "_literal_pass"] = float(np.mean(lit <= tol))
        out[k + "_unresolved"] = float(np.mean(bnd > tol * np.abs(ref[k])))
        out[k + "_bound_use"] = float(np.max(np.where(bnd > 0, diff / np.where(bnd > 0, bnd, 1.0), 0.0)))
        assert out[k] <= tol, (k, out[k], _worst(gated, got, ref, k))
    fg = closure(got, c)
    fr = closure(ref, c)
    E = np.asarray(ref["E"])
    cE = c * E
    safe = np.where(cE > 0, cE, 1.0)
    resolved = E >= 1e-30 * (fm.get("E") or np.max(np.abs(E)))
    if prec == "fp32":
        for k in ("fxx", "fxy", "fyy"):
            err = np.where(resolved, np.abs(fg[k] - fr[k]), 0.0)
            out[k] = float(np.max(err))
            assert out[k] <= TOL_F_ABS_FP32, (k, out[k])
    else:
        for k in ("fxx", "fyy"):
            out[k] = float(np.where(resolved, rel_error(fg[k], fr[k]), 0.0).max())
            assert out[k] <= tol, (k, out[k])
        bf = np.where(cE > 0, (ref["bound"]["Nxy"] + np.abs(fr["fxy"]) * c * ref["bound"]["E"]) / safe, 0.0)
        bf = bf + 2 * U64 * np.abs(fr["fxy"])
        r = rel_error(fg["fxy"], fr["fxy"], den_min=bf / tol)
        out["fxy"] = float(np.where(resolved, r, 0.0).max())
        assert out["fxy"] <= tol, ("fxy", out["fxy"])
    if report is not None:
        report.append(out)
    return out


def check_state(g_abs, r_dev, Bseg, I_err, prec):
    """The carried state per segment, direction and group: the exported segment averages (absolute, formed in
    FP64 as B_ref + deviation) against the oracle's deviations plus B of the segment's cell, within the bound of
    the path's state plus the FP64 roundings of the two absolute values (2 u64 |Ibar| each)."""
    r_abs = np.asarray(r_dev) + Bseg
    allow = np.asarray(I_err) + 4 * U64 * np.abs(r_abs) + 1e-300
    err = np.abs(np.asarray(g_abs) - r_abs)
    assert np.all(err <= allow), float(np.max(err / allow))
    tol = TOL[prec]
    lit = err / np.maximum(np.abs(np.asarray(r_dev)), 1e-30 * np.abs(r_abs).max())
    return {"state_bound_use": float(np.max(err / allow)), "state_literal_pass": float(np.mean(lit <= tol))}
