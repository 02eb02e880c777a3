"""Pins of the oracle's running error bound (CPU): the bound it reports for a path's arithmetic must hold for an
independent emulation of that arithmetic (tests/fp_emulation.py), element by element, over two steps with the
state carried, and must fail for a model whose unit roundoff is 64 times too small (so it is not vacuous)."""
import numpy as np
import pytest

import error_model
import fp_emulation
import oracle
import synth


def _case(name, seed):
    wl = synth.WORKLOADS[name]
    d = wl.inputs(seed)
    geom = oracle.Geometry.from_workload(wl)
    return wl, d, geom


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name,seed", [("fc16_g4_d32", 0), ("fc16_g4_d32", 5)])
def test_bound_holds_for_emulated_path_over_two_steps(prec, name, seed):
    wl, d, geom = _case(name, seed)
    tr = oracle.tracks(geom)
    em = error_model.model(prec, wl.n_polar, d["B"], d["bnd"])
    dev_o = dev_e = err = None
    used = []
    for step in range(2):
        ref = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=dev_o, I_as_deviation=True,
                           I_prev_is_deviation=True, errmodel=em, I_err=err)
        emu = fp_emulation.emulate(tr, geom.mu, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], prec,
                                   dev_prev=dev_e)
        e = np.abs(emu - ref["I"])
        b = ref["I_err"]
        assert np.all(e <= b), (step, float(np.max(e / np.maximum(b, 1e-300))))
        used.append(float(np.max(e / np.maximum(b, 1e-300))))
        dev_o, dev_e, err = ref["I"], emu, ref["I_err"]
    # the bound is within a few hundred of the actual error (first-order worst case, summed along characteristics)
    assert max(used) > 1e-3, used


@pytest.mark.parametrize("seed", [0, 1])
def test_bound_holds_with_the_hardware_approximations_at_their_allowances(seed):
    """The FP32 path computes 2^x with ex2.approx and 1/x with rcp.approx; the bound allows them relative errors of
    2^-21 and 2^-22 (above the accuracies the PTX ISA gives them).  The emulation with every 2^x and 1/x off by those
    allowances (seeded signs) must stay within it over two steps; a bound that left the approximations' error out
    is exceeded here (by a quarter, measured on a mutant of the oracle)."""
    wl, d, geom = _case("fc16_g4_d32", 3)
    tr = oracle.tracks(geom)
    em = error_model.model("fp32", wl.n_polar, d["B"], d["bnd"])
    dev_o = dev_e = err = None
    for step in range(2):
        ref = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=dev_o, I_as_deviation=True,
                           I_prev_is_deviation=True, errmodel=em, I_err=err)
        emu = fp_emulation.emulate(tr, geom.mu, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], "fp32",
                                   dev_prev=dev_e, approx=(2.0 ** -21, 2.0 ** -22, 100 * seed + step))
        e = np.abs(emu - ref["I"])
        assert np.all(e <= ref["I_err"]), (step, float(np.max(e / np.maximum(ref["I_err"], 1e-300))))
        dev_o, dev_e, err = ref["I"], emu, ref["I_err"]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bound_with_too_small_unit_roundoff_is_violated(prec):
    """A planted mistake in the model (u 64 times too small, the intrinsic errors likewise) must be caught by the
    emulation somewhere: the bound tracks the arithmetic, it is not vacuous."""
    wl, d, geom = _case("fc16_g4_d32", 1)
    tr = oracle.tracks(geom)
    em = error_model.model(prec, wl.n_polar, d["B"], d["bnd"])
    for k in ("u", "e_exp", "e_rcp"):
        if k in em:
            em[k] /= 64.0
    ref = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_as_deviation=True, errmodel=em)
    emu = fp_emulation.emulate(tr, geom.mu, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], prec)
    assert np.any(np.abs(emu - ref["I"]) > ref["I_err"])


def test_moment_bounds_scale_with_unit_roundoff_and_cover_magnitudes():
    """Bookkeeping of the moment bounds: first order in the model's error constants (all of them doubled roughly
    double the bound beyond the fixed FP64 assembly term: between 2x, less the fixed series truncation, and 4x for
    the u^2 terms of the two-word B), and at least k_sum u times the deviation magnitude for the FP32 model."""
    wl, d, geom = _case("fc16_g4_d32", 2)
    em = error_model.model("fp32", wl.n_polar, d["B"], d["bnd"])
    r1 = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], want_I=False, errmodel=em)
    em2 = dict(em, **{k: 2 * em[k] for k in ("u", "e_exp", "e_rcp", "abs_unit")})
    r2 = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], want_I=False, errmodel=em2)
    for k in oracle.BOUND_NAMES:
        fixed = 8 * 2.0 ** -53 * (r1["dev"][k] + r1["plk"][k])
        v1, v2 = r1["bound"][k] - fixed, r2["bound"][k] - fixed
        live = v1 > 0
        ratio = v2[live] / v1[live]
        assert np.all((ratio > 1.9) & (ratio < 4.01)), (k, float(ratio.min()), float(ratio.max()))
        assert np.all(r1["bound"][k] >= em["k_sum"] * em["u"] * r1["dev"][k] * (1 - 1e-12)), k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_bound_holds_when_B_changes_between_steps(prec):
    """Step 2 with a new B: the path's stored deviations refer to the old B (B_ref), the oracle's are re-referenced
    to the new B in double (that rounding added to the carried bound)."""
    wl, d, geom = _case("fc16_g4_d32", 3)
    tr = oracle.tracks(geom)
    cells = tr["cell"]
    B2 = d["B"] * np.exp(np.random.default_rng(9).uniform(-0.3, 0.3, d["B"].shape))
    em1 = error_model.model(prec, wl.n_polar, d["B"], d["bnd"])
    r1 = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_as_deviation=True, errmodel=em1)
    e1 = fp_emulation.emulate(tr, geom.mu, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], prec)
    jump = (d["B"] - B2)[:, cells].T
    dev2 = r1["I"] + jump
    err2 = r1["I_err"] + 2 * 2.0 ** -53 * (np.abs(dev2) + np.abs(jump))
    em2 = error_model.model(prec, wl.n_polar, B2, d["bnd"], Bref=d["B"])
    r2 = oracle.sweep(geom, d["kappa"], B2, d["c"], d["dt"], d["bnd"], I_prev=dev2, I_as_deviation=True,
                      I_prev_is_deviation=True, errmodel=em2, I_err=err2)
    e2 = fp_emulation.emulate(tr, geom.mu, d["kappa"], B2, d["c"], d["dt"], d["bnd"], prec, dev_prev=e1,
                              Bref=d["B"])
    assert np.all(np.abs(e2 - r2["I"]) <= r2["I_err"])
