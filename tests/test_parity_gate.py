"""The parity gate itself (tests/parity.py) on the CPU: it passes the reference's own values and fails a result
with one error planted just above the stated tolerance, in each of its checks, while an error just below passes.

The reference is the binary128 oracle with the FP32 or FP64 path's error model on the 16^2 workload; the
"result" is a copy of its moments with one value changed in one cell (mistakes are planted in data handed to the
gate, on the CPU)."""
import numpy as np
import pytest

import oracle
import parity
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

NAMES = ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy")


@pytest.fixture(scope="module")
def refs():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=0)
    geom = oracle.Geometry.from_workload(wl)
    return {p: parity.reference(geom, d, p, wl.n_polar) for p in ("fp32", "fp64")}, d["c"]


def copy_of(r):
    return {k: np.array(r[k], dtype=np.float64) for k in NAMES}


def failing_check(got, r, prec, c):
    """None when the gate passes `got`, else the name of the first check that failed."""
    try:
        parity.compare(got, r, prec, c)
        return None
    except AssertionError as e:
        return e.args[0][0]


def cell_where(mask, score):
    """(group, cell) of the largest score among the cells where mask holds."""
    s = np.where(mask, score, -np.inf)
    g, i = np.unravel_index(np.argmax(s), s.shape)
    assert np.isfinite(s[g, i])
    return g, i


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_reference_passes_its_own_gate(refs, prec):
    r, c = refs[0][prec], refs[1]
    out = parity.compare(copy_of(r), r, prec, c)
    assert all(out[k] == 0.0 for k in NAMES)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["E", "Nxx", "Nyy"])
def test_literal_moments_fail_just_above_the_tolerance(refs, prec, name):
    r, c = refs[0][prec], refs[1]
    tol = parity.TOL[prec]
    x = np.asarray(r[name])
    g, i = cell_where(np.abs(x) > 1e-20 * np.abs(x).max(), np.abs(x))
    # E with the N's scaled alike leaves the factors f = N / (c E) unchanged; an N alone moves its factor, which the
    # FP32 path holds to 1e-6 absolute, tighter than 2e-5 of N: below the tolerance only the moment's own check
    # is asked to pass
    scaled = ("E", "Nxx", "Nxy", "Nyy") if name == "E" else (name,)
    for factor, fails in ((0.5, False), (1.5, True)):
        got = copy_of(r)
        for n in scaled:
            got[n][g, i] = np.asarray(r[n])[g, i] * (1 + factor * tol)
        check = failing_check(got, r, prec, c)
        assert (check == name) is fails, (name, factor, check)
        if prec == "fp64" or name == "E":
            assert (check is None) is not fails, (name, factor, check)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["Fx", "Fy", "Nxy"])
def test_signed_moments_resolved_cells_held_to_the_tolerance(refs, prec, name):
    """Where the path's arithmetic resolves a signed moment to the tolerance (bound <= tol |x|), the literal
    metric applies."""
    r, c = refs[0][prec], refs[1]
    tol = parity.TOL[prec]
    x, b = np.asarray(r[name]), np.asarray(r["bound"][name])
    g, i = cell_where((b < 0.5 * tol * np.abs(x)) & (np.abs(x) > 1e-20 * np.abs(x).max()), np.abs(x))
    for factor, fails in ((0.5, False), (1.5, True)):
        got = copy_of(r)
        got[name][g, i] = x[g, i] + factor * tol * abs(x[g, i])
        check = failing_check(got, r, prec, c)
        assert (check == name) is fails, (name, factor, check)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("name", ["Fx", "Fy", "Nxy"])
def test_signed_moments_unresolved_cells_held_to_the_derived_bound(refs, prec, name):
    """Where the arithmetic cannot resolve the tolerance (bound > tol |x|, the moment near zero), an error
    within the derived bound passes and one beyond it fails."""
    r, c = refs[0][prec], refs[1]
    tol = parity.TOL[prec]
    x, b = np.asarray(r[name]), np.asarray(r["bound"][name])
    floor = tol * 1e-30 * np.abs(x).max()
    mask = (b > 4 * tol * np.abs(x)) & (b > 4 * floor)
    if not mask.any():
        pytest.skip(f"no unresolved {name} cell in this case")
    g, i = cell_where(mask, b)
    for factor, fails in ((0.5, False), (2.0, True)):
        got = copy_of(r)
        got[name][g, i] = x[g, i] + factor * b[g, i]
        check = failing_check(got, r, prec, c)
        assert (check == name) is fails, (name, factor, check)


def test_fp32_factors_held_to_their_absolute_tolerance(refs):
    """f = N / (c E) of the FP32 path to 1e-6 absolute: a change of N_xx that moves f_xx by 2e-6 fails, even
    where N_xx itself stays within its relative tolerance; 0.5e-6 passes."""
    r, c = refs[0]["fp32"], refs[1]
    E, N = np.asarray(r["E"]), np.asarray(r["Nxx"])
    f = N / (c * E)
    g, i = cell_where((f > 0.2) & (E > 1e-20 * E.max()), E)
    for df, fails in ((0.5e-6, False), (2e-6, True)):
        got = copy_of(r)
        got["Nxx"][g, i] = N[g, i] + df * c * E[g, i]
        assert df / f[g, i] < parity.TOL["fp32"]           # the moment alone passes its own check
        check = failing_check(got, r, "fp32", c)
        assert check == ("fxx" if fails else None), (df, check)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_carried_state_check(refs, prec):
    """parity.check_state: the carried segment averages are held per segment, direction and group to the bound of
    the path's state (plus the FP64 roundings of the absolute values); one value beyond it fails."""
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(seed=0)
    geom = oracle.Geometry.from_workload(wl)
    r = parity.reference(geom, d, prec, wl.n_polar, want_I=True)
    Bseg = d["B"].T[oracle.tracks(geom, "double")["cell"]]
    dev, err = np.asarray(r["I"]), np.asarray(r["I_err"])
    exact = dev + Bseg
    assert parity.check_state(exact, dev, Bseg, err, prec)["state_bound_use"] <= 1.0
    allow = err + 4 * parity.U64 * np.abs(exact)
    s, g = np.unravel_index(np.argmax(allow), allow.shape)
    for factor, fails in ((0.5, False), (2.0, True)):
        got = exact.copy()
        got[s, g] += factor * allow[s, g]
        try:
            parity.check_state(got, dev, Bseg, err, prec)
            failed = False
        except AssertionError:
            failed = True
        assert failed is fails, factor
