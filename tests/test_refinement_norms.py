"""Host logic: the mesh-refinement norms of Sec. 5 (||dy_h|| = ||y_h - y_2h||_L2, rho_h = ||dy_2h|| / ||dy_h||)."""
import numpy as np
import pytest

pytest.importorskip("torch")
from paper_2305_11998_gb300.multistep import refinement_norms  # noqa: E402


def test_rate_of_a_power_law_sequence():
    # y_h = y* + C h^p on halved spacings: every difference shrinks by 2^p, so rho = 2^p exactly
    rng = np.random.default_rng(0)
    ystar, C = rng.random(50), rng.random(50) + 0.5
    for p in (1, 2, 3):
        ys = [ystar + C * (1.0 / 2 ** k) ** p for k in range(1, 5)]
        r = refinement_norms(ys, 0.25)
        assert r[0] == {"norm": None, "rho": None} and r[1]["rho"] is None
        for k in (2, 3):
            assert r[k]["rho"] == pytest.approx(2.0 ** p, rel=1e-12)


def test_norm_is_the_volume_weighted_l2_difference():
    a, b = np.array([1.0, 2.0, 3.0]), np.array([1.0, 4.0, 1.0])
    r = refinement_norms([a, b], 0.5)
    assert r[1]["norm"] == pytest.approx(np.sqrt(0.5 * (4.0 + 4.0)), rel=1e-15)


def test_identical_solutions_give_zero_norm_and_no_rate():
    y = np.ones(4)
    r = refinement_norms([y, y, y], 1.0)
    assert r[1]["norm"] == 0.0 and r[2]["norm"] == 0.0 and r[2]["rho"] is None
