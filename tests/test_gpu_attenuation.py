"""GPU: the segment attenuation (Eqs. 12-13) over tau from below 1e-9 to above 1e3, through the C ABI.

One cell, cold (B = 0 and I^{n-1} = 0, so Q = 0), every edge driven at I_in = 1.  Every segment then starts from
I_in and its average is Ibar = alpha I_in + (1 - alpha) I_in e^-tau = I_in (1 - e^-tau)/tau = I_in E1(tau), with
tau = kappa~ l / sin zeta (Eq. 13; l the in-plane length from the track export, zeta the direction's polar
angle).  Groups carry kappa log-spaced over twelve decades, so the segments cover both branches of the FP32
E1 (the even series below tau = 1/2, (1 - e^-tau)/tau above) and the FP64 path's expm1.  The reference is
-expm1(-tau)/tau in FP64 on the host.

FP32 bound: tau is formed from FP32 kappa~, l and 1/(2 sin zeta) (a few u of relative error, which moves E1 by
at most as much since |d ln E1 / d ln tau| <= 1), e^-tau/2 by ex2.approx (~2^-22 relative), and 1 - e^-tau
loses up to e^-tau / (1 - e^-tau) < 1.6x of that above tau = 1/2: ~1.5e-6 in all; the test allows 8e-6.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

C_LIGHT = 29.98
DT = 1.0e15            # 1/(c dt) ~ 3e-17 cm^-1: kappa~ = kappa to far below the smallest kappa


@pytest.fixture(scope="module")
def molc():
    import paper_2305_11998_gb300 as m
    m.load()
    return m


@pytest.mark.parametrize("prec,tol", [("fp32", 8e-6), ("fp64", 1e-14)])
def test_segment_average_is_E1_over_twelve_decades_of_tau(molc, prec, tol):
    mu, cphi, sphi, w = molc.quadrature_product(2, 8)
    G = 25
    kappa = np.logspace(-9, 3, G)
    P = molc.Plan(1, 1, 1.0, 1.0, mu, cphi, sphi, w, G, 0.05)
    dev = dict(device="cuda", dtype=torch.float64)
    k = torch.tensor(kappa[:, None], **dev)
    B = torch.zeros((G, 1), **dev)
    bnd = torch.ones((4, G), **dev)
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    P.sweep(prec, k, B, C_LIGHT, DT, I, bnd)
    got = P.intensity_export(prec, I).cpu().numpy()          # [segment][group]
    assert P.device_status() == 0
    tr = P.tracks()
    # the polar sine of every segment's direction (direction-major canonical order)
    sinz = np.sqrt(1.0 - mu ** 2)
    seg_dir = np.zeros(tr["len"].size, dtype=np.int64)
    for m in range(P.info.n_dir):
        r0, r1 = tr["dir_ray_off"][m], tr["dir_ray_off"][m + 1]
        seg_dir[tr["ray_seg_off"][r0]:tr["ray_seg_off"][r1]] = m
    kt = kappa + 1.0 / (C_LIGHT * DT)
    tau = kt[None, :] * (tr["len"] / sinz[seg_dir])[:, None]
    ref = -np.expm1(-tau) / tau
    assert tau.min() < 1e-9 and tau.max() > 1e3
    assert np.any(tau < 0.5) and np.any(tau > 0.5)
    err = np.abs(got - ref) / ref
    assert err.max() <= tol, (float(err.max()), float(tau.flat[np.argmax(err)]))
    P.close()


@pytest.mark.parametrize("prec,tol", [("fp32", 8e-6), ("fp64", 1e-14)])
def test_hand_worked_characteristic(molc, prec, tol):
    # the characteristic of tests/golden/single_ray_3x3.txt (cells and lengths worked out by hand): the library's
    # grid reproduces it and, with Q = 0, its segment averages are I_in,s (1 - e^-tau_s) / tau_s
    import math
    import os
    rows = [ln.split() for ln in open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                                   "single_ray_3x3.txt")) if ln.strip() and not ln.startswith("#")]
    direction, ray, edge = (int(x) for x in rows[0])
    cells = [int(r[0]) for r in rows[1:]]
    lens = [float(r[1]) * math.sqrt(2.0) for r in rows[1:]]
    mu, cphi, sphi, w = molc.quadrature_product(1, 4)
    P = molc.Plan(3, 3, 3.0, 3.0, mu, cphi, sphi, w, 1, 3.0 * math.sqrt(2.0) / 4.0)
    tr = P.tracks()
    rg = tr["dir_ray_off"][direction] + ray
    s0, s1 = tr["ray_seg_off"][rg], tr["ray_seg_off"][rg + 1]
    assert tr["entry"][rg] == edge and tr["cell"][s0:s1].tolist() == cells
    assert np.allclose(tr["len"][s0:s1], lens, rtol=0, atol=1e-14)
    dev = dict(device="cuda", dtype=torch.float64)
    kappa = 0.3 + 0.7 * np.arange(9, dtype=float)
    k = torch.tensor(kappa[None, :], **dev)
    B = torch.zeros((1, 9), **dev)
    bnd = torch.zeros((4, 1), **dev)
    bnd[edge] = 1.0
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    P.sweep(prec, k, B, C_LIGHT, DT, I, bnd)
    got = P.intensity_export(prec, I).cpu().numpy()[s0:s1, 0]
    sinz = math.sqrt(3.0) / 2.0
    Iin = 1.0
    for j, (cell, ln) in enumerate(zip(cells, lens)):
        tau = (kappa[cell] + 1.0 / (C_LIGHT * DT)) * ln / sinz
        ref = Iin * (-math.expm1(-tau)) / tau
        assert abs(got[j] - ref) <= tol * ref, (j, got[j], ref)
        Iin *= math.exp(-tau)
    assert P.device_status() == 0
    P.close()
