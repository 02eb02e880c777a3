"""GPU: full-size parity on sampled groups, closure, state export/import, symmetry, device status."""
import math

import numpy as np
import pytest

import oracle
import parity
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def molc():
    import paper_2305_11998_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def host(d):
    return {k: v.cpu().numpy() for k, v in d.items()}


def test_full_size_512_sampled_groups(molc):
    """The production workload (512^2, 17 groups, 128 directions, h/2, three fronts) in the launch
    configuration the benchmark times; the group holding the Planck peak of the hot region checked against the
    binary128 oracle (the floor of the relative metric is taken over all groups of the GPU output)."""
    wl = synth.WORKLOADS["fc512_g17_d128"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    got = host(P.sweep("fp32", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"])))
    assert P.device_status() == 0
    n_upd = P.info.n_updates
    P.close()
    del I
    torch.cuda.empty_cache()
    assert n_upd > 1.4e9
    groups = [11]     # the Planck peak of the hot region
    geom = oracle.Geometry.from_workload(wl)
    ref = parity.reference(geom, d, "fp32", wl.n_polar, groups=groups)
    fm = {k: float(np.abs(v).max()) for k, v in got.items()}
    parity.compare({k: v[groups] for k, v in got.items()}, ref, "fp32", d["c"], floor_max=fm)


def test_full_size_512_fp64_sampled_group(molc):
    """The plain FP64 sweep (the speed-up denominator of the benchmark) at the production size in the launch
    configuration the benchmark times, the group holding the Planck peak of the hot region against the binary128
    oracle at the FP64 tolerance."""
    wl = synth.WORKLOADS["fc512_g17_d128"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp64")
    P.intensity_init("fp64", I, B)
    got = host(P.sweep("fp64", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"])))
    assert P.device_status() == 0
    P.close()
    del I
    torch.cuda.empty_cache()
    groups = [11]
    ref = parity.reference(oracle.Geometry.from_workload(wl), d, "fp64", wl.n_polar, groups=groups)
    fm = {k: float(np.abs(v).max()) for k, v in got.items()}
    parity.compare({k: v[groups] for k, v in got.items()}, ref, "fp64", d["c"], floor_max=fm)


def test_closure_and_grey_average(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(3)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp64")
    P.intensity_init("fp64", I, B)
    m = P.sweep("fp64", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"]))
    f = P.closure(m, d["c"], grey=True)
    mh = host(m)
    cE = d["c"] * mh["E"]
    for k, n in (("fxx", "Nxx"), ("fxy", "Nxy"), ("fyy", "Nyy")):
        assert np.allclose(f[k].cpu().numpy(), mh[n] / cE, rtol=1e-15, atol=0)
    g = f["grey"].cpu().numpy()
    # <f>_E = sum_g f_g E_g / sum_g E_g   (Eq. 8), the oracle's average of the same moments
    ref = oracle.grey_eddington(mh["E"], mh["Nxx"], mh["Nxy"], mh["Nyy"], d["c"])
    for i in range(3):
        assert np.allclose(g[i], ref[i], rtol=1e-13, atol=1e-16)
    # trace bound of the closure
    fx, fy = f["fxx"].cpu().numpy(), f["fyy"].cpu().numpy()
    assert np.all((fx >= 0) & (fy >= 0) & (fx + fy <= 1 + 1e-12))
    P.close()


def test_grey_coefficients_against_their_definition(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(2)
    P = molc.Plan.from_workload(wl)
    k, B = dev(d["kappa"]), dev(d["B"])
    I = P.new_intensity("fp64")
    P.intensity_init("fp64", I, B)
    m = P.sweep("fp64", k, B, d["c"], d["dt"], I, dev(d["bnd"]))
    got = {kk: v.cpu().numpy() for kk, v in P.grey_coefficients(m, k, B).items()}
    mh = host(m)
    ref = oracle.grey_coefficients(mh["E"], mh["Fx"], mh["Fy"], d["kappa"], d["B"])
    for kk in ("kappa_E", "kappa_B", "KRx", "KRy"):
        assert np.allclose(got[kk], ref[kk], rtol=1e-13, atol=0), kk
    scale = np.max(np.abs(d["kappa"])) * (np.abs(mh["Fx"]) + np.abs(mh["Fy"])).sum(0) / mh["E"].sum(0)
    for kk in ("eta_x", "eta_y"):
        assert np.all(np.abs(got[kk] - ref[kk]) <= 1e-13 * scale), kk
    P.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_export_import_roundtrip(molc, prec):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity(prec)
    rng = np.random.default_rng(0)
    canon = rng.uniform(0.0, 1.0, (P.info.n_segments, wl.G)) * d["B"].max()
    P.intensity_init(prec, I, B)
    P.intensity_import(prec, I, dev(canon), B)
    back = P.intensity_export(prec, I).cpu().numpy()
    tol = 1e-15 if prec == "fp64" else 2e-7
    assert np.max(np.abs(back - canon)) <= tol * np.abs(canon).max()
    # a partial group range leaves the others alone
    before = P.intensity_export(prec, I).cpu().numpy()
    P.intensity_import(prec, I, dev(np.zeros((P.info.n_segments, 1))), B, g_begin=2)
    after = P.intensity_export(prec, I).cpu().numpy()
    assert np.array_equal(after[:, [0, 1, 3]], before[:, [0, 1, 3]])
    # zero is stored as the deviation -B of the segment's cell: exact in FP64, within FP32 rounding of B
    Bseg = d["B"][2][P.tracks()["cell"]]
    floor = 1e-30 * d["B"].max()      # FP32 states resolve deviations down to ~1e-68 of max B
    assert np.all(np.abs(after[:, 2]) <= (0.0 if prec == "fp64" else 6e-8) * Bseg + (prec == "fp32") * floor)
    # a swept state imported into a fresh buffer gives the same next step
    k, bnd = dev(d["kappa"]), dev(d["bnd"])
    P.intensity_init(prec, I, B)
    P.sweep(prec, k, B, d["c"], d["dt"], I, bnd)
    snap = P.intensity_export(prec, I)
    J = P.new_intensity(prec)
    P.intensity_init(prec, J, B)
    P.intensity_import(prec, J, snap, B)
    a = host(P.sweep(prec, k, B, d["c"], d["dt"], I, bnd))
    b = host(P.sweep(prec, k, B, d["c"], d["dt"], J, bnd))
    # the canonical format holds segment averages, not deviations: the round trip is exact to rounding of
    # the averages, so the next step agrees to that on E and to it times c E on the signed moments
    tol = 1e-13 if prec == "fp64" else 2e-6
    cE = d["c"] * a["E"]
    for kk in ("E", "Nxx", "Nyy"):
        assert np.all(np.abs(a[kk] - b[kk]) <= tol * np.abs(a[kk]) + 1e-300), kk
    for kk in ("Fx", "Fy", "Nxy"):
        assert np.all(np.abs(a[kk] - b[kk]) <= tol * cE), kk
    P.close()


def test_fp32_state_scale_follows_the_intensities(molc):
    """The FP32 state works in units scaled by a power of two that follows max(B, boundary) step by step, so
    a run on 2^k B is exactly 2^k times the run on B, for any k, and a cold medium under a hot boundary (the
    boundary ~1e13 times the largest B) needs no range of its own."""
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)

    def run(fac, steps=2):
        B = dev(d["B"] * fac)
        I = P.new_intensity("fp32")
        P.intensity_init("fp32", I, B)
        for _ in range(steps):
            m = host(P.sweep("fp32", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"] * fac)))
        assert P.device_status() == 0
        return m

    m0 = run(1.0)
    for fac in (2.0 ** 30, 2.0 ** -200, 2.0 ** 150):
        m = run(fac)
        for k in m0:
            assert np.array_equal(m[k], m0[k] * fac), (fac, k)
    # a state initialised at one level and swept at another rescales itself (no range error)
    B = dev(d["B"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    m = host(P.sweep("fp32", dev(d["kappa"]), dev(d["B"] * 2.0 ** 40), d["c"], d["dt"], I, dev(d["bnd"] * 2.0 ** 40)))
    assert P.device_status() == 0 and all(np.isfinite(v).all() for v in m.values())
    P.close()
    # cold start under the hot left edge, against the binary128 oracle
    wc = synth.Workload("cold16", 16, 16, 6.0, 4, 0.01, 10.0, 2, 16, 2, 1, cold_start=True)
    dc = wc.inputs(0)
    assert dc["bnd"].max() > 1e10 * dc["B"].max()
    Pc = molc.Plan.from_workload(wc)
    Bc = dev(dc["B"])
    Ic = Pc.new_intensity("fp32")
    Pc.intensity_init("fp32", Ic, Bc)
    got = host(Pc.sweep("fp32", dev(dc["kappa"]), Bc, dc["c"], dc["dt"], Ic, dev(dc["bnd"])))
    assert Pc.device_status() == 0
    Pc.close()
    ref = parity.reference(oracle.Geometry.from_workload(wc), dc, "fp32", wc.n_polar)
    parity.compare(got, ref, "fp32", dc["c"])


def _rot(a, n):
    a = a.reshape(a.shape[:-1] + (n, n))
    out = np.empty_like(a)
    for iy in range(n):
        for ix in range(n):
            out[..., ix, n - 1 - iy] = a[..., iy, ix]
    return out.reshape(a.shape[:-2] + (n * n,))


def test_rotation_symmetry_on_gpu(molc):
    wl = synth.Workload("sym", 12, 12, 6.0, 3, 0.01, 10.0, 2, 16, 2, 1)
    d = wl.inputs(4)
    n = wl.nx
    P = molc.Plan.from_workload(wl)

    def step(kappa, B, bnd):
        Bd = dev(B)
        I = P.new_intensity("fp64")
        P.intensity_init("fp64", I, Bd)
        return host(P.sweep("fp64", dev(kappa), Bd, d["c"], d["dt"], I, dev(bnd)))

    base = step(d["kappa"], d["B"], d["bnd"])
    bnd_r = np.zeros_like(d["bnd"])
    bnd_r[synth.EDGE_BOTTOM] = d["bnd"][synth.EDGE_LEFT]
    rot = step(_rot(d["kappa"], n), _rot(d["B"], n), bnd_r)
    cE = _rot(d["c"] * base["E"], n)
    exp = {"E": base["E"], "Fx": -base["Fy"], "Fy": base["Fx"], "Nxx": base["Nyy"], "Nyy": base["Nxx"],
           "Nxy": -base["Nxy"]}
    for k, v in exp.items():
        assert np.max(np.abs(rot[k] - _rot(v, n)) / cE) < 1e-13, k
    P.close()


def test_device_status_flags_bad_inputs(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    bnd = dev(d["bnd"])
    for prec in ("fp64", "fp32"):
        I = P.new_intensity(prec)
        P.intensity_init(prec, I, B)
        P.sweep(prec, dev(d["kappa"]), B, d["c"], d["dt"], I, bnd)
        assert P.device_status() == 0
        bad = d["kappa"].copy()
        bad[1, 17] = np.nan
        P.sweep(prec, dev(bad), B, d["c"], d["dt"], I, bnd)
        assert P.device_status() == 4
        assert P.device_status() == 0          # reading clears it
        badB = d["B"].copy()
        badB[0, 3] = -1.0
        P.sweep(prec, dev(d["kappa"]), dev(badB), d["c"], d["dt"], I, bnd)
        assert P.device_status() == 4
        badb = d["bnd"].copy()
        badb[2, 1] = np.inf
        P.sweep(prec, dev(d["kappa"]), B, d["c"], d["dt"], I, dev(badb))
        assert P.device_status() == 4
    with pytest.raises(molc.MolcError) as e:
        P.sweep("fp32", dev(d["kappa"]), B, -1.0, d["dt"], I, bnd)
    assert e.value.code == 1
    P.close()


def test_kernel_timing_hook(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    P.kernel_timing(True)
    for _ in range(3):
        P.sweep("fp32", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"]))
    ms, n = P.kernel_time()
    assert n == 3 and ms > 0
    P.kernel_timing(False)
    P.sweep("fp32", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"]))
    assert P.kernel_time() == (0.0, 0)
    P.close()


def test_binding_rejects_tensors_of_the_wrong_size_or_type(molc):
    # checked on the host before any launch: no kernel ever sees a buffer shorter than the plan needs
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    with pytest.raises(ValueError):
        P.sweep("fp32", k[:-1], B, d["c"], d["dt"], I, bnd)                   # kappa one group short
    with pytest.raises(ValueError):
        P.sweep("fp32", k.float(), B, d["c"], d["dt"], I, bnd)               # FP32 inputs
    with pytest.raises(ValueError):
        P.sweep("fp32", k, B, d["c"], d["dt"], I, bnd[:, :1])                # boundary of one group
    with pytest.raises(ValueError):
        P.sweep("fp64", k, B, d["c"], d["dt"], I, bnd)                       # an FP32 state as FP64
    out = P.new_moments()
    out["Fy"] = out["Fy"][:1]
    with pytest.raises(ValueError):
        P.sweep("fp32", k, B, d["c"], d["dt"], I, bnd, out=out)              # a short moment array
    torch.cuda.synchronize()
    assert P.device_status() == 0
    P.close()
