"""GPU parity: the CUDA sweeps (through the C ABI) against the binary128 oracle on the same seeded inputs.

FP64 path: relative 1e-12.  FP32 path: relative 2e-5 on E and F, 1e-6 absolute on the Eddington factors.  The
signed moments are held to the literal metric where the path's arithmetic resolves them and to the oracle's
derived bound of that arithmetic elsewhere (tests/parity.py); the carried state per segment to that bound too.
Large cases are compared on sampled groups (the groups of a sweep are independent).
"""
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


def run_gpu(molc, wl, d, prec, steps=1, quad=None, layout="uniform", renorm=True, spacing=None, export=False):
    P = molc.Plan.from_workload(wl, quad=quad, layout=layout, renorm=renorm, spacing=spacing)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    outs, Is = [], []
    for _ in range(steps):
        outs.append(host(P.sweep(prec, k, B, d["c"], d["dt"], I, bnd)))
        if export:
            Is.append(P.intensity_export(prec, I).cpu().numpy())
    assert P.device_status() == 0
    P.close()
    return outs, Is


def run_oracle(wl, d, prec, steps=1, quad=None, layout=0, renorm=1, spacing=None, want_I=False, groups=None):
    """The binary128 oracle with the error model of path `prec` over `steps` steps; between steps it carries
    its state as deviations from B (fixed B here) and the bound of the path's state.  Returns the results
    (moments, bounds, state) per step."""
    geom = oracle.Geometry.from_workload(wl, quad=quad, layout=layout, renorm=renorm, spacing=spacing)
    outs = []
    dev = err = None
    for _ in range(steps):
        r = parity.reference(geom, d, prec, wl.n_polar, groups=groups, I_prev=dev, I_err=err,
                             want_I=(steps > 1 or want_I))
        dev, err = r.get("I"), r.get("I_err")
        outs.append(r)
    return outs


C0 = synth.WORKLOADS["fc16_g4_d32"]


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_one_step_vs_binary128(molc, prec, seed):
    d = C0.inputs(seed)
    got, gI = run_gpu(molc, C0, d, prec, export=True)
    ref = run_oracle(C0, d, prec, want_I=True)
    parity.compare(got[0], ref[0], prec, d["c"])
    # carried state, per segment, direction and group, within the bound of the path's state
    Bseg = d["B"][:, oracle.tracks(oracle.Geometry.from_workload(C0), "double")["cell"]].T
    parity.check_state(gI[0], ref[0]["I"], Bseg, ref[0]["I_err"], prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_multistep_vs_binary128(molc, prec):
    d = C0.inputs(7)
    got, gI = run_gpu(molc, C0, d, prec, steps=4, export=True)
    ref = run_oracle(C0, d, prec, steps=4)
    Bseg = d["B"][:, oracle.tracks(oracle.Geometry.from_workload(C0), "double")["cell"]].T
    for g_, gi_, r_ in zip(got, gI, ref):
        parity.compare(g_, r_, prec, d["c"])
        parity.check_state(gi_, r_["I"], Bseg, r_["I_err"], prec)


def test_fp32_ten_steps_64x64_sampled_groups(molc):
    """The 64^2 workload: 64^2 cells, 17 groups, 4 x 32 directions, h/4, ten steps with the state carried; the
    GPU sweeps all groups, three are followed by the binary128 oracle with the carried state bound."""
    wl = synth.WORKLOADS["fc64_g17_d128"]
    d = wl.inputs(0)
    got, _ = run_gpu(molc, wl, d, "fp32", steps=wl.steps)
    groups = [0, 8, 16]
    ref = run_oracle(wl, d, "fp32", steps=wl.steps, groups=groups)
    for g_, r_ in zip(got, ref):
        fm = {k: float(np.abs(v).max()) for k, v in g_.items()}
        parity.compare({k: v[groups] for k, v in g_.items()}, r_, "fp32", d["c"], floor_max=fm)


def test_fp64_64x64_sampled_groups_vs_binary128(molc):
    wl = synth.WORKLOADS["fc64_g17_d128"]
    d = wl.inputs(1)
    got, _ = run_gpu(molc, wl, d, "fp64")
    groups = [0, 8, 11, 16]
    ref = run_oracle(wl, d, "fp64", groups=groups)
    fm = {k: float(np.abs(v).max()) for k, v in got[0].items()}
    parity.compare({k: v[groups] for k, v in got[0].items()}, ref[0], "fp64", d["c"], floor_max=fm)


# Varied shapes: rectangular cells, G = 1, odd polar counts (every FP32 template), the paper's layout,
# no renormalisation, near-vacuum and very thick media.
VARIANTS = [
    dict(nx=1, ny=1, G=1, npol=1, naz=4, div=3),
    dict(nx=7, ny=3, G=5, npol=3, naz=8, div=2, L=(3.0, 1.0)),
    dict(nx=5, ny=9, G=2, npol=5, naz=12, div=3),
    dict(nx=6, ny=6, G=3, npol=6, naz=8, div=2, layout="paper"),
    dict(nx=8, ny=5, G=4, npol=7, naz=4, div=2, renorm=False),
    dict(nx=4, ny=4, G=17, npol=8, naz=16, div=4),
    dict(nx=10, ny=10, G=2, npol=2, naz=20, div=1, thick=True),
    dict(nx=10, ny=10, G=2, npol=4, naz=8, div=2, thin=True),
    dict(nx=3, ny=4, G=37, npol=2, naz=8, div=2),          # FP32: two group chunks, the last one partial
]


def variant_inputs(v, seed=0):
    rng = np.random.default_rng(seed)
    nx, ny = v["nx"], v["ny"]
    Lx, Ly = v.get("L", (2.0, 2.0))
    q = synth.product_quadrature(v["npol"], v["naz"])
    G = v["G"]
    if v.get("thick"):
        kappa = rng.uniform(1e4, 1e7, (G, nx * ny))
    elif v.get("thin"):
        kappa = rng.uniform(0.0, 1e-3, (G, nx * ny))
    else:
        kappa = np.exp(rng.uniform(np.log(1e-2), np.log(1e3), (G, nx * ny)))
    B = np.exp(rng.uniform(np.log(1e-6), 0.0, (G, nx * ny)))
    bnd = rng.uniform(0, 1, (4, G))
    wl = synth.Workload("var", nx, ny, Lx, G, 0.01, 10.0, v["npol"], v["naz"], v["div"], 1)
    wl.L = Lx
    h = min(Lx / nx, Ly / ny)
    return wl, q, dict(kappa=kappa, B=B, bnd=bnd, c=1.0, dt=0.3), Ly, h / v["div"]


@pytest.mark.parametrize("vi", range(len(VARIANTS)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_variants_vs_binary128(molc, prec, vi):
    v = VARIANTS[vi]
    wl, q, d, Ly, sp = variant_inputs(v, vi)
    layout = v.get("layout", "uniform")
    renorm = v.get("renorm", layout == "uniform")
    P = molc.Plan(v["nx"], v["ny"], wl.L, Ly, q.mu, q.cos_phi, q.sin_phi, q.w, v["G"], sp, layout, renorm)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    res = []
    for _ in range(2):
        res.append(host(P.sweep(prec, k, B, d["c"], d["dt"], I, bnd)))
    assert P.device_status() == 0
    P.close()
    geom = oracle.Geometry(v["nx"], v["ny"], wl.L, Ly, q.mu, q.cos_phi, q.sin_phi, q.w, sp,
                           0 if layout == "uniform" else 1, int(renorm))
    Iq = Ie = None
    for step in range(2):
        r = parity.reference(geom, d, prec, v["npol"], I_prev=Iq, I_err=Ie, want_I=True)
        Iq, Ie = r["I"], r["I_err"]
        parity.compare(res[step], r, prec, d["c"])


def test_equilibrium_on_gpu(molc):
    # homogeneous medium, I^{n-1} = B, every edge at B: E = 4 pi B / c, F = 0, f = 1/3 (exact)
    q = synth.product_quadrature(4, 16)
    nx = ny = 12
    P = molc.Plan(nx, ny, 3.0, 3.0, q.mu, q.cos_phi, q.sin_phi, q.w, 3, 0.1)
    Bv = np.array([1.0, 1e-3, 5e-8])
    kap = np.array([0.5, 50.0, 5e5])
    B = dev(np.repeat(Bv[:, None], nx * ny, 1))
    k = dev(np.repeat(kap[:, None], nx * ny, 1))
    bnd = dev(np.repeat(Bv[None, :], 4, 0))
    c = 29.98
    for prec, tol in (("fp64", 1e-14), ("fp32", 1e-7)):
        I = P.new_intensity(prec)
        P.intensity_init(prec, I, B)
        for _ in range(2):
            m = host(P.sweep(prec, k, B, c, 2e-3, I, bnd))
        cE = c * m["E"]
        assert np.max(np.abs(cE / (4 * math.pi * Bv[:, None]) - 1)) < tol
        assert np.max(np.abs(m["Fx"]) / cE) < tol and np.max(np.abs(m["Fy"]) / cE) < tol
        f = P.closure({kk: dev(vv) for kk, vv in m.items()}, c, grey=True)
        for kk in ("fxx", "fyy"):
            assert np.max(np.abs(f[kk].cpu().numpy() - 1 / 3)) < tol
        assert np.max(np.abs(f["fxy"].cpu().numpy())) < tol
        assert np.max(np.abs(f["grey"].cpu().numpy()[[0, 2]] - 1 / 3)) < tol
    P.close()
