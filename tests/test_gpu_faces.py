"""GPU: face-average moments of Eq. 16 (plans created with MOLC_FACES) against the binary128 oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 2e-5}


@pytest.fixture(scope="module")
def molc():
    import paper_2305_11998_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


CASES = [
    dict(name="fc16", layout="uniform"),
    dict(name="rect_paper", layout="paper"),
]


def case_inputs(case):
    if case["name"] == "fc16":
        wl = synth.WORKLOADS["fc16_g4_d32"]
        d = wl.inputs(1)
        q = wl.quadrature()
        return wl, d, q, wl.L, wl.L, wl.spacing
    # rectangular cells, three polar cosines, the paper's vertex-band layout
    rng = np.random.default_rng(3)
    nx, ny, G = 6, 4, 3
    q = synth.product_quadrature(3, 8)
    wl = synth.Workload("rect", nx, ny, 3.0, G, 0.01, 10.0, 3, 8, 2, 1)
    d = dict(kappa=np.exp(rng.uniform(np.log(1e-2), np.log(1e3), (G, nx * ny))),
             B=np.exp(rng.uniform(np.log(1e-6), 0.0, (G, nx * ny))), bnd=rng.uniform(0, 1, (4, G)), c=1.0, dt=0.3)
    return wl, d, q, 3.0, 1.0, 0.2


@pytest.mark.parametrize("ci", range(len(CASES)))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_face_moments_against_binary128(molc, prec, ci):
    case = CASES[ci]
    wl, d, q, lx, ly, sp = case_inputs(case)
    renorm = case["layout"] == "uniform"
    P = molc.Plan(wl.nx, wl.ny, lx, ly, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, sp, case["layout"], renorm,
                  faces=True)
    nf = (wl.nx + 1) * wl.ny + wl.nx * (wl.ny + 1)
    assert P.info.n_faces == nf
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    got = []
    for _ in range(2):
        P.sweep(prec, k, B, d["c"], d["dt"], I, bnd)
        got.append({kk: v.cpu().numpy() for kk, v in P.face_moments(prec, I, d["c"]).items()})
    assert P.device_status() == 0
    geom = oracle.Geometry(wl.nx, wl.ny, lx, ly, q.mu, q.cos_phi, q.sin_phi, q.w, sp,
                           0 if case["layout"] == "uniform" else 1, int(renorm))
    Iq = None
    tol = TOL[prec]
    for step in range(2):
        r = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], I_prev=Iq, precision="quad",
                         I_as_deviation=True, I_prev_is_deviation=True, want_faces=True)
        Iq = r["I"]
        g = got[step]
        E = r["face_E"]
        floor = 1e-30 * np.abs(E).max()
        for kk in ("E", "Nxx", "Nyy"):
            ref = r["face_" + kk]
            den = np.maximum(np.abs(ref), 1e-30 * np.abs(ref).max())
            assert np.max(np.abs(g[kk] - ref) / den) <= tol, (prec, step, kk)
        cE = np.maximum(d["c"] * np.abs(E), d["c"] * floor)
        for kk in ("Fx", "Fy", "Nxy"):
            assert np.max(np.abs(g[kk] - r["face_" + kk]) / cE) <= tol, (prec, step, kk)
    P.close()


def test_face_moments_need_the_flag(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, dev(d["B"]))
    with pytest.raises(molc.MolcError):
        P.face_moments("fp32", I, d["c"])
    Pf = molc.Plan.from_workload(wl, faces=True)
    with pytest.raises(molc.MolcError):
        molc.Batch([Pf])           # batched sweeps produce no face moments
    P.close()
    Pf.close()
