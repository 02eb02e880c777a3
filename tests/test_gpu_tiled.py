"""GPU: the tiled FP32 sweep against the bundle FP32 sweep (plans created with MOLC_BALANCE keep the bundle sweep).

Both evaluate every segment update of Eqs. 11-13 with the same FP32 operations in the same order along each
characteristic, so the carried state (exported as canonical segment averages) must agree bit for bit over several
steps; only the order of the moment sums differs (per-quadrant partials in the tiled sweep), so the moments agree
to the FP64-class accuracy of those sums.
"""
import numpy as np
import pytest

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


def run(molc, wl, d, steps, **kw):
    P = molc.Plan.from_workload(wl, **kw)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    res = []
    for _ in range(steps):
        m = P.sweep("fp32", k, B, d["c"], d["dt"], I, bnd)
        res.append(({kk: v.cpu().numpy() for kk, v in m.items()}, P.intensity_export("fp32", I).cpu().numpy()))
    assert P.device_status() == 0
    info = P.info
    P.close()
    return res, info


@pytest.mark.parametrize("name", ["fc16_g4_d32", "fc64_g17_d128"])
def test_tiled_state_matches_bundle_sweep_bit_for_bit(molc, name):
    wl = synth.WORKLOADS[name]
    d = wl.inputs(4)
    tiled, ti = run(molc, wl, d, 3)
    bundle, bi = run(molc, wl, d, 3, balance=True)
    assert ti.fp32_tile_items > 0 and bi.fp32_tile_items == 0
    for (mt, It), (mb, Ib) in zip(tiled, bundle):
        assert np.array_equal(It, Ib)
        cE = d["c"] * np.abs(mb["E"])
        for k in ("E", "Nxx", "Nyy"):
            assert np.max(np.abs(mt[k] - mb[k]) / np.maximum(np.abs(mb[k]), 1e-300)) < 1e-12, k
        for k in ("Fx", "Fy", "Nxy"):
            assert np.max(np.abs(mt[k] - mb[k]) / np.maximum(cE, 1e-300)) < 1e-12, k
