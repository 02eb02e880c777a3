"""GPU: the tiled FP32 sweep (MOLC_TILED) against the default bundle FP32 sweep.

Both evaluate every segment update of Eqs. 11-13 with the same FP32 operations in the same order along each
characteristic, so the carried state (exported as canonical segment averages) must agree bit for bit over several
steps.  Their moment sums differ in order (the FP32 runs of one azimuth pair cover both senses in the moment gather
and one quadrant's sense in the tiled sweep), so the moments of each are held to the binary128 oracle through the
parity gate instead.
"""
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
    tiled, ti = run(molc, wl, d, 3, tiled=True)
    bundle, bi = run(molc, wl, d, 3)
    assert ti.fp32_tile_items > 0 and bi.fp32_tile_items == 0
    geom = oracle.Geometry.from_workload(wl)
    groups = list(range(wl.G)) if wl.G <= 4 else [0, 8, 16]
    dev_, err = None, None
    for (mt, It), (mb, Ib) in zip(tiled, bundle):
        assert np.array_equal(It, Ib)
        ref = parity.reference(geom, d, "fp32", wl.n_polar, groups=groups, I_prev=dev_, I_err=err, want_I=True)
        dev_, err = ref["I"], ref["I_err"]
        for m in (mt, mb):
            fm = {k: float(np.abs(v).max()) for k, v in m.items()}
            parity.compare({k: v[groups] for k, v in m.items()}, ref, "fp32", d["c"], floor_max=fm)
