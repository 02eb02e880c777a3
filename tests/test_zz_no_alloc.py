"""GPU: molc_sweep_static_scratch, the allocation-free variant of molc_sweep, against molc_sweep.

Collected last (file name) so that it also runs after every other GPU test in the same process; it must pass
alone in a fresh process as well.  Both entry points run the same kernels on the same inputs, so the carried
intensity states must agree bit for bit; the moments differ only by the order of the FP64 atomic additions.
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


def assert_moments_close(a, b, c):
    """Same arithmetic up to the summation order of the FP64 reductions: 1e-12 relative on the positive
    moments (floor 1e-30 max|x|), 1e-12 of c E on the signed ones."""
    a = {k: v.cpu().numpy() for k, v in a.items()}
    b = {k: v.cpu().numpy() for k, v in b.items()}
    cE = c * np.abs(b["E"])
    for k in ("E", "Nxx", "Nyy"):
        den = np.maximum(np.abs(b[k]), 1e-30 * np.abs(b[k]).max())
        assert np.max(np.abs(a[k] - b[k]) / den) <= 1e-12, k
    for k in ("Fx", "Fy", "Nxy"):
        den = np.maximum(cE, 1e-30 * cE.max())
        assert np.max(np.abs(a[k] - b[k]) / den) <= 1e-12, k


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_matches_sweep_two_calls_in_a_row(molc, prec):
    wl = synth.WORKLOADS["fc64_g17_d128"]      # 64^2 x 17 groups: 3.3 MB (FP64) / 1.4 MB (FP32) of workspace
    d = wl.inputs(2)
    P = molc.Plan.from_workload(wl)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I_ref = P.new_intensity(prec).zero_()     # zeroed so the padding bytes compare equal too
    I_new = P.new_intensity(prec).zero_()
    P.intensity_init(prec, I_ref, B)
    P.intensity_init(prec, I_new, B)
    out_new = P.new_moments(k.device)
    for _ in range(2):
        ref = P.sweep(prec, k, B, d["c"], d["dt"], I_ref, bnd)
        got = P.sweep_static_scratch(prec, k, B, d["c"], d["dt"], I_new, bnd, out=out_new)
        torch.cuda.synchronize()
        assert_moments_close(got, ref, d["c"])
        assert torch.equal(I_new, I_ref)      # carried state: identical bytes
    assert P.device_status() == 0
    P.close()


def test_static_scratch_rejects_plans_beyond_its_size(molc):
    # 256^2 cells x 17 groups needs 53 MB of FP64 workspace, more than the 16 MiB array: rejected on the host
    wl = synth.Workload("big", 256, 256, 6.0, 17, 0.001, 100.0, 2, 8, 2, 1)
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp64")
    P.intensity_init("fp64", I, B)
    with pytest.raises(molc.MolcError) as e:
        P.sweep_static_scratch("fp64", dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"]))
    assert e.value.code == 1 and "static scratch" in str(e.value)
    assert P.device_status() == 0
    P.close()
