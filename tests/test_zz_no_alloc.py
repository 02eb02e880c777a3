"""GPU: molc_sweep_static_scratch, the allocation-free variant of molc_sweep, against molc_sweep.

Collected last (file name) so that it also runs after every other GPU test in the same process; it must pass
alone in a fresh process as well.  Both entry points run the same kernels on the same inputs, so the carried
intensity states must agree bit for bit; the moments differ at most by the order of FP64 additions (the FP64
path's atomics; the FP32 sweep's sums are deterministic).  After the
first call (which looks the array up), further calls must leave the device's free memory unchanged.
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


def assert_moments_close(a, b, c, E=None):
    """Same arithmetic up to the summation order of the FP64 reductions: 1e-12 relative on the positive
    moments (floor 1e-30 max|x|), 1e-12 of c E on the signed ones."""
    a = {k: v.cpu().numpy() for k, v in a.items()}
    b = {k: v.cpu().numpy() for k, v in b.items()}
    cE = c * np.abs(b["E"] if E is None else E)
    for k in ("E", "Nxx", "Nyy"):
        den = np.maximum(np.abs(b[k]), 1e-30 * np.abs(b[k]).max())
        assert np.max(np.abs(a[k] - b[k]) / den) <= 1e-12, k
    for k in ("Fx", "Fy", "Nxy"):
        den = np.maximum(cE, 1e-30 * cE.max())
        assert np.max(np.abs(a[k] - b[k]) / den) <= 1e-12, k


def free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


@pytest.mark.parametrize("prec,tiled", [("fp64", False), ("fp32", False), ("fp32", True)])
def test_static_scratch_matches_sweep_two_calls_in_a_row(molc, prec, tiled):
    wl = synth.WORKLOADS["fc64_g17_d128"]      # 64^2 x 17 groups: within the array's size
    d = wl.inputs(2)
    P = molc.Plan.from_workload(wl, tiled=tiled)
    assert (P.info.fp32_tile_items > 0) == tiled
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I_ref = P.new_intensity(prec).zero_()     # zeroed so the padding bytes compare equal too
    I_new = P.new_intensity(prec).zero_()
    P.intensity_init(prec, I_ref, B)
    P.intensity_init(prec, I_new, B)
    out_ref, out_new = P.new_moments(k.device), P.new_moments(k.device)
    for _ in range(2):
        P.sweep(prec, k, B, d["c"], d["dt"], I_ref, bnd, out=out_ref)
        P.sweep_static_scratch(prec, k, B, d["c"], d["dt"], I_new, bnd, out=out_new)
        torch.cuda.synchronize()
        assert_moments_close(out_new, out_ref, d["c"])
        assert torch.equal(I_new, I_ref)      # carried state: identical bytes
    # nothing is allocated by further calls: the device's free memory stays the same
    I_scr = I_new.clone()
    f0 = free_bytes()
    for _ in range(3):
        P.sweep_static_scratch(prec, k, B, d["c"], d["dt"], I_scr, bnd, out=out_new)
    assert free_bytes() == f0
    assert P.device_status() == 0
    P.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_face_moments(molc, prec):
    """A MOLC_FACES plan: the face accumulators are cleared by each call, so the face moments of Eq. 16 after the
    allocation-free call equal those after molc_sweep from the same state."""
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(1)
    P = molc.Plan.from_workload(wl, faces=True)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I_ref, I_new = P.new_intensity(prec).zero_(), P.new_intensity(prec).zero_()
    P.intensity_init(prec, I_ref, B)
    P.intensity_init(prec, I_new, B)
    for _ in range(2):
        ref = P.sweep(prec, k, B, d["c"], d["dt"], I_ref, bnd)
        fref = P.face_moments(prec, I_ref, d["c"])
        got = P.sweep_static_scratch(prec, k, B, d["c"], d["dt"], I_new, bnd)
        fgot = P.face_moments(prec, I_new, d["c"])
        torch.cuda.synchronize()
        assert_moments_close(got, ref, d["c"])
        assert_moments_close(fgot, fref, d["c"], E=fref["E"].cpu().numpy())
        assert torch.equal(I_new, I_ref)
    assert P.device_status() == 0
    P.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_static_scratch_ray_balance(molc, prec):
    """A MOLC_BALANCE plan: the allocation-free call adds its rays to the balance record with the floor of its
    own B and boundary, so on a fresh record it gives exactly the residual molc_sweep gives from the same state."""
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(3)
    P = molc.Plan.from_workload(wl, balance=True)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I_ref, I_new = P.new_intensity(prec).zero_(), P.new_intensity(prec).zero_()
    P.intensity_init(prec, I_ref, B)
    P.intensity_init(prec, I_new, B)
    got = P.sweep_static_scratch(prec, k, B, d["c"], d["dt"], I_new, bnd)   # first call: record starts at 0
    r_new = P.ray_balance()
    ref = P.sweep(prec, k, B, d["c"], d["dt"], I_ref, bnd)                  # starts a new record
    r_ref = P.ray_balance()
    assert_moments_close(got, ref, d["c"])
    assert torch.equal(I_new, I_ref)
    assert r_new == r_ref and 0 < r_ref < (1e-13 if prec == "fp64" else 4e-6)
    assert P.device_status() == 0
    P.close()


@pytest.mark.parametrize("prec,n,tiled", [("fp64", 384, False), ("fp32", 512, False), ("fp32", 224, True)])
def test_static_scratch_rejects_plans_beyond_its_size(molc, prec, n, tiled):
    # FP64: 384^2 cells x 17 groups need 120 MB of accumulators; FP32: 512^2 x 17 cell-groups need 89 MB of cell
    # tables (20 B each); tiled FP32: 224^2 x 17 cell-groups need ~0.2 GB of cell tables, quadrant partials and
    # boundary buffer; all above the 64 MiB array.  Rejected on the host, nothing launched.
    wl = synth.Workload("big", n, n, 6.0, 17, 0.001, 100.0, 2, 8, 2, 1)
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl, tiled=tiled)
    B = dev(d["B"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    with pytest.raises(molc.MolcError) as e:
        P.sweep_static_scratch(prec, dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"]))
    assert e.value.code == 1 and "static scratch" in str(e.value)
    assert P.device_status() == 0
    P.close()
