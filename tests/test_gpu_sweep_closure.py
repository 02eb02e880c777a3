"""GPU: molc_sweep_closure (one step and its Eddington factors in one call) against molc_sweep + molc_closure.

The fused call forms f = N/(cE) where each cell's moments are assembled, with the same operations as
molc_closure, so its factors equal molc_closure applied to its own moments bit for bit.  Its moments and state
equal molc_sweep's bit for bit on the FP32 path (no atomics) and to the FP64 summation order on the FP64 path
(FP64 atomics).  Cases: one group chunk, two chunks (G = 37), and split cell lists (paper layout at a fine
spacing, cells crossed by more than 256 segment entries).
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


def plans(molc):
    wl = synth.WORKLOADS["fc64_g17_d128"]
    yield "fc64", wl, molc.Plan.from_workload(wl)
    wl = synth.Workload("g37", 20, 20, 6.0, 37, 0.001, 100.0, 3, 16, 2, 1)
    yield "g37", wl, molc.Plan.from_workload(wl)
    wl = synth.Workload("paper8", 8, 8, 6.0, 17, 0.001, 100.0, 2, 16, 40, 1)
    q = wl.quadrature()
    # tiled: ~270 moment entries per cell and quadrant, summed in parts of 64
    yield "paper8_tiled", wl, molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, 0.02,
                                        "paper", False, tiled=True)
    # the bundle sweep: ~1100 entries per cell in the moment gather, parts of 256
    yield "paper8_bundle", wl, molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, 0.02,
                                         "paper", False)
    yield "fc64_tiled", synth.WORKLOADS["fc64_g17_d128"], molc.Plan.from_workload(synth.WORKLOADS["fc64_g17_d128"],
                                                                                   tiled=True)


def close(a, b, c):
    """FP64 summation-order agreement: 1e-12 relative on E, Nxx, Nyy, 1e-12 of cE on Fx, Fy, Nxy."""
    cE = c * np.abs(b["E"])
    for k in ("E", "Nxx", "Nyy"):
        den = np.maximum(np.abs(b[k]), 1e-30 * np.abs(b[k]).max())
        assert np.max(np.abs(a[k] - b[k]) / den) <= 1e-12, k
    for k in ("Fx", "Fy", "Nxy"):
        assert np.max(np.abs(a[k] - b[k]) / np.maximum(cE, 1e-30 * cE.max())) <= 1e-12, k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_sweep_closure_matches_sweep_then_closure(molc, prec):
    for name, wl, P in plans(molc):
        if name == "paper8_bundle":   # split cell lists: ~1100 segment entries per cell, parts of 256
            assert P.info.n_split_cells == wl.ncell
        d = wl.inputs(5)
        k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
        I_ref = P.new_intensity(prec).zero_()
        I_new = P.new_intensity(prec).zero_()
        P.intensity_init(prec, I_ref, B)
        P.intensity_init(prec, I_new, B)
        for _ in range(2):
            ref = P.sweep(prec, k, B, d["c"], d["dt"], I_ref, bnd)
            f_ref = P.closure(ref, d["c"])
            got, f_got = P.sweep_closure(prec, k, B, d["c"], d["dt"], I_new, bnd)
            f_own = P.closure(got, d["c"])
            torch.cuda.synchronize()
            for kk in ("fxx", "fxy", "fyy"):
                assert torch.equal(f_got[kk], f_own[kk]), (name, kk)      # the same bits as molc_closure
            if prec == "fp32":
                for kk in got:
                    assert torch.equal(got[kk], ref[kk]), (name, kk)
                for kk in ("fxx", "fxy", "fyy"):
                    assert torch.equal(f_got[kk], f_ref[kk]), (name, kk)
                assert torch.equal(I_new, I_ref), name
            else:
                close({kk: v.cpu().numpy() for kk, v in got.items()},
                      {kk: v.cpu().numpy() for kk, v in ref.items()}, d["c"])
        assert P.device_status() == 0, name
        P.close()


def test_sweep_closure_rejects_missing_factor_arrays(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    P = molc.Plan.from_workload(wl)
    B = dev(d["B"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    out = P.new_moments()
    m = molc.molc._Moments(*[out[k].data_ptr() for k in molc.molc.MOMENTS])
    import ctypes as C
    rc = P._lib.molc_sweep_closure(P._h, 1, C.c_void_p(dev(d["kappa"]).data_ptr()), C.c_void_p(B.data_ptr()),
                                   float(d["c"]), float(d["dt"]), C.c_void_p(I.data_ptr()),
                                   C.c_void_p(dev(d["bnd"]).data_ptr()), C.byref(m), None, None, None, None)
    assert rc == 1 and b"NULL factor" in P._lib.molc_last_error()
    P.close()
