"""The C-ABI library on the host: it loads, exports every symbol include/molc.h declares, rejects bad
arguments with status codes, and its characteristic-grid planner reproduces the oracle's (no GPU needed)."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_2305_11998_gb300 as molc
import synth

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "molc.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(molc_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = molc.load()
    names = declared_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(molc.EXPORTED)


def test_quadrature_product_matches_generator():
    for npol, naz in [(1, 4), (2, 16), (3, 24), (4, 32), (8, 64)]:
        mu, c, s, w = molc.quadrature_product(npol, naz)
        q = synth.product_quadrature(npol, naz)
        assert np.allclose(mu, q.mu, rtol=0, atol=1e-15)
        assert np.allclose(w, q.w, rtol=1e-13, atol=0)
        assert abs(w.sum() / (4 * np.pi) - 1) < 1e-14
        assert np.allclose(c, q.cos_phi, atol=2e-16) and np.allclose(s, q.sin_phi, atol=2e-16)
    with pytest.raises(molc.MolcError):
        molc.quadrature_product(2, 6)


@pytest.mark.parametrize("name,layout", [("fc16_g4_d32", "uniform"), ("fc16_g4_d32", "paper"),
                                         ("fc64_g17_d128", "uniform")])
def test_planner_matches_oracle_tracks(name, layout):
    wl = synth.WORKLOADS[name]
    lay = 0 if layout == "uniform" else 1
    spacing = wl.spacing if layout == "uniform" else wl.h / 1.5
    P = molc.Plan.from_workload(wl, spacing=spacing, layout=layout, renorm=(layout == "uniform"), host_only=True)
    tr = P.tracks()
    ref = oracle.tracks(oracle.Geometry.from_workload(wl, spacing=spacing, layout=lay,
                                                      renorm=int(layout == "uniform")), "quad")
    for k in ("dir_ray_off", "ray_seg_off", "entry", "cell"):
        assert np.array_equal(tr[k], ref[k]), k
    # widths, lengths and areas are differences of coordinates of size ~L: absolute error ~1e-15 L
    L = wl.L
    assert np.max(np.abs(tr["width"] - ref["width"])) < 1e-14 * L
    assert np.max(np.abs(tr["len"] - ref["len"])) < 1e-14 * L
    assert np.max(np.abs(tr["area"] - ref["area"])) < 1e-14 * L * wl.h
    info = P.info
    assert info.n_segments == tr["cell"].size == ref["cell"].size
    assert info.n_updates == info.n_segments * wl.G
    assert P.intensity_count() == info.n_updates
    P.close()


def test_threaded_planner_matches_oracle_tracks():
    """A grid large enough (cells x azimuth pairs >= 2^17) that molc_create traces the azimuth pairs and sums their
    areas on several host threads: the same characteristic grid as the oracle's own generator."""
    wl = synth.Workload("grid128", 128, 128, 6.0, 2, 0.001, 100.0, 2, 32, 2, 1)
    P = molc.Plan.from_workload(wl, host_only=True)
    assert wl.ncell * P.info.n_azim_pairs >= 1 << 17
    tr = P.tracks()
    ref = oracle.tracks(oracle.Geometry.from_workload(wl, spacing=wl.spacing, layout=0, renorm=1), "quad")
    for k in ("dir_ray_off", "ray_seg_off", "entry", "cell"):
        assert np.array_equal(tr[k], ref[k]), k
    L = wl.L
    assert np.max(np.abs(tr["width"] - ref["width"])) < 1e-14 * L
    assert np.max(np.abs(tr["len"] - ref["len"])) < 1e-14 * L
    assert np.max(np.abs(tr["area"] - ref["area"])) < 1e-14 * L * wl.h
    P.close()


def test_invalid_arguments_are_rejected():
    q = synth.product_quadrature(2, 8)
    with pytest.raises(molc.MolcError) as e:
        molc.Plan(0, 4, 1.0, 1.0, q.mu, q.cos_phi, q.sin_phi, q.w, 2, 0.1, host_only=True)
    assert e.value.code == 1
    with pytest.raises(molc.MolcError):   # spacing <= 0
        molc.Plan(4, 4, 1.0, 1.0, q.mu, q.cos_phi, q.sin_phi, q.w, 2, 0.0, host_only=True)
    with pytest.raises(molc.MolcError):   # a direction without its opposite
        molc.Plan(4, 4, 1.0, 1.0, q.mu[1:], q.cos_phi[1:], q.sin_phi[1:], q.w[1:], 2, 0.1, host_only=True)
    with pytest.raises(molc.MolcError):   # mu out of range
        bad = q.mu.copy()
        bad[0] = 1.5
        molc.Plan(4, 4, 1.0, 1.0, bad, q.cos_phi, q.sin_phi, q.w, 2, 0.1, host_only=True)
    with pytest.raises(molc.MolcError):   # spacing so coarse that some cell is missed: renormalisation impossible
        molc.Plan(16, 16, 1.0, 1.0, q.mu, q.cos_phi, q.sin_phi, q.w, 2, 0.5, host_only=True)
    P = molc.Plan(4, 4, 1.0, 1.0, q.mu, q.cos_phi, q.sin_phi, q.w, 2, 0.1, host_only=True)
    lib = molc.load()
    assert lib.molc_intensity_init(P._h, 1, None, None, None) == 1     # NULL arrays
    assert lib.molc_sweep(P._h, 7, None, None, 1.0, 1.0, None, None, None, None) == 1
    assert b"NULL" in lib.molc_last_error() or len(lib.molc_last_error()) > 0
    P.close()


@pytest.mark.parametrize("fine", [False, True])
def test_split_cell_count_follows_the_entry_lists(fine):
    # the moment gather of the bundle sweep (the default FP32 sweep; also with MOLC_BALANCE): a cell's gather list holds
    # one entry per (track segment, sense) crossing it, padded to a multiple of 4; lists longer than 256 entries are
    # summed in parts (n_split_cells)
    wl = synth.Workload("paper8", 8, 8, 6.0, 17, 0.001, 100.0, 2, 16, 40, 1)
    q = wl.quadrature()
    h = 0.02 if fine else 0.5
    P = molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, h, "paper", False,
                  host_only=True, balance=True)
    assert P.info.fp32_tile_cells == 0
    cells = P.tracks()["cell"]
    entries = np.bincount(cells, minlength=wl.ncell) // wl.n_polar   # export: every polar cosine and sense
    padded = (entries + 3) // 4 * 4
    assert P.info.n_split_cells == int(np.sum(padded > 256))
    assert (P.info.n_split_cells > 0) == fine
    P.close()


def test_balance_check_does_not_combine_with_face_moments():
    wl = synth.WORKLOADS["fc16_g4_d32"]
    with pytest.raises(molc.MolcError):
        molc.Plan.from_workload(wl, host_only=True, faces=True, balance=True)
    P = molc.Plan.from_workload(wl, host_only=True, balance=True)
    P.close()


def test_host_only_plans_are_refused_by_device_calls():
    """A MOLC_HOST_ONLY plan holds nothing on a device: every call that would touch one returns
    MOLC_ERR_INVALID_ARG naming MOLC_HOST_ONLY, before any CUDA call (the arguments are host buffers that are never
    read); the host calls accept it."""
    import ctypes as C
    from paper_2305_11998_gb300 import molc as mm
    wl = synth.WORKLOADS["fc16_g4_d32"]
    P = molc.Plan.from_workload(wl, host_only=True, tiled=True)
    lib = molc.load()
    buf = np.zeros(1 << 16)                      # host memory standing in for every device array
    ptr = C.c_void_p(buf.ctypes.data)
    mom = mm._Moments(*([buf.ctypes.data] * len(mm.MOMENTS)))
    d, n = C.c_double(), C.c_int()
    parts = (C.c_double * 3)()
    calls = {
        "intensity_init": lambda: lib.molc_intensity_init(P._h, 1, ptr, ptr, None),
        "sweep": lambda: lib.molc_sweep(P._h, 1, ptr, ptr, 1.0, 1.0, ptr, ptr, C.byref(mom), None),
        "sweep_closure": lambda: lib.molc_sweep_closure(P._h, 0, ptr, ptr, 1.0, 1.0, ptr, ptr, C.byref(mom), ptr,
                                                        ptr, ptr, None),
        "sweep_static_scratch": lambda: lib.molc_sweep_static_scratch(P._h, 1, ptr, ptr, 1.0, 1.0, ptr, ptr,
                                                                      C.byref(mom), None),
        "closure": lambda: lib.molc_closure(P._h, C.byref(mom), 1.0, ptr, ptr, ptr, None, None),
        "grey_coefficients": lambda: lib.molc_grey_coefficients(P._h, C.byref(mom), ptr, ptr, ptr, None),
        "face_moments": lambda: lib.molc_face_moments(P._h, 0, ptr, 1.0, C.byref(mom), None),
        "intensity_export": lambda: lib.molc_intensity_export(P._h, 1, ptr, 0, 1, ptr, None),
        "intensity_import": lambda: lib.molc_intensity_import(P._h, 0, ptr, 0, 1, ptr, ptr, None),
        "ray_balance": lambda: lib.molc_ray_balance(P._h, C.byref(d)),
        "kernel_timing": lambda: lib.molc_kernel_timing(P._h, 1),
        "kernel_time": lambda: lib.molc_kernel_time(P._h, C.byref(d), C.byref(n)),
        "kernel_time_parts": lambda: lib.molc_kernel_time_parts(P._h, parts, C.byref(n)),
        "device_status": lambda: lib.molc_device_status(P._h, C.byref(n)),
    }
    for name, call in calls.items():
        assert call() == 1, name
        assert b"MOLC_HOST_ONLY" in lib.molc_last_error(), (name, lib.molc_last_error())
    plans = (C.c_void_p * 1)(P._h)
    out = C.c_void_p()
    assert lib.molc_batch_create(plans, 1, C.byref(out)) == 1 and not out.value
    assert b"MOLC_HOST_ONLY" in lib.molc_last_error()
    # the host calls
    assert P.intensity_count() == P.info.n_updates
    assert lib.molc_intensity_bytes(P._h, 1) > 0 and lib.molc_intensity_bytes(P._h, 0) > 0
    assert P.tracks()["cell"].size == P.info.n_segments
    P.retile(tile_cells=4)
    assert P.info.fp32_tile_cells == 4
    P.close()
