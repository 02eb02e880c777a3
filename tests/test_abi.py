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
