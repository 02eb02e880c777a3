"""GPU: the paper's characteristic grid at production ray spacing (Sec. 3 construction, Sec. 4 problem).

10 x 10 cells on 6 cm (h_mat = 0.6 cm) with h_moc = 1e-3 cm: the vertex bands halved down to 1e-3 cm give
~2.7e3 characteristics per azimuth pair (hundreds per cell per direction) and optical thicknesses down to
~1e-6 per segment, the regime of the small-tau branch; every cell's entry list is split into parts for the
moment gather.  Both GPU paths against the oracle on sampled groups (17 groups, 4 x 36 = 144 directions as in
the paper)."""
import numpy as np
import pytest

import oracle
import parity
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paper_layout_production_spacing(prec):
    import paper_2305_11998_gb300 as molc
    wl = synth.Workload("fc10_paper", 10, 10, 6.0, 17, 0.001, 100.0, 4, 36, 600, 1)
    d = wl.inputs(2)
    q = wl.quadrature()
    h_moc = 1e-3
    P = molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, h_moc, "paper", False)
    assert P.info.n_tracks > 1.5e5
    dev = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
    B = dev(d["B"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    got = {k: v.cpu().numpy() for k, v in P.sweep(prec, dev(d["kappa"]), B, d["c"], d["dt"], I, dev(d["bnd"])).items()}
    assert P.device_status() == 0
    P.close()
    # Both paths against the binary128 oracle on two sampled groups: with ~1.6e5 segment terms per cell, the FP64
    # path's own summation bound (gamma_{n-1} of the cell's n terms) is part of the oracle's derived bound.
    groups = [0, 11]
    geom = oracle.Geometry(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, h_moc, 1, 0)
    n_terms = int(np.bincount(oracle.tracks(geom, "double")["cell"], minlength=wl.ncell).max())
    assert n_terms > 5000
    ref = parity.reference(geom, d, prec, wl.n_polar, groups=groups)
    fm = {k: float(np.abs(v).max()) for k, v in got.items()}
    parity.compare({k: v[groups] for k, v in got.items()}, ref, prec, d["c"], floor_max=fm)
