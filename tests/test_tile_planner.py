"""CPU: the tiled FP32 layout of the characteristic grid (Sec. 3, MOLC_TILED) is built and checked by the library's
planner on host-only plans of every shape the GPU tests sweep.  Plan creation fails unless every invariant the tiled kernels
rely on holds (each segment of each sense one record with its cell and length, pieces chained in traversal order
through adjacent tiles along their direction and later in the quadrant's wavefront, moment entries covering every
slot once in its record's cell, the work queue topologically ordered, item states disjoint)."""
import numpy as np
import pytest

import synth

VARIANTS = [
    dict(nx=1, ny=1, G=1, npol=1, naz=4, div=3),
    dict(nx=7, ny=3, G=5, npol=3, naz=8, div=2, L=(3.0, 1.0)),
    dict(nx=5, ny=9, G=2, npol=5, naz=12, div=3),
    dict(nx=6, ny=6, G=3, npol=6, naz=8, div=2, layout="paper"),
    dict(nx=8, ny=5, G=4, npol=7, naz=4, div=2, renorm=False),
    dict(nx=4, ny=4, G=17, npol=8, naz=16, div=4),
    dict(nx=10, ny=10, G=2, npol=2, naz=20, div=1),
    dict(nx=3, ny=4, G=37, npol=2, naz=8, div=2),
    dict(nx=33, ny=17, G=6, npol=4, naz=12, div=2),     # ragged tiles in both directions
]


@pytest.fixture(scope="module")
def molc():
    import paper_2305_11998_gb300 as m
    return m


@pytest.mark.parametrize("vi", range(len(VARIANTS)))
def test_tiled_layout_of_variants(molc, vi):
    v = VARIANTS[vi]
    Lx, Ly = v.get("L", (2.0, 2.0))
    q = synth.product_quadrature(v["npol"], v["naz"])
    h = min(Lx / v["nx"], Ly / v["ny"])
    layout = v.get("layout", "uniform")
    P = molc.Plan(v["nx"], v["ny"], Lx, Ly, q.mu, q.cos_phi, q.sin_phi, q.w, v["G"], h / v["div"], layout,
                  v.get("renorm", layout == "uniform"), host_only=True, tiled=True)
    i = P.info
    assert i.fp32_tile_cells >= 1 and i.fp32_tile_groups >= 1
    n_tiles = -(-v["nx"] // i.fp32_tile_cells) * -(-v["ny"] // i.fp32_tile_cells)
    assert i.fp32_tile_items == 4 * n_tiles * -(-v["G"] // i.fp32_tile_groups)
    P.close()


@pytest.mark.parametrize("name", ["fc16_g4_d32", "fc64_g17_d128"])
def test_tiled_layout_of_workloads(molc, name):
    P = molc.Plan.from_workload(synth.WORKLOADS[name], host_only=True, tiled=True)
    assert P.info.fp32_tile_items > 0
    P.close()


def test_paper_production_spacing_keeps_the_bundle_sweep(molc):
    """Vertex bands halved to 1e-3 cm on 0.6 cm cells: ~9e3 piece segments per cell and quadrant, more than a work
    item holds in shared memory even with one-cell tiles, so the plan sweeps FP32 without tiles."""
    wl = synth.Workload("fc10_paper", 10, 10, 6.0, 17, 0.001, 100.0, 4, 36, 600, 1)
    q = wl.quadrature()
    P = molc.Plan(wl.nx, wl.ny, wl.L, wl.L, q.mu, q.cos_phi, q.sin_phi, q.w, wl.G, 1e-3, "paper", False,
                  host_only=True, tiled=True)
    assert P.info.fp32_tile_items == 0 and P.info.n_split_cells > 0
    P.close()


def test_faces_and_balance_plans_are_not_tiled(molc):
    wl = synth.WORKLOADS["fc16_g4_d32"]
    for kw in ({"faces": True}, {"balance": True}, {}):
        P = molc.Plan.from_workload(wl, host_only=True, tiled=bool(kw), **kw)
        assert P.info.fp32_tile_cells == 0
        P.close()
