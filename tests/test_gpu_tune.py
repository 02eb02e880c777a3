"""GPU: MOLC_AUTOTUNE with the tuning cache.  A tuned plan records its configuration (bundle sweep: staging
depth; tiled sweep: tile side, groups per work item, block threads) in the JSON file; a later plan with the same
signature takes it without timing (tuned_from_cache), one with another signature is tuned and added; an entry
the library cannot apply is re-tuned.  The configuration changes no segment update: autotuned tiled and bundle
plans carry the same state bit for bit."""
import json

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


@pytest.fixture
def path(tmp_path, molc):
    yield tmp_path / "tune.json"
    molc.tune_cache(None)


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def entries(path):
    d = json.loads(path.read_text())
    assert d["format"] == "molc-tune-cache" and d["version"] == 1
    return d["entries"]


WL = synth.Workload("t24", 24, 24, 6.0, 6, 0.001, 100.0, 2, 16, 2, 1)


def test_bundle_depth_recorded_and_reused(molc, path):
    assert molc.tune_cache(str(path)) == 0
    A = molc.Plan.from_workload(WL, autotune=True)
    assert A.info.tuned_from_cache == 0 and A.info.fp32_sweep_depth in (3, 4, 6)
    es = entries(path)
    assert len(es) == 1
    e = es[0]
    assert e["sweep_depth"] == A.info.fp32_sweep_depth and e["tile_cells"] == 0 and e["best_ms"] > 0
    assert e["key"].startswith("24x24 cells, 6 groups, 32 directions") and "SMs" in e["device"]
    B = molc.Plan.from_workload(WL, autotune=True)                     # same signature: from the file
    assert B.info.tuned_from_cache == 1 and B.info.fp32_sweep_depth == A.info.fp32_sweep_depth
    other = synth.Workload("t24b", 24, 24, 6.0, 7, 0.001, 100.0, 2, 16, 2, 1)
    C = molc.Plan.from_workload(other, autotune=True)                  # another group count: tuned, added
    assert C.info.tuned_from_cache == 0 and len(entries(path)) == 2
    plain = molc.Plan.from_workload(WL)                                # no MOLC_AUTOTUNE: cache not consulted
    assert plain.info.tuned_from_cache == 0 and plain.info.fp32_sweep_depth == 4
    for P in (A, B, C, plain):
        P.close()


def test_edited_entries_apply_or_are_retuned(molc, path):
    assert molc.tune_cache(str(path)) == 0
    A = molc.Plan.from_workload(WL, autotune=True)
    A.close()
    d = json.loads(path.read_text())
    for depth, applied in ((3, True), (6, True), (5, False)):    # 5: no such compiled depth
        d["entries"][0]["sweep_depth"] = depth
        path.write_text(json.dumps(d))
        assert molc.tune_cache(str(path)) == 1
        P = molc.Plan.from_workload(WL, autotune=True)
        assert P.info.tuned_from_cache == int(applied)
        assert P.info.fp32_sweep_depth == depth if applied else P.info.fp32_sweep_depth in (3, 4, 6)
        P.close()
    assert entries(path)[0]["sweep_depth"] in (3, 4, 6)              # the re-tuned choice replaced depth 5


def step(P, d, steps=2):
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity("fp32")
    P.intensity_init("fp32", I, B)
    for _ in range(steps):
        out = P.sweep("fp32", k, B, d["c"], d["dt"], I, bnd)
    torch.cuda.synchronize()
    assert P.device_status() == 0
    return P.intensity_export("fp32", I).cpu().numpy(), {k: v.cpu().numpy() for k, v in out.items()}


def test_tiled_configuration_recorded_and_reused(molc, path):
    wl = synth.WORKLOADS["fc64_g17_d128"]
    d = wl.inputs(4)
    assert molc.tune_cache(str(path)) == 0
    T = molc.Plan.from_workload(wl, tiled=True, autotune=True)
    assert T.info.fp32_tile_items > 0 and T.info.tuned_from_cache == 0
    e = entries(path)[0]
    assert (e["tile_cells"], e["tile_groups"], e["block_threads"]) == \
        (T.info.fp32_tile_cells, T.info.fp32_tile_groups, T.info.fp32_block_threads)
    assert e["sweep_depth"] == 0
    T2 = molc.Plan.from_workload(wl, tiled=True, autotune=True)
    assert T2.info.tuned_from_cache == 1
    assert (T2.info.fp32_tile_cells, T2.info.fp32_tile_groups, T2.info.fp32_block_threads) == \
        (T.info.fp32_tile_cells, T.info.fp32_tile_groups, T.info.fp32_block_threads)
    # any configuration: the same segment updates as the bundle sweep (the moments of both against the oracle:
    # test_gpu_tiled.py); the same configuration: the same moments, bit for bit
    R = molc.Plan.from_workload(wl)
    s_t, m_t = step(T, d)
    s_t2, m_t2 = step(T2, d)
    s_r, _ = step(R, d)
    assert np.array_equal(s_t, s_r) and np.array_equal(s_t2, s_t)
    for k in m_t:
        assert np.array_equal(m_t[k], m_t2[k]), k
    for P in (T, T2, R):
        P.close()


def test_unwritable_cache_leaves_plans_tuned(molc, tmp_path):
    """A cache path whose directory does not exist reads as an empty cache; tuning still runs and the plan is
    created, the entry is simply not recorded."""
    path = tmp_path / "no_such_dir" / "tune.json"
    try:
        assert molc.tune_cache(str(path)) == 0
        P = molc.Plan.from_workload(WL, autotune=True)
        assert P.info.tuned_from_cache == 0 and P.info.fp32_sweep_depth in (3, 4, 6)
        assert not path.exists()
        Q = molc.Plan.from_workload(WL, autotune=True)          # nothing recorded: tuned again
        assert Q.info.tuned_from_cache == 0
        P.close()
        Q.close()
    finally:
        molc.tune_cache(None)
