"""GPU: batched FP32 sweep over uneven instances (one launch per kernel class), CUDA-graph replay, autotuner.

The batched kernels run the same per-instance arithmetic as molc_sweep + molc_closure, and the FP32 path is
deterministic (no atomics), so every result is compared bit for bit with the per-instance calls.  A batch of
instances with 1-4 polar cosines is also followed step by step by the binary128 oracle through the parity gate
of the per-instance tests (tests/parity.py).
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


# uneven instances: cells per side, groups, polar x azimuthal directions, ray spacing h/div (three polar classes,
# G = 37 spans two group chunks)
SHAPES = [(16, 4, 2, 16, 2), (24, 17, 3, 24, 4), (32, 8, 4, 32, 2), (12, 32, 2, 16, 4), (20, 37, 4, 16, 2),
          (8, 17, 3, 8, 2)]


def make_instances(molc, autotune=False, tiled=False):
    out = []
    for i, (n, G, npol, naz, div) in enumerate(SHAPES):
        wl = synth.Workload(f"b{i}", n, n, 6.0, G, 0.001, 100.0, npol, naz, div, 1)
        d = wl.inputs(10 + i)
        P = molc.Plan.from_workload(wl, autotune=autotune, tiled=tiled)
        out.append((wl, d, P))
    return out


def new_args(P, wl, d, closure):
    B = dev(d["B"])
    I = P.new_intensity("fp32").zero_()
    P.intensity_init("fp32", I, B)
    a = dict(kappa=dev(d["kappa"]), B=B, c=d["c"], dt=d["dt"], I=I, bnd=dev(d["bnd"]), out=P.new_moments())
    if closure:
        a["f"] = {k: torch.empty((wl.G, wl.ncell), dtype=torch.float64, device="cuda") for k in ("fxx", "fxy", "fyy")}
    return a


def per_instance_step(P, a):
    P.sweep("fp32", a["kappa"], a["B"], a["c"], a["dt"], a["I"], a["bnd"], out=a["out"])
    if "f" in a:
        f = P.closure(a["out"], a["c"])
        for k in ("fxx", "fxy", "fyy"):
            a["f"][k].copy_(f[k])


def assert_same(a, b):
    assert torch.equal(a["I"], b["I"])
    for k in a["out"]:
        assert torch.equal(a["out"][k], b["out"][k]), k
    if "f" in a:
        for k in a["f"]:
            assert torch.equal(a["f"][k], b["f"][k]), k


@pytest.mark.parametrize("tiled", [False, True])
def test_batch_matches_per_instance(molc, tiled):
    """Bit for bit: the bundle kernels (one launch per class) or the tiled sweep (one persistent launch over the
    items of every instance, the longest wavefronts first)."""
    inst = make_instances(molc, tiled=tiled)
    assert all((P.info.fp32_tile_items > 0) == tiled for _, _, P in inst)
    ref = [new_args(P, wl, d, closure=(i % 2 == 0)) for i, (wl, d, P) in enumerate(inst)]
    got = [new_args(P, wl, d, closure=(i % 2 == 0)) for i, (wl, d, P) in enumerate(inst)]
    batch = molc.Batch([P for _, _, P in inst])
    batch.bind(got)
    for _ in range(3):
        for (wl, d, P), a in zip(inst, ref):
            per_instance_step(P, a)
        batch.sweep()
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert_same(a, b)
    for _, _, P in inst:
        assert P.device_status() == 0
    batch.close()


def test_batch_steps_replayed_from_a_cuda_graph(molc):
    inst = make_instances(molc)
    eager = [new_args(P, wl, d, closure=True) for wl, d, P in inst]
    graph = [new_args(P, wl, d, closure=True) for wl, d, P in inst]
    be = molc.Batch([P for _, _, P in inst])
    be.bind(eager)
    bg = molc.Batch([P for _, _, P in inst])
    bg.bind(graph)
    # two steps per graph, replayed twice = four steps
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        bg.sweep()
        bg.sweep()
    for _ in range(2):
        g.replay()
    for _ in range(4):
        be.sweep()
    torch.cuda.synchronize()
    for a, b in zip(graph, eager):
        assert_same(a, b)
    be.close()
    bg.close()


def test_autotuned_plans_give_identical_results(molc):
    base = make_instances(molc)[:3]
    tuned = make_instances(molc, autotune=True)[:3]
    for (wl, d, P), (_, _, Q) in zip(base, tuned):
        assert Q.info.fp32_sweep_depth in (3, 4, 6)
        assert P.info.fp32_sweep_depth == 4
        a = new_args(P, wl, d, closure=False)
        b = new_args(Q, wl, d, closure=False)
        for _ in range(2):
            per_instance_step(P, a)
            per_instance_step(Q, b)
        torch.cuda.synchronize()
        assert_same(a, b)
        assert Q.device_status() == 0


def test_batch_rejects_bad_arguments(molc):
    inst = make_instances(molc)[:2]
    batch = molc.Batch([P for _, _, P in inst])
    with pytest.raises(molc.MolcError):
        batch.sweep()                         # nothing bound yet
    args = [new_args(P, wl, d, closure=False) for wl, d, P in inst]
    args[1]["c"] = -1.0
    with pytest.raises(molc.MolcError):
        batch.bind(args)
    batch.close()


# one instance per polar count 1-4 (odd NP takes the warp-cooperative state copies), G = 37 over
# two group chunks, and an instance with twice the ray density
ORACLE_SHAPES = [(16, 5, 1, 16, 2), (20, 6, 2, 24, 2), (24, 4, 3, 32, 4), (16, 37, 3, 16, 2), (12, 8, 4, 16, 2)]


def test_batched_instances_vs_binary128(molc):
    """Every instance of a batch against the binary128 oracle, over three steps with the state carried (the
    oracle carries its deviations and the bound of the path's state), through the same gate as the per-instance
    parity tests; the factors the batch forms in its moment assembly against N / (c E) of its own moments."""
    import oracle
    import parity
    inst = []
    for i, (n, G, npol, naz, div) in enumerate(ORACLE_SHAPES):
        wl = synth.Workload(f"o{i}", n, n, 6.0, G, 0.001, 100.0, npol, naz, div, 1)
        inst.append((wl, wl.inputs(20 + i), molc.Plan.from_workload(wl)))
    args = [new_args(P, wl, d, closure=True) for wl, d, P in inst]
    batch = molc.Batch([P for _, _, P in inst])
    batch.bind(args)
    carried = [(None, None)] * len(inst)
    for _ in range(3):
        batch.sweep()
        torch.cuda.synchronize()
        for j, ((wl, d, P), a) in enumerate(zip(inst, args)):
            geom = oracle.Geometry.from_workload(wl)
            dev_prev, err_prev = carried[j]
            ref = parity.reference(geom, d, "fp32", wl.n_polar, I_prev=dev_prev, I_err=err_prev, want_I=True)
            carried[j] = (ref["I"], ref["I_err"])
            got = {k: v.cpu().numpy() for k, v in a["out"].items()}
            parity.compare(got, ref, "fp32", d["c"])
            cE = d["c"] * got["E"]
            for k, nm in (("fxx", "Nxx"), ("fxy", "Nxy"), ("fyy", "Nyy")):
                f = a["f"][k].cpu().numpy()
                want = got[nm] / cE
                assert np.all(np.abs(f - want) <= 8 * 2.0 ** -53 * np.abs(want) + 1e-300), (j, k)
    for _, _, P in inst:
        assert P.device_status() == 0
        P.close()
    batch.close()


def test_batch64_at_full_size_sampled_vs_binary128(molc):
    """The batched pattern at its benchmark size: the 64 seeded instances of synth.batch_instances (38.6 GB of FP32
    state) stepped once by molc_batch_sweep; for the largest instance with 2 and with 3 polar cosines (4: the 512^2
    test of test_gpu_misc.py), the group holding the Planck peak of the hot region (1 keV) is checked against the
    binary128 oracle, the floor of the relative metric taken over all groups of that instance's GPU output.
    (Default staging depths: the autotuner's choice changes no arithmetic.)"""
    import oracle
    import parity
    wls = synth.batch_instances(64)
    plans = [molc.Plan.from_workload(wl) for wl in wls]
    ins = [wl.inputs(seed=wl.extra["seed"]) for wl in wls]
    args = [new_args(P, wl, d, closure=False) for wl, d, P in zip(wls, ins, plans)]
    batch = molc.Batch(plans)
    batch.bind(args)
    batch.sweep()
    torch.cuda.synchronize()
    assert all(P.device_status() == 0 for P in plans)
    assert sum(P.info.n_updates for P in plans) > 9e9
    largest = {}
    for i, (wl, P) in enumerate(zip(wls, plans)):
        if wl.n_polar not in largest or P.info.n_updates > plans[largest[wl.n_polar]].info.n_updates:
            largest[wl.n_polar] = i
    assert sorted(largest) == [2, 3, 4]
    results = {}
    del largest[4]
    for npol, i in largest.items():
        results[i] = {k: v.cpu().numpy() for k, v in args[i]["out"].items()}
    batch.close()
    for P in plans:
        P.close()
    del args
    torch.cuda.empty_cache()
    for npol, i in sorted(largest.items()):
        wl, d, got = wls[i], ins[i], results[i]
        edges = wl.edges()
        g = int(np.searchsorted(edges, 2.8, side="right") - 1)     # group of the 1 keV Planck peak (2.82 kT)
        ref = parity.reference(oracle.Geometry.from_workload(wl), d, "fp32", wl.n_polar, groups=[g])
        fm = {k: float(np.abs(v).max()) for k, v in got.items()}
        parity.compare({k: v[[g]] for k, v in got.items()}, ref, "fp32", d["c"], floor_max=fm)
