"""GPU: one instance split into contiguous group ranges (the multi-GPU partition), the shards swept one after another
on one GPU against the unsharded sweep.

Every group is swept independently (Sec. 3: kappa_g, B_g and I_g of one group never meet another's), so a plan
built over a group range on the same characteristic grid reproduces those groups of the full plan.  The FP32 state
works in units scaled by a power of two that follows the plan's max(B, boundary); the inputs here give every group
the same maximum, so every shard takes the full plan's scale and the FP32 results must agree bit for bit (state,
moments, Eddington factors).  The FP64 path adds with atomics in no fixed order: agreement to 1e-12.
"""
import numpy as np
import pytest

import synth
from paper_2305_11998_gb300 import dist as pdist

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def molc():
    import paper_2305_11998_gb300 as m
    m.load()
    return m


def dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def same_max_inputs(wl, seed, M=1e-2):
    d = wl.inputs(seed)
    for g in range(wl.G):
        f = M / max(d["B"][g].max(), d["bnd"][:, g].max())
        d["B"][g] *= f
        d["bnd"][:, g] *= f
    return d


def run(molc, wl, d, prec, groups=None, steps=2):
    P = molc.Plan.from_workload(wl, groups=groups)
    k, B, bnd = dev(d["kappa"]), dev(d["B"]), dev(d["bnd"])
    I = P.new_intensity(prec)
    P.intensity_init(prec, I, B)
    res = []
    for _ in range(steps):
        m, f = P.sweep_closure(prec, k, B, d["c"], d["dt"], I, bnd)
        res.append(({kk: v.cpu().numpy() for kk, v in m.items()}, {kk: v.cpu().numpy() for kk, v in f.items()},
                    P.intensity_export(prec, I).cpu().numpy()))
    assert P.device_status() == 0
    P.close()
    return res


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("world", [2, 4])
def test_group_shards_reproduce_the_unsharded_sweep(molc, prec, world):
    wl = synth.WORKLOADS["fc64_g17_d128"]
    d = same_max_inputs(wl, 6)
    full = run(molc, wl, d, prec)
    seen = []
    for rank in range(world):
        groups = pdist.shard_groups(wl.G, world, rank)
        seen += list(groups)
        part = run(molc, wl, pdist.shard_inputs(d, groups), prec, groups=groups)
        for (mf, ff, If), (mp, fp, Ip) in zip(full, part):
            if prec == "fp32":
                assert np.array_equal(If[:, groups.start:groups.stop], Ip)
                for k in mp:
                    assert np.array_equal(mf[k][groups.start:groups.stop], mp[k]), k
                for k in fp:
                    assert np.array_equal(ff[k][groups.start:groups.stop], fp[k]), k
            else:
                cE = d["c"] * np.abs(mf["E"][groups.start:groups.stop])
                for k in mp:
                    a, b = mp[k], mf[k][groups.start:groups.stop]
                    den = np.abs(b) if k in ("E", "Nxx", "Nyy") else cE
                    den = np.maximum(den, 1e-30 * np.abs(b).max())
                    assert np.max(np.abs(a - b) / den) <= 1e-12, k
    assert sorted(seen) == list(range(wl.G))
