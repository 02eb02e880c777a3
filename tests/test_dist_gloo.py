"""Multi-rank host logic on CPU: two gloo ranks on 127.0.0.1.

The sweep shards by groups (one instance split into contiguous group ranges, one per rank) with no data exchange
on the path; these tests check the host side of that: the timing collective (max over ranks), the group shards
and the slices of the inputs, that sweeping group shards on separate ranks reproduces the unsharded sweep exactly
(oracle, CPU), and the all-gather that hands every rank all groups' results.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2305_11998_gb300 import dist as pdist  # noqa: E402

WORLD = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ws, rk, lr = pdist.env()
        assert (ws, rk, lr) == (world, rank, rank)
        # timing collective: every rank sees the slowest rank's time
        t = pdist.max_over_ranks(10.0 + 5.0 * rank)
        # group shard of a tiny instance, swept by the oracle on this rank only
        import oracle
        import synth
        wl = synth.WORKLOADS["fc16_g4_d32"]
        d = wl.inputs(3)      # every rank holds the same instance here
        geom = oracle.Geometry.from_workload(wl)
        groups = list(pdist.shard_groups(wl.G, ws, rk))
        r = oracle.sweep(geom, d["kappa"], d["B"], d["c"], d["dt"], d["bnd"], groups=groups, precision="double",
                         want_I=False, threads=1)
        # all-gather of the per-group results into every rank (the grey closure's consumer of all groups)
        gathered = pdist.gather_groups(torch.tensor(r["E"]), wl.G, pdist.shard_groups(wl.G, ws, rk), ws)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), t=t, groups=np.array(groups), gathered=gathered.numpy(),
                 **{k: r[k] for k in ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy")})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_groups_and_reduce_time(tmp_path):
    port = _free_port()
    mp.start_processes(_rank_main, args=(WORLD, port, str(tmp_path)), nprocs=WORLD, join=True,
                       start_method="spawn")
    res = [np.load(tmp_path / f"rank{r}.npz") for r in range(WORLD)]
    assert all(float(x["t"]) == 15.0 for x in res)
    covered = np.concatenate([x["groups"] for x in res])
    import oracle
    import synth
    wl = synth.WORKLOADS["fc16_g4_d32"]
    assert sorted(covered.tolist()) == list(range(wl.G))
    d = wl.inputs(3)
    full = oracle.sweep(oracle.Geometry.from_workload(wl), d["kappa"], d["B"], d["c"], d["dt"], d["bnd"],
                        precision="double", want_I=False, threads=1)
    for x in res:
        g = x["groups"]
        for k in ("E", "Fx", "Fy", "Nxx", "Nxy", "Nyy"):
            assert np.array_equal(x[k], full[k][g]), k     # groups are independent: bit-identical
        assert np.array_equal(x["gathered"], full["E"])   # every rank ends with all groups


def test_shard_groups_cover_and_balance():
    for G in (1, 4, 17, 32):
        for world in (1, 2, 3, 4, 8):
            shards = [pdist.shard_groups(G, world, r) for r in range(world)]
            assert [g for s in shards for g in s] == list(range(G))
            sizes = [len(s) for s in shards]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        pdist.shard_groups(4, 2, 2)


def test_local_reduction_and_gather():
    assert pdist.max_over_ranks(3.5) == 3.5      # not distributed: the value itself
    local = torch.arange(6.0).reshape(2, 3)
    assert pdist.gather_groups(local, 2, range(0, 2), 1) is local


def test_shard_inputs_slice_groups():
    import synth
    wl = synth.WORKLOADS["fc16_g4_d32"]
    d = wl.inputs(0)
    s = pdist.shard_inputs(d, range(1, 3))
    assert np.array_equal(s["kappa"], d["kappa"][1:3]) and np.array_equal(s["B"], d["B"][1:3])
    assert s["bnd"].shape == (4, 2) and s["bnd"].flags["C_CONTIGUOUS"] and np.array_equal(s["bnd"], d["bnd"][:, 1:3])
