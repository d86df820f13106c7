"""Replica mode of the benchmark (the path has no exchange between GPUs: each
rank advances its own instances and the job's throughput is the sum of all
ranks' particle-steps over the slowest rank's time).  Runs as two gloo ranks
on the CPU."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from tests.inputs import workload


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r advanced 1000 (r + 1) particle-steps in 0.5 + 0.25 r seconds
        v, a, t = bench.replica_throughput(1000.0 * (rank + 1), 0.5 + 0.25 * rank, dist, "cpu")
        cfgs = bench.replica_configs("batched48", 1000, rank, 64)
        out[rank] = (v, a, t, sorted(c["instance"] for c in cfgs))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_ranks():
    ws = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(ws, _free_port(), out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        v, a, t, inst = res[r]
        assert a == 3000.0 and t == 0.75 and v == pytest.approx(4000.0)
    # every instance number appears on exactly one rank
    i0, i1 = res[0][3], res[1][3]
    assert len(i0) == len(i1) == 48 and not set(i0) & set(i1)


def test_single_rank_is_plain_ratio():
    assert bench.replica_throughput(600.0, 2.0) == (300.0, 600.0, 2.0)


def test_replica_instances_draw_independent_particles():
    """Two ranks' copies of one instance differ only in the instance number,
    which enters the random counter: their loaded particles must differ."""
    st = []
    for inst in (0, 1):
        cfg = workload(n1=16, n2=8, n_init=200, instance=inst)
        o = oracle.Sim(cfg)
        o.load_volume(0, 200)
        st.append(o.particles(0)[0])
    assert st[0].shape == st[1].shape
    assert not np.allclose(st[0], st[1])


def test_batch_subset_keeps_the_first_instances():
    """bench --instances N --particles P: the first N instances of the
    48-instance batch, unchanged except for the particle count (small runs,
    e.g. under a profiler)."""
    sub = bench.workloads("batched48", 2000, 8)
    full = bench.workloads("batched48")
    assert len(sub) == 8 and len(full) == 48
    assert [(c["n1"], c["n2"], c["alpha"], c["B"]) for c in sub] == [(c["n1"], c["n2"], c["alpha"], c["B"])
                                                                  for c in full[:8]]
    assert all(sp["n_init"] == 2000 for c in sub for sp in c["species"])
