"""Host-side multi-process paths on the CPU (gloo, world size 2): unit sharding
and replica combination, the distribution the library uses across GPUs."""
import math
import os
import socket

import pytest
import torch.multiprocessing as mp

import workloads as W
from paper_1511_03614_gb300 import prepare_feynman
from paper_1511_03614_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _fake_unit_results(prep, lo, hi, seed):
    """Deterministic stand-ins for per-unit integration results (no GPU here)."""
    out = []
    for k in range(lo, hi):
        u = prep.units[k]
        out.append(dict(value=math.sin(k + 1) + 0.01 * seed, sigma=0.01 * (1 + k % 3), order=u.order))
    return out


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    prep = prepare_feynman(W.box())
    sl = shard.shard_slices(prep.units, world)
    b, e = sl[rank]
    mine = _fake_unit_results(prep, b, e, 0)
    allres = shard.gather(mine, world)
    val, err = shard.combine_shards(allres, prep.int_orders)
    reps = shard.gather(_fake_unit_results(prep, 0, len(prep.units), rank + 1), world)
    comb = shard.combine_replicas(reps)
    if rank == 0:
        q.put((val, err, [c["value"] for c in comb], [c["sigma"] for c in comb]))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_slices_cover_every_unit_once():
    prep = prepare_feynman(W.box())
    for world in (1, 2, 3, 5):
        sl = shard.shard_slices(prep.units, world)
        assert len(sl) == world and sl[0][0] == 0 and sl[-1][1] == len(prep.units)
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        assert all(b > a for a, b in sl)


def test_two_gloo_ranks_match_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    val, err, rv, rs = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    prep = prepare_feynman(W.box())
    single = _fake_unit_results(prep, 0, len(prep.units), 0)
    v1, e1 = shard.combine_shards([single], prep.int_orders)
    for K in prep.int_orders:
        assert abs(val[K] - v1[K]) < 1e-12 and abs(err[K] - e1[K]) < 1e-12
    # two replicas with equal errors: the mean of the two values, error / sqrt(2)
    a = _fake_unit_results(prep, 0, len(prep.units), 1)
    b = _fake_unit_results(prep, 0, len(prep.units), 2)
    for k in range(len(prep.units)):
        assert abs(rv[k] - (a[k]["value"] + b[k]["value"]) / 2) < 1e-12
        assert abs(rs[k] - a[k]["sigma"] / math.sqrt(2)) < 1e-12
