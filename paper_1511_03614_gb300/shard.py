"""Host-side distribution of units over processes (one GPU each).

The units (sector, eps order) are independent integrals, the paper's first
layer of parallelism (Sec. 2.3-2.5: a pool of workers, one integrand each, on
threads or MPI ranks; ``-part i/n`` splits the integrands of an order).  Two
host-only schemes, with no device collective:

* shards: rank r integrates a contiguous slice of the units, balanced by an
  estimate of the work (instructions x dimension); the per-unit results are
  gathered on the host and summed per order (mean-square errors, Sec. 4.3);
* replicas: every rank integrates every unit with its own seed; the replicas'
  per-unit estimates are combined with inverse-variance weights.
"""
from __future__ import annotations

import math


def unit_cost(unit):
    return (len(unit.program.code) + 8) * (unit.dim + 2)


def shard_slices(units, world):
    """Contiguous [begin, end) per rank, balanced by ``unit_cost``; every unit in exactly one slice."""
    costs = [unit_cost(u) for u in units]
    total = float(sum(costs))
    out = []
    b = 0
    acc = 0.0
    for r in range(world):
        if r == world - 1:
            out.append((b, len(units)))
            break
        goal = total * (r + 1) / world
        e = b
        while e < len(units) - (world - 1 - r) and (acc + costs[e] <= goal or e == b):
            acc += costs[e]
            e += 1
        out.append((b, e))
        b = e
    return out


def combine_shards(per_rank_units, orders):
    """Per order: sum of unit values, sqrt of the sum of squared errors (Sec. 4.3).
    Records of complex units (``part`` 1: imaginary) give complex values, with errors
    complex(sigma_re, sigma_im)."""
    val = {K: [0.0, 0.0] for K in orders}
    err = {K: [0.0, 0.0] for K in orders}
    cplx = False
    for units in per_rank_units:
        for u in units:
            p = u.get("part", 0)
            cplx = cplx or p == 1
            val[u["order"]][p] += u["value"]
            err[u["order"]][p] += u["sigma"] ** 2
    if cplx:
        return ({K: complex(*v) for K, v in val.items()},
                {K: complex(math.sqrt(e[0]), math.sqrt(e[1])) for K, e in err.items()})
    return {K: v[0] for K, v in val.items()}, {K: math.sqrt(e[0]) for K, e in err.items()}


def combine_replicas(per_rank_units):
    """Inverse-variance combination of replicas' estimates of the same units."""
    n = len(per_rank_units[0])
    out = []
    for k in range(n):
        ests = [units[k] for units in per_rank_units]
        if any(e["sigma"] <= 0 for e in ests):
            exact = [e["value"] for e in ests if e["sigma"] <= 0]
            out.append(dict(ests[0], value=sum(exact) / len(exact), sigma=0.0))
            continue
        w = [1.0 / e["sigma"] ** 2 for e in ests]
        v = sum(wi * e["value"] for wi, e in zip(w, ests)) / sum(w)
        out.append(dict(ests[0], value=v, sigma=math.sqrt(1.0 / sum(w))))
    return out


def gather(obj, world):
    """All ranks' ``obj`` on every rank (torch.distributed object gather; host only)."""
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out
