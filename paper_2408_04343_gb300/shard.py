"""The step protocol of a system split by neuron range (snp_shard_*).

A shard runs phase 1 of the step for its neurons (rule choice, consumption,
delay status), writing their emissions into its slice of a full-length
emission vector; the shards' slices are exchanged so that every shard holds
the whole vector; the shards' activity flags are OR-ed (no shard active: the
system is at a fixed point and the step is not executed); then each shard
runs phase 2 for its neurons (the in-flow from the whole vector).  This
module holds only that protocol -- the ranges, the order of the calls, the
exchange -- over shards that provide ``select(k) -> bool`` and
``receive()``: the CUDA shards of libsnp, or any other implementation of the
two phases.

Exchanges:
* ``local_exchange``: shards of one process (one or several devices), the
  slices copied between their emission tensors;
* ``collective_exchange``: one shard per rank of a torch.distributed group
  (NCCL between GPUs, gloo on CPU): an in-place all_gather of the equal-size
  slices of the emission vector, and an all_reduce (max) of the activity.
"""
from __future__ import annotations


def shard_ranges(q: int, world: int):
    """Equal chunks of ceil(q / world) neurons: rank r owns [r c, min(q, (r+1) c)).
    The emission vector has world * c + 1 entries (the last ones never emit)."""
    c = -(-q // world)
    return [(min(q, r * c), min(q, (r + 1) * c)) for r in range(world)], c


def run(shards, n: int, k0: int, exchange, any_active) -> int:
    """Up to n steps of the sharded system from absolute step k0; returns the
    steps executed (fewer at a fixed point)."""
    k = k0
    for _ in range(n):
        act = [sh.select(k) for sh in shards]       # every shard runs phase 1
        if not any_active(any(act)):
            break
        exchange()
        for sh in shards:
            sh.receive()
        k += 1
    return k - k0


def local_exchange(slices):
    """slices: per shard (E tensor, lo, hi).  Copies each shard's slice into
    every other shard's vector (device to device, peer copies across GPUs)."""
    def ex():
        for E_dst, _, _ in slices:
            for E_src, lo, hi in slices:
                if E_src is not E_dst and hi > lo:
                    E_dst[lo:hi].copy_(E_src[lo:hi])
    return ex


def collective_exchange(E, rank: int, world: int, chunk: int):
    """One shard per rank: E is this rank's emission vector (world * chunk + 1
    entries).  Returns (exchange, any_active) over the default process group."""
    import torch
    import torch.distributed as dist

    def ex():
        view = E[:world * chunk]
        dist.all_gather_into_tensor(view, view[rank * chunk:(rank + 1) * chunk].clone())

    def any_active(a: bool) -> bool:
        t = torch.tensor([1 if a else 0], dtype=torch.int32, device=E.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return bool(t.item())

    return ex, any_active
