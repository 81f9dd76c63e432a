"""The sharded step's host protocol (paper_2408_04343_gb300/shard.py) on the
CPU, with the oracle's range phases as the shards: the neuron ranges, the
step loop, the local exchange and the fixed-point stop, for 1 to 5 shards,
against the whole system's oracle run.  The CUDA shards follow the same
protocol (tests/test_gpu_shard.py); here nothing needs a GPU."""
import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import shard, synth


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


@pytest.mark.parametrize("q,world", [(1, 1), (1, 3), (5, 4), (10, 3), (1000, 4), (1001, 5)])
def test_ranges_cover_every_neuron_once(q, world):
    ranges, chunk = shard.shard_ranges(q, world)
    assert len(ranges) == world and chunk == -(-q // world)
    got = [i for lo, hi in ranges for i in range(lo, hi)]
    assert got == list(range(q))                      # contiguous, in order, no overlap
    assert all(0 <= lo <= hi <= q for lo, hi in ranges)
    assert all(hi - lo <= chunk for lo, hi in ranges)


class _NumpyShard:
    """An oracle range shard whose emission vector is a numpy slice, for
    shard.local_exchange-style copies."""

    def __init__(self, d, lo, hi, mode, seed):
        self.sh = oracle.RangeShard(d, lo, hi)
        self.mode, self.seed = mode, seed

    def select(self, k):
        return self.sh.select(k, self.mode, self.seed)

    def receive(self):
        self.sh.receive()


def _exchange(shards):
    def ex():
        for dst in shards:
            for src in shards:
                if src is not dst:
                    dst.sh.E[src.sh.lo:src.sh.hi] = src.sh.E[src.sh.lo:src.sh.hi]
    return ex


@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("mode", [oracle.FIRST, oracle.PHILOX])
def test_protocol_over_range_shards_equals_the_whole_system(world, mode):
    d = synth.random_system(777, 21, outdeg=(1, 9), rules=(2, 4), d_range=(0, 3), spikes=(0, 9))
    ranges, _ = shard.shard_ranges(d.q, world)
    shs = [_NumpyShard(d, lo, hi, mode, 99) for lo, hi in ranges]
    done = shard.run(shs, 40, 0, _exchange(shs), lambda a: a)
    st = oracle.initial_state(d)
    ex, _ = oracle.run(d, st, 40, mode, 99)
    assert done == ex
    for s_ in shs:
        lo, hi = s_.sh.lo, s_.sh.hi
        assert (s_.sh.C[lo:hi] == st[0][lo:hi]).all()
        assert (s_.sh.D[lo:hi] == st[1][lo:hi]).all()
        assert (s_.sh.P[lo:hi] == st[2][lo:hi]).all()


def test_protocol_stops_at_the_fixed_point_and_resumes_at_k0():
    """A system that halts: the loop stops at the first step no shard is
    active in, reports the executed steps, and a second run from that step
    executes nothing."""
    # every neuron holds a forgetting rule for exactly 1 spike and starts with 1
    q = 12
    offs = np.arange(q + 1, dtype=np.int64)
    one = np.ones(q, np.int32)
    d = synth.SystemDesc(q=q, init_spikes=one, rule_offsets=offs, rule_k=one, rule_j=np.zeros(q, np.int32),
                         rule_c=one, rule_p=np.zeros(q, np.int32), rule_d=np.zeros(q, np.int32),
                         syn_offsets=np.zeros(q + 1, np.int64), syn_targets=np.zeros(0, np.int32))
    ranges, _ = shard.shard_ranges(q, 3)
    shs = [_NumpyShard(d, lo, hi, oracle.FIRST, 0) for lo, hi in ranges]
    done = shard.run(shs, 10, 0, _exchange(shs), lambda a: a)
    assert done == 1                                   # step 0 forgets every spike, step 1 is a fixed point
    assert shard.run(shs, 10, done, _exchange(shs), lambda a: a) == 0
    assert all((s_.sh.C[s_.sh.lo:s_.sh.hi] == 0).all() for s_ in shs)
