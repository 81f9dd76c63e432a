"""The bench's multi-rank plumbing on CPU with gloo, world size 2.

Independent systems shard across ranks with no data-path collective; the
only collectives are the barrier around the timed region and the max/sum
reductions of the timing and the work.  These run here on the gloo backend.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert (w, r) == (ws, rank)
    bench.barrier(w)
    mx = bench.max_over_ranks(w, float(rank + 1) * 1.5)
    sm = bench.sum_over_ranks(w, float(rank + 1))
    out.put((rank, mx, sm))
    dist.destroy_process_group()


def test_rank_reductions_gloo_world2():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res == [(0, 3.0, 3.0), (1, 3.0, 3.0)]


def test_reference_arm_under_torchrun_two_ranks():
    """`bench.py --impl reference` launched as the driver launches N > 1:
    rank 0 alone runs the oracle and prints one JSON line, rank 1 exits 0."""
    pytest.importorskip("torch")
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, PYTHONPATH=ROOT)
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    assert j["impl"] == "reference" and j["n_gpus"] == 2 and j["value"] > 0
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["cpu_baseline"]["kind"] == "oracle"


def _shard_worker(rank, ws, port, out, mode, seed, nsteps):
    """One rank of a system split by neuron range: this rank's neurons run the
    definition's two phases (the oracle's range phases, test infrastructure),
    the emission slices travel by an in-place all_gather over gloo, the
    activity by an all_reduce; the protocol is paper_2408_04343_gb300.shard."""
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import numpy as np
    import torch
    import torch.distributed as dist
    import oracle
    from paper_2408_04343_gb300 import shard, synth
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    d = _shard_system()
    ranges, chunk = shard.shard_ranges(d.q, ws)
    lo, hi = ranges[rank]
    E = torch.zeros(ws * chunk + 1, dtype=torch.int32)
    sh = oracle.RangeShard(d, lo, hi)
    sh.E = E.numpy()[:d.q]           # the shard's emission vector is the exchanged tensor

    class Local:
        def select(self, k):
            return sh.select(k, mode, seed)

        def receive(self):
            sh.receive()

    ex, any_active = shard.collective_exchange(E, rank, ws, chunk)
    done = shard.run([Local()], nsteps, 0, ex, any_active)
    # gather every rank's slice of the state
    parts = []
    for arr in (sh.C, sh.D, sh.P):
        mine = torch.zeros(chunk, dtype=torch.int32)
        mine[:hi - lo] = torch.from_numpy(arr[lo:hi].copy())
        allp = [torch.zeros(chunk, dtype=torch.int32) for _ in range(ws)]
        dist.all_gather(allp, mine)
        parts.append(torch.cat(allp)[:d.q].numpy())
    out.put((rank, done, [p.tolist() for p in parts]))
    dist.destroy_process_group()


def _shard_system():
    import numpy as np
    sys.path.insert(0, ROOT)
    from paper_2408_04343_gb300 import synth
    return synth.random_system(2500, 77, outdeg=(2, 12), rules=(2, 4), d_range=(0, 3), spikes=(0, 12))


@pytest.mark.parametrize("mode_name", ["first", "philox"])
def test_sharded_step_gloo_world2_matches_the_oracle(mode_name):
    """A system split by neuron range over two gloo ranks on CPU: phase 1 on
    each rank, the emission slices all-gathered, the activity all-reduced,
    phase 2 on each rank (the protocol of shard.py that the CUDA shards
    follow) gives the whole system's oracle result bit for bit."""
    torch = pytest.importorskip("torch")
    import numpy as np
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    mode, seed, nsteps = (oracle.FIRST if mode_name == "first" else oracle.PHILOX), 4242, 40
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q, mode, seed, nsteps)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    d = _shard_system()
    st = oracle.initial_state(d)
    ex, _ = oracle.run(d, st, nsteps, mode, seed)
    for rank, done, (C, D, P) in res:
        assert done == ex
        assert (np.asarray(C) == st[0]).all() and (np.asarray(D) == st[1]).all() and (np.asarray(P) == st[2]).all()
