"""Parity at the full sizes of the skewed and batched workloads, in the
launch configuration the bench times, against the oracle on sampled steps
or sampled systems.

* skewed: 2,097,152 neurons, truncated Zipf(2.1) out-degree on [1, 4096],
  Philox; every state after steps 1, 2, 10 and 40 on the engine AUTO picks
  (the L2 gather), and after steps 1 and 8 on the tiled engine (four source
  partitions, several waves of CTAs).
* batch: all 8,192 systems (q log-uniform in 64..65,536) advanced 500 steps
  by one batch; 32 systems spread over the size range are compared in full
  with the oracle, and every system's executed step count is checked.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()


def _run_and_compare(d, engine, checkpoints, mode, seed):
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, engine=engine, seed=seed)
    st = oracle.initial_state(d)
    k = 0
    for target in checkpoints:
        n = target - k
        done = gs.step(n)
        ex, S = oracle.run(d, st, n, mode, seed, step0=k)
        assert done == ex, (target, done, ex)
        C, D, P, kk = gs.get_state()
        assert kk == k + ex
        assert (C == st[0]).all(), f"C differs after step {kk}"
        assert (D == st[1]).all(), f"D differs after step {kk}"
        assert (P == st[2]).all(), f"P differs after step {kk}"
        if ex:
            assert (gs.spiking() == S).all(), f"S differs after step {kk}"
        k += ex
        if ex < n:
            break
    info = gs.info()
    gs.close()
    return info


def test_skewed_2m_full_size_sampled():
    d, _, mode = synth.skewed_2m()
    # AUTO: the tiled engine in one wave of 4-CTA clusters with byte accumulators
    info = _run_and_compare(d, libsnp.SNP_ENGINE_AUTO, (1, 2, 10, 40), mode, d.seed)
    assert info.engine == libsnp.SNP_ENGINE_TILED
    info = _run_and_compare(d, libsnp.SNP_ENGINE_LAUNCH, (1, 8), mode, d.seed)
    assert info.engine == libsnp.SNP_ENGINE_LAUNCH


def test_batch_8k_full_size_sampled_systems():
    procs = max(1, min(16, os.cpu_count() or 1))
    descs, nsteps, mode = synth.batch_8k(processes=procs)
    assert len(descs) == 8192
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(procs) as ex:   # packing runs in the library, outside the GIL
        systems = list(ex.map(lambda d: libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=d.seed), descs))
    b = libsnp.Batch()
    t = b.submit(systems, [nsteps] * len(systems))
    done = b.wait(t)
    assert len(done) == len(systems)
    order = np.argsort([d.q for d in descs], kind="stable")
    picks = [int(order[i]) for i in np.linspace(0, len(order) - 1, 32).astype(int)]
    for i in picks:
        d = descs[i]
        st = oracle.initial_state(d)
        ex, S = oracle.run(d, st, nsteps, mode, d.seed)
        assert done[i] == ex, (i, d.q, done[i], ex)
        C, D, P, k = systems[i].get_state()
        assert k == ex
        assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all(), (i, d.q)
        if ex:
            assert (systems[i].spiking() == S).all(), (i, d.q)
    assert all(0 <= x <= nsteps for x in done)
    b.close()
    for g in systems:
        g.close()
