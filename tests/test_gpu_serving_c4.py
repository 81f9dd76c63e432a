"""Served-form parity on the serving workload's own distribution.

A fixed subset of 200 requests drawn exactly as the serving workload draws
them: Poisson arrivals (100 requests/s), each request its own system with q
log-uniform in [1e3, 1e6], a step count log-uniform in [10, 1e4], out-degree
U{2..32}, 2-4 rules per neuron, d in [0, 5], spikes U[0, 20], Philox keyed by
the request's own seed.  They are submitted at their arrival times to one
batch under a 150 GB device-memory budget, so small requests share the
persistent resident launch while large ones (q > 65,536) run concurrently
on the grid-wide engines.  Every request's executed step count, C, D, P and
S must equal (1) the same system stepped alone with snp_step and (2) the
CPU oracle (its pull form, pinned step by step to the definition), element
by element.
"""
import os
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

RATE_PER_S = 100.0
SUBSET_SEED = 5012     # the fixed subset: 200 requests, 76 with q > 65,536, 48 with > 1,000 steps
N_REQUESTS = 200


@pytest.fixture(scope="module")
def requests_and_systems():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()
    reqs = synth.serving_requests(RATE_PER_S, N_REQUESTS, seed=SUBSET_SEED)
    descs = synth.serving_systems(reqs, processes=min(16, os.cpu_count() or 1))
    return reqs, descs


def test_subset_covers_the_large_and_long_paths(requests_and_systems):
    reqs, _ = requests_and_systems
    assert sum(r.q > 65536 for r in reqs) >= 50            # grid-wide engines beside the resident launch
    assert sum(r.steps > 1000 for r in reqs) >= 30
    assert any(r.q > 500_000 and r.steps > 3000 for r in reqs)
    assert min(r.q for r in reqs) >= 1000 and max(r.q for r in reqs) <= 1_000_000


def test_served_equals_alone_equals_oracle(requests_and_systems):
    reqs, descs = requests_and_systems
    sel = libsnp.SNP_SELECT_PHILOX
    with ThreadPoolExecutor(8) as ex:
        systems = list(ex.map(lambda i: libsnp.System(descs[i], select=sel, seed=reqs[i].seed, deferred=True),
                              range(len(reqs))))
    b = libsnp.Batch(mem_budget=150 << 30)
    t0 = time.perf_counter()
    tickets = []
    for r, g in zip(reqs, systems):     # Poisson arrivals: submit at each request's arrival time
        dt = t0 + (r.arrival_s - reqs[0].arrival_s) - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        tickets.append(b.submit([g], [r.steps]))
    served = []
    for r, g, t in zip(reqs, systems, tickets):
        done = b.wait(t)[0]
        C, D, P, k = g.get_state()
        served.append((done, C, D, P, g.spiking(), k))
        g.close()                       # returns its memory to the batch
    inf = b.info()
    assert inf.finished == len(reqs) and inf.waiting == 0 and inf.running == 0
    assert inf.peak_resident_bytes <= 150 << 30
    b.close()
    long_large = 0
    for i, (r, d) in enumerate(zip(reqs, descs)):
        done, C, D, P, S, k = served[i]
        assert k == done, i
        # alone: the same system and seed stepped by snp_step, outside any batch
        alone = libsnp.System(d, select=sel, seed=r.seed)
        assert alone.step(r.steps) == done, i
        aC, aD, aP, ak = alone.get_state()
        assert ak == k and (aC == C).all() and (aD == D).all() and (aP == P).all(), i
        assert (alone.spiking() == S).all(), i
        alone.close()
        # the oracle
        st = oracle.initial_state(d)
        ex, oS = oracle.PullRunner(d).run(st, r.steps, oracle.PHILOX, r.seed)
        assert ex == done, (i, ex, done)
        assert (st[0] == C).all() and (st[1] == D).all() and (st[2] == P).all(), i
        if ex:
            assert (oS == S).all(), i
        long_large += r.q > 65536 and done > 1000
    assert long_large >= 5      # requests that ran long on the grid-wide engines, compared in full
