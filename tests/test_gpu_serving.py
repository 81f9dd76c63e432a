"""The served form: continuous batching with admission by device memory.

Checks that (1) every request's result is identical alone and in the mix
(and, for small ones, identical to the oracle); (2) requests that arrive
while others run are admitted and finish without waiting for the earlier
long ones; (3) the device memory held by the batch never exceeds its budget
while requests wait on the host for memory to free up.
"""
import time

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


def _requests(n, seed, q_range=(500, 120000), steps_range=(5, 300)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        q = int(np.exp(rng.uniform(np.log(q_range[0]), np.log(q_range[1]))))
        steps = int(np.exp(rng.uniform(np.log(steps_range[0]), np.log(steps_range[1]))))
        rules = int(rng.integers(2, 5))
        d = synth.random_system(q, 7000 + 13 * i + seed, outdeg=(2, 32), rules=(rules, rules), d_range=(0, 5),
                                spikes=(0, 20))
        out.append((d, steps, int(rng.integers(1, 2**62))))
    return out


def test_mix_equals_alone_and_oracle():
    reqs = _requests(24, 1)
    b = libsnp.Batch(mem_budget=8 << 30)
    systems, tickets = [], []
    for d, steps, seed in reqs:
        g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=seed, deferred=True)
        systems.append(g)
        tickets.append(b.submit([g], [steps]))
        time.sleep(0.002)   # arrivals spread over time, while earlier ones run
    for (d, steps, seed), g, t in zip(reqs, systems, tickets):
        done = b.wait(t)[0]
        alone = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=seed)
        assert alone.step(steps) == done
        a = alone.get_state()
        m = g.get_state()
        for x, y in zip(a[:3], m[:3]):
            assert (x == y).all()
        assert a[3] == m[3]
        assert (alone.spiking() == g.spiking()).all()
        if d.q <= 5000:
            st = oracle.initial_state(d)
            ex, S = oracle.run(d, st, steps, oracle.PHILOX, seed)
            assert ex == done and (st[0] == m[0]).all() and (st[1] == m[1]).all() and (st[2] == m[2]).all()
        alone.close()
        g.close()
    inf = b.info()
    assert inf.finished == len(reqs) and inf.waiting == 0 and inf.running == 0
    b.close()


def test_200_requests_against_oracle_and_alone():
    """A fixed subset of 200 served requests (q log-uniform in 300..20,000,
    3..120 steps, arrivals spread while earlier ones run): every request's
    result equals the oracle's and the same system stepped alone."""
    reqs = _requests(200, 9, q_range=(300, 20000), steps_range=(3, 120))
    b = libsnp.Batch(mem_budget=4 << 30)
    systems, tickets = [], []
    for d, steps, seed in reqs:
        g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=seed, deferred=True)
        systems.append(g)
        tickets.append(b.submit([g], [steps]))
        time.sleep(0.0005)
    for (d, steps, seed), g, t in zip(reqs, systems, tickets):
        done = b.wait(t)[0]
        m = g.get_state()
        st = oracle.initial_state(d)
        ex, S = oracle.run(d, st, steps, oracle.PHILOX, seed)
        assert ex == done and m[3] == ex
        assert (st[0] == m[0]).all() and (st[1] == m[1]).all() and (st[2] == m[2]).all()
        if ex:
            assert (g.spiking() == S).all()
        alone = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=seed)
        assert alone.step(steps) == done
        a = alone.get_state()
        assert all((x == y).all() for x, y in zip(a[:3], m[:3]))
        alone.close()
        g.close()
    inf = b.info()
    assert inf.finished == len(reqs) and inf.waiting == 0 and inf.running == 0
    b.close()


def test_late_short_request_overtakes_long_one():
    long_d = synth.random_system(400000, 5, outdeg=(8, 24), rules=(4, 4), d_range=(0, 5), spikes=(0, 20))
    short_d = synth.random_system(2000, 6, outdeg=(2, 32), rules=(3, 3), d_range=(0, 5), spikes=(0, 20))
    b = libsnp.Batch()
    gl = libsnp.System(long_d, select=libsnp.SNP_SELECT_PHILOX, seed=1, deferred=True)
    gs = libsnp.System(short_d, select=libsnp.SNP_SELECT_PHILOX, seed=2, deferred=True)
    tl = b.submit([gl], [40000])  # about half a second of device time
    time.sleep(0.05)
    ts = b.submit([gs], [20])
    b.wait(ts)
    assert not b.poll(tl), "the short request should finish while the long one still runs"
    b.wait(tl)
    b.close()


def test_admission_respects_memory_budget():
    reqs = _requests(16, 2, q_range=(20000, 60000), steps_range=(50, 120))
    sizes = []
    for d, _, _ in reqs:
        g = libsnp.System(d, deferred=True)
        sizes.append(g.info().device_bytes)
        g.close()
    budget = int(max(sizes) * 2.5)   # at most two or three requests resident at once
    b = libsnp.Batch(mem_budget=budget)
    systems = [libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=s, deferred=True) for d, _, s in reqs]
    tickets = [b.submit([g], [steps]) for g, (_, steps, _) in zip(systems, reqs)]
    peak_seen = 0
    pending = list(zip(tickets, systems))
    while pending:
        t, g = pending[0]
        if b.poll(t):
            C = g.config()
            assert C.shape[0] == g.q
            g.close()          # returns its memory to the batch
            pending.pop(0)
        inf = b.info()
        peak_seen = max(peak_seen, inf.resident_bytes)
        time.sleep(0.001)
    inf = b.info()
    assert inf.peak_resident_bytes <= budget
    assert peak_seen <= budget
    assert inf.finished == len(reqs)
    b.close()


def test_wait_reports_memory_held_by_finished_systems():
    """The budget is hard: a request that fits only once a finished system
    is destroyed is not admitted, and waiting on it reports SNP_ERR_BUSY
    instead of blocking forever; after the destroy it runs and matches the
    same system stepped alone."""
    d = synth.random_system(30000, 41, outdeg=(4, 16), rules=(3, 3), d_range=(0, 4), spikes=(0, 20))
    size = libsnp.System(d, deferred=True)
    budget = int(size.info().device_bytes * 1.5)   # room for one system, not two
    size.close()
    b = libsnp.Batch(mem_budget=budget)
    ga = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=1, deferred=True)
    gb = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=2, deferred=True)
    ta = b.submit([ga], [40])
    tb = b.submit([gb], [40])
    b.wait(ta)
    with pytest.raises(libsnp.SnpError) as ei:
        b.wait(tb)
    assert ei.value.status == libsnp.SNP_ERR_BUSY
    assert not b.poll(tb) and b.info().waiting == 1
    ga.close()
    done = b.wait(tb)[0]
    alone = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=2)
    assert alone.step(40) == done
    assert all((x == y).all() for x, y in zip(alone.get_state()[:3], gb.get_state()[:3]))
    assert b.info().peak_resident_bytes <= budget
    alone.close()
    gb.close()
    b.close()


def test_request_larger_than_budget_is_refused():
    d = synth.random_system(50000, 3, outdeg=(4, 16))
    g = libsnp.System(d, deferred=True)
    b = libsnp.Batch(mem_budget=1 << 20)
    with pytest.raises(libsnp.SnpError) as ei:
        b.submit([g], [10])
    assert ei.value.status == libsnp.SNP_ERR_OOM
    b.close()
