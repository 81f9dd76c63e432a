"""GPU parity: the CUDA path through the C-ABI against the CPU oracle.

Bit-exact on every compared step: configuration C, spiking vector S (global
rule ids), delay status D and pending rules P, and the executed step count.
"""
import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ENGINES = {"launch": libsnp.SNP_ENGINE_LAUNCH, "resident": libsnp.SNP_ENGINE_RESIDENT,
           "tiled": libsnp.SNP_ENGINE_TILED, "auto": libsnp.SNP_ENGINE_AUTO}
SEL = {oracle.FIRST: libsnp.SNP_SELECT_FIRST, oracle.PHILOX: libsnp.SNP_SELECT_PHILOX}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()


def compare(desc, nsteps, mode, seed, *, engine="launch", prop=libsnp.SNP_PROP_PULL, chunks=(1,),
            check_every=True):
    """Steps the GPU system in chunks and compares with the oracle after each."""
    gs = libsnp.System(desc, select=SEL[mode], engine=ENGINES[engine], prop=prop, seed=seed)
    st = oracle.initial_state(desc)
    k = 0
    last_S = np.full(desc.q, -1, np.int32)
    ci = 0
    while k < nsteps:
        n = min(chunks[ci % len(chunks)], nsteps - k)
        ci += 1
        done = gs.step(n)
        ex, S = oracle.run(desc, st, n, mode, seed, step0=k)
        assert done == ex, (k, done, ex)
        if ex:
            last_S = S
        if check_every or k + n >= nsteps or ex < n:
            C, D, P, kk = gs.get_state()
            assert kk == k + ex
            assert (C == st[0]).all(), f"C differs after step {k + ex}"
            assert (D == st[1]).all(), f"D differs after step {k + ex}"
            assert (P == st[2]).all(), f"P differs after step {k + ex}"
            assert (gs.spiking() == last_S).all(), f"S differs after step {k + ex}"
        k += ex
        if ex < n:
            break
    gs.close()
    return k


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled"])
@pytest.mark.parametrize("q", [1, 2, 31, 32, 33, 100, 1000, 4099])
def test_ragged_sizes_every_step(engine, q):
    d = synth.random_system(q, 50 + q, outdeg=(1, 8), rules=(2, 4), d_range=(0, 3), spikes=(0, 10))
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 40, mode, 977 + q, engine=engine)


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled", "auto"])
def test_small_1k_workload_every_step(engine):
    d, nsteps, mode = synth.small_1k()
    compare(d, nsteps, mode, d.seed, engine=engine)


def test_small_1k_push_every_step():
    d, nsteps, mode = synth.small_1k()
    compare(d, nsteps, mode, d.seed, prop=libsnp.SNP_PROP_PUSH)
    compare(d, 60, oracle.PHILOX, 5, prop=libsnp.SNP_PROP_PUSH)


def _rule_shape(name):
    """Rule tables on both sides of the compiled-record limits (at most four
    rules per neuron, K + L <= 14, c < 64, p < 32, d < 32)."""
    if name == "compiled_edge":
        # k <= 5 and j in {0, 1, 2, 4, 8}: K <= 6, L <= 8, K + L up to 14
        d = synth.random_system(6000, 11, outdeg=(2, 12), rules=(2, 4), k_range=(1, 5), d_range=(0, 6),
                                spikes=(0, 3000))
        fire = d.rule_j > 0
        rng = np.random.default_rng(12)
        d.rule_j[:] = np.where(fire | (d.rule_p > 0), rng.choice([0, 1, 2, 4, 8], size=d.rule_j.size), 0)
        return d, True
    if name == "wide_k":
        return synth.random_system(6000, 13, outdeg=(2, 12), rules=(2, 4), k_range=(1, 12), j_range=(0, 7),
                                   d_range=(0, 6), spikes=(0, 3000)), False
    if name == "many_rules":
        return synth.random_system(6000, 14, outdeg=(2, 12), rules=(5, 6), d_range=(0, 4), spikes=(0, 40)), False
    if name == "long_delay":
        return synth.random_system(6000, 15, outdeg=(2, 12), rules=(3, 4), d_range=(0, 40), spikes=(0, 40)), False
    raise ValueError(name)


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled"])
@pytest.mark.parametrize("shape", ["compiled_edge", "wide_k", "many_rules", "long_delay"])
def test_compiled_rule_records_and_fallback(engine, shape):
    d, compiled = _rule_shape(shape)
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, engine=ENGINES[engine])
    assert gs.info().compiled_rules == int(compiled)
    gs.close()
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 48, mode, 31 + len(shape), engine=engine, check_every=False, chunks=(7, 13))


@pytest.mark.parametrize("outdeg,paired", [((1, 2), False), ((12, 24), True)])
def test_tiled_paired_and_run_layouts(outdeg, paired):
    """The tiled gather pads each target's in-edges to pairs only when that
    adds at most 1/8 of the words; low in-degree systems keep the run-merging
    layout.  One system of each kind (one source partition at this size)."""
    d = synth.random_system(50000, 21 + outdeg[0], outdeg=outdeg, rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    indeg = np.bincount(d.syn_targets, minlength=d.q)
    odd_frac = float((indeg & 1).sum()) / d.num_syn
    assert (odd_frac <= 0.125) == paired
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 40, mode, 5 + outdeg[0], engine="tiled", check_every=False, chunks=(9, 31))


@pytest.mark.parametrize("q,outdeg", [(400000, (4, 8)), (1 << 20, (2, 6))])
def test_tiled_cluster_sizes_and_two_launch_form(q, outdeg):
    """16-bit emissions (p up to 1000) cut the sources into several
    partitions: 400k neurons -> a cluster of several CTAs per range (one
    launch per step); 1M neurons -> more partitions than a cluster holds,
    the two-launch form with in-flow arrays."""
    d = synth.random_system(q, 90 + outdeg[1], outdeg=outdeg, rules=(3, 4), p_range=(1, 1000), d_range=(0, 5),
                            spikes=(0, 20))
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 8, mode, 17, engine="tiled", check_every=False, chunks=(3, 5))


@pytest.mark.parametrize("p_max", [3, 15])
def test_tiled_run_length_layout(p_max):
    """Long runs of in-edges per CTA thread (600k neurons, out-degree
    8..24) take the run-length layout: 24-bit entries (the source's bit
    index in the packed emissions, then the target advance), the target
    carried as a running offset; 2-bit emissions in one source partition,
    4-bit ones (p up to 15) in two."""
    d = synth.random_system(600000, 66 if p_max == 3 else 67, outdeg=(8, 24), rules=(3, 4), p_range=(1, p_max),
                            d_range=(0, 5), spikes=(0, 20))
    gs = libsnp.System(d, engine=libsnp.SNP_ENGINE_TILED)
    info = gs.info()
    gs.close()
    assert info.e_bits == (2 if p_max == 3 else 4)
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 12, mode, 29, engine="tiled", check_every=False, chunks=(1, 4, 7))


def test_auto_engine_choice():
    """AUTO: CTA-resident for small systems; tiled for one wave of tiled
    clusters (the 2M-neuron Zipf system with byte accumulators in 4-CTA
    clusters); the L2 gather for a large low-degree system whose in-flows
    need 32-bit accumulators (p up to 100), where the tiled layout takes
    several waves whose emission copies outweigh the entry stream; every
    choice matches the oracle."""
    cases = [(synth.random_system(3000, 61, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20)),
              libsnp.SNP_ENGINE_RESIDENT),
             (synth.random_system(200000, 62, outdeg=(8, 24), rules=(3, 4), d_range=(0, 5), spikes=(0, 20)),
              libsnp.SNP_ENGINE_TILED),
             (synth.random_system(1 << 21, 63, zipf=(2.1, 1, 4096), rules=(3, 3), d_range=(0, 3), spikes=(0, 20)),
              libsnp.SNP_ENGINE_TILED),
             (synth.random_system(1 << 21, 64, zipf=(2.1, 1, 4096), rules=(3, 3), p_range=(1, 100), d_range=(0, 3),
                                  spikes=(0, 20)),
              libsnp.SNP_ENGINE_LAUNCH)]
    for d, want in cases:
        gs = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=3)
        assert gs.info().engine == want, (d.q, gs.info().engine)
        done = gs.step(6)
        st = oracle.initial_state(d)
        ex, _ = oracle.run(d, st, 6, oracle.PHILOX, 3)
        C, D, P, _ = gs.get_state()
        assert done == ex and (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all()
        gs.close()


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled"])
def test_chunked_calls_and_graphs(engine):
    """Calls of many sizes (crossing the captured-graph chunk length)."""
    d = synth.random_system(3000, 99, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    compare(d, 400, oracle.PHILOX, 4242, engine=engine, chunks=(1, 7, 48, 49, 100, 3), check_every=True)


def test_push_matches_with_delays_and_skew():
    d = synth.random_system(20000, 5, zipf=(2.1, 1, 4096), rules=(3, 3), d_range=(0, 3), spikes=(0, 20))
    compare(d, 60, oracle.PHILOX, 31, prop=libsnp.SNP_PROP_PUSH, chunks=(1, 10, 49))
    compare(d, 60, oracle.PHILOX, 31, chunks=(1, 10, 49))


def test_sort_system_sorts():
    for v in ([3, 2, 1], [5, 1, 4, 4, 2], list(range(40, 0, -1))):
        d = synth.sort_system(v)
        for eng in ("launch", "resident", "tiled"):
            n = compare(d, 1000, oracle.FIRST, 0, engine=eng, chunks=(1, 50))
            assert n == max(v) + 1
        gs = libsnp.System(d)
        gs.step(1000)
        assert gs.config()[2 * len(v):].tolist() == sorted(v)


def test_hand_delay_traces():
    from tests.test_oracle import make_desc
    cases = [
        make_desc(2, [[(1, 0, 1, 1, 3)], []], [(0, 1)], [1, 0]),
        make_desc(3, [[(1, 0, 1, 1, 2)], [], [(1, 0, 1, 1, 0)]], [(2, 0), (0, 1)], [1, 0, 1]),
        make_desc(4, [[(1, 0, 1, 1, 1)], [], [(2, 0, 2, 1, 0)], [(1, 0, 1, 1, 0)]],
                  [(0, 1), (2, 0), (3, 2)], [1, 0, 1, 1]),
    ]
    for d in cases:
        for eng in ("launch", "resident", "tiled"):
            compare(d, 20, oracle.FIRST, 0, engine=eng)
        compare(d, 20, oracle.FIRST, 0, prop=libsnp.SNP_PROP_PUSH)


def test_checkpoint_resume_is_bit_exact():
    d = synth.random_system(5000, 3, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    a = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=77)
    a.step(60)
    ref = a.get_state()
    b = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=77)
    b.step(30)
    C, D, P, k = b.get_state()
    c = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=77, engine=libsnp.SNP_ENGINE_RESIDENT)
    c.set_state(C, D, P, k)
    c.step(30)
    got = c.get_state()
    for x, y in zip(ref[:3], got[:3]):
        assert (x == y).all()
    assert ref[3] == got[3] == 60


@pytest.mark.parametrize("where", ["numpy", "pinned", "device"])
@pytest.mark.parametrize("kw", [dict(engine=libsnp.SNP_ENGINE_LAUNCH), dict(engine=libsnp.SNP_ENGINE_TILED),
                                dict(engine=libsnp.SNP_ENGINE_RESIDENT), dict(prop=libsnp.SNP_PROP_PUSH),
                                dict(form=libsnp.SNP_FORM_ELL)], ids=["launch", "tiled", "resident", "push", "ell"])
def test_set_state_from_host_and_device_memory(kw, where):
    """snp_set_state checks and permutes the state on the device: resuming
    from a checkpoint held in pageable, pinned or device memory continues
    bit for bit on every engine and form."""
    d = synth.random_system(6000, 13, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    a = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=5)
    a.step(40)
    ref = a.get_state()
    ref_S = a.spiking()
    b = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=5)
    b.step(17)
    C, D, P, k = b.get_state()
    if where == "pinned":
        C, D, P = (torch.from_numpy(x).pin_memory() for x in (C, D, P))
    elif where == "device":
        C, D, P = (torch.from_numpy(x).cuda() for x in (C, D, P))
    c = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=5, **kw)
    c.step(3)
    c.set_state(C, D, P, k)
    assert (c.spiking() == -1).all()
    got0 = c.get_state()
    assert all((np.asarray(x.cpu() if hasattr(x, "cpu") else x) == y).all() for x, y in zip((C, D, P), got0[:3]))
    assert got0[3] == 17
    assert c.step(23) == 23
    got = c.get_state()
    for x, y in zip(ref[:3], got[:3]):
        assert (x == y).all()
    assert ref[3] == got[3] == 40
    assert (c.spiking() == ref_S).all()
    for g in (a, b, c):
        g.close()


def test_set_state_rejects_bad_values_and_keeps_the_state():
    d = synth.random_system(3000, 14, outdeg=(4, 16), rules=(3, 3), d_range=(1, 5), spikes=(0, 20))
    g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=9)
    g.step(11)
    C, D, P, k = g.get_state()
    pend = np.flatnonzero(P >= 0)
    idle = np.flatnonzero(P == -1)
    assert len(pend) and len(idle)
    i, j = int(pend[len(pend) // 2]), int(idle[len(idle) // 2])
    r_other = int(d.rule_offsets[j])   # a rule of another neuron
    bad_cases = [("C", j, -1, "negative spike count at neuron %d" % j),
                 ("D", i, 70000, "D out of range at neuron %d" % i),
                 ("D", j, 2, "D > 0 without a pending rule at neuron %d" % j),
                 ("P", i, r_other, "pending rule does not belong to neuron %d" % i)]
    for name, at, val, msg in bad_cases:
        arrs = {"C": C.copy(), "D": D.copy(), "P": P.copy()}
        arrs[name][at] = val
        with pytest.raises(libsnp.SnpError) as ei:
            g.set_state(arrs["C"], arrs["D"], arrs["P"], 99)
        assert ei.value.status == libsnp.SNP_ERR_INVALID
        assert msg in str(ei.value)
        C2, D2, P2, k2 = g.get_state()
        assert (C2 == C).all() and (D2 == D).all() and (P2 == P).all() and k2 == k
    # two bad neurons: the smaller id is reported
    lo, hi = sorted((i, j))
    arrs = {"C": C.copy(), "D": D.copy(), "P": P.copy()}
    arrs["C"][lo] = -3
    arrs["C"][hi] = -4
    with pytest.raises(libsnp.SnpError) as ei:
        g.set_state(arrs["C"], arrs["D"], arrs["P"], 99)
    assert "at neuron %d" % lo in str(ei.value)
    # still steps exactly like an untouched copy
    h = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=9)
    h.step(11)
    assert g.step(9) == h.step(9)
    assert all((x == y).all() for x, y in zip(g.get_state()[:3], h.get_state()[:3]))
    g.close()
    h.close()


def test_device_outputs_and_stream():
    d = synth.random_system(3000, 8, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    s = torch.cuda.Stream()
    g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=3, stream=s)
    g.step(25, wait=False)
    out = torch.empty(d.q, dtype=torch.int32, device="cuda")
    g.config(out)
    s.synchronize()
    st = oracle.initial_state(d)
    oracle.run(d, st, 25, oracle.PHILOX, 3)
    assert (out.cpu().numpy() == st[0]).all()


def test_overflow_is_reported():
    from tests.test_oracle import make_desc
    d = make_desc(2, [[(1, 1, 1, 1000, 0)], []], [(0, 1)], [10, 2**31 - 600])
    for eng in (libsnp.SNP_ENGINE_LAUNCH, libsnp.SNP_ENGINE_RESIDENT, libsnp.SNP_ENGINE_TILED):
        g = libsnp.System(d, engine=eng)
        with pytest.raises(libsnp.SnpError) as ei:
            g.step(5)
        assert ei.value.status == libsnp.SNP_ERR_OVERFLOW


def test_in_flow_beyond_int32_from_one_partition():
    """40,000 neurons each send 60,000 spikes to one hub in the same step
    (2.4e9 > INT32_MAX).  The tiled engine, whose per-partition shared
    accumulators are 32-bit, refuses the system; AUTO and the other engines
    report the overflow, as the oracle does."""
    import oracle as orc
    n = 40000
    q = n + 1
    ones = np.ones(n, np.int32)
    offs = np.concatenate([[0], np.arange(n + 1)]).astype(np.int64)   # neuron 0: no rule, no synapse
    d = synth.SystemDesc(q=q, init_spikes=np.concatenate([[0], ones]).astype(np.int32), rule_offsets=offs,
                         rule_k=ones, rule_j=0 * ones, rule_c=ones, rule_p=60000 * ones, rule_d=0 * ones,
                         syn_offsets=offs, syn_targets=0 * ones)
    with pytest.raises(orc.OracleOverflow):
        orc.run(d, orc.initial_state(d), 2)
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.System(d, engine=libsnp.SNP_ENGINE_TILED)
    assert ei.value.status == libsnp.SNP_ERR_UNSUPPORTED
    for eng in (libsnp.SNP_ENGINE_AUTO, libsnp.SNP_ENGINE_LAUNCH):
        g = libsnp.System(d, engine=eng)
        assert g.info().engine != libsnp.SNP_ENGINE_TILED
        with pytest.raises(libsnp.SnpError) as ei:
            g.step(2)
        assert ei.value.status == libsnp.SNP_ERR_OVERFLOW
        g.close()


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled"])
def test_compiled_records_at_huge_spike_counts(engine):
    """Spike counts spread up to 2^31 - 100 with periodic rules (period 2..7
    per neuron, so every neuron compiles): the compiled table's index
    K + (n - K) mod L is taken for counts far above any the other tests
    reach; the chosen rules and the state match the oracle."""
    rng = np.random.default_rng(44)
    q = 4096
    offs, ks, js, cs, ps, ds = [0], [], [], [], [], []
    for _ in range(q):
        j = int(rng.integers(2, 8))
        for _ in range(3):
            k = int(rng.integers(0, 6))
            ks.append(k); js.append(j); cs.append(int(rng.integers(0, k + 1)))
            ps.append(int(rng.integers(1, 4))); ds.append(int(rng.integers(0, 3)))
        offs.append(len(ks))
    a32 = lambda x: np.asarray(x, np.int32)
    init = rng.integers(0, 2**31 - 100, size=q)
    init[:64] = np.arange(64)                         # and the smallest counts
    d = synth.SystemDesc(q=q, init_spikes=a32(init), rule_offsets=np.asarray(offs, np.int64), rule_k=a32(ks),
                         rule_j=a32(js), rule_c=a32(cs), rule_p=a32(ps), rule_d=a32(ds),
                         syn_offsets=np.zeros(q + 1, np.int64), syn_targets=a32([]))
    g = libsnp.System(d, engine=ENGINES[engine])
    assert g.info().compiled_rules == 1
    g.close()
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 6, mode, 91, engine=engine)


def test_halted_system_reports_zero_steps():
    from tests.test_oracle import make_desc
    d = make_desc(3, [[], [(2, 0, 2, 1, 0)], []], [(1, 0)], [5, 1, 0])
    for eng in ("launch", "resident", "tiled"):
        g = libsnp.System(d, engine=ENGINES[eng])
        assert g.step(10) == 0
        assert g.config().tolist() == [5, 1, 0]
        assert (g.spiking() == -1).all()


def test_batch_matches_alone_and_oracle():
    rng = np.random.default_rng(11)
    sizes = synth.batch_sizes(rng, 48, 64, 6000)
    descs = [synth.random_system(int(q), 1000 + i, outdeg=(4, 16), rules=(3, 3), d_range=(0, 4),
                                 spikes=(0, 10)) for i, q in enumerate(sizes)]
    steps = [int(x) for x in rng.integers(1, 120, size=len(descs))]
    systems = [libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=d.seed) for d in descs]
    b = libsnp.Batch()
    t = b.submit(systems, steps)
    done = b.wait(t)
    for d, g, n, dn in zip(descs, systems, steps, done):
        st = oracle.initial_state(d)
        ex, S = oracle.run(d, st, n, oracle.PHILOX, d.seed)
        assert dn == ex
        C, D, P, k = g.get_state()
        assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all() and k == ex
        if ex:
            assert (g.spiking() == S).all()
        alone = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=d.seed, engine=libsnp.SNP_ENGINE_LAUNCH)
        alone.step(n)
        assert (alone.config() == C).all()
    b.close()


def test_busy_system_is_refused_during_batch():
    d = synth.random_system(60000, 1, outdeg=(8, 24), rules=(4, 4), d_range=(0, 5), spikes=(0, 20))
    g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=1)
    b = libsnp.Batch()
    t = b.submit([g], [300])
    if not b.poll(t):
        with pytest.raises(libsnp.SnpError) as ei:
            g.step(1)
        assert ei.value.status == libsnp.SNP_ERR_BUSY
    b.wait(t)
    g.step(1)
    b.close()


@pytest.mark.parametrize("p_range,q", [((1, 15), 70000), ((1, 200), 90000), ((1, 1000), 120000)])
def test_tiled_emission_widths_and_partitions(p_range, q):
    """4-, 8- and 16-bit packed emissions; the 16-bit case needs two source
    partitions (the partial sums wait in shared memory)."""
    d = synth.random_system(q, 77 + q, outdeg=(4, 16), rules=(3, 4), p_range=p_range, d_range=(0, 5),
                            spikes=(0, 20))
    g = libsnp.System(d, engine=libsnp.SNP_ENGINE_TILED)
    inf = g.info()
    assert inf.e_bits == {15: 4, 200: 8, 1000: 16}[p_range[1]]
    g.close()
    compare(d, 25, oracle.PHILOX, 5, engine="tiled", chunks=(1, 24))


def test_large_1m_full_size_sampled():
    """The 1,048,576-neuron workload in the launch configuration the bench
    times (tiled engine, two source partitions, Philox selection): every
    state is compared after steps 1, 2, 3, 10, 58 and 150; the L2-gather
    engine after steps 1 and 49."""
    d, _, mode = synth.large_1m()
    g = libsnp.System(d, engine=libsnp.SNP_ENGINE_TILED)
    assert g.info().e_bits == 2
    g.close()
    compare(d, 150, mode, d.seed, engine="tiled", chunks=(1, 1, 1, 7, 48, 92))
    compare(d, 49, mode, d.seed, engine="launch", chunks=(1, 48))
