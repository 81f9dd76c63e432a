"""Rules whose expression is a finite union of a^k(a^j)* terms, on the GPU,
against the oracle: every form and engine, both selections, forced choices,
branch steps and batches.  rule_k/rule_j hold decoys that would make no rule
applicable, so a kernel that read the plain (k, j) instead of the union
would differ at once."""
import dataclasses
import itertools

import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth, tree

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


def union_system(q, seed, rules=(2, 4), terms=(1, 3), outdeg=(1, 8)):
    base = synth.random_system(q, seed, outdeg=outdeg, rules=rules, d_range=(0, 3), spikes=(0, 10))
    return synth.with_unions(base, seed + 1, terms=terms)


def compare(desc, nsteps, mode, seed, chunks=(1, 3, 7), compiled=1, **kw):
    gs = libsnp.System(desc, select=SEL[mode], seed=seed, **kw)
    assert gs.info().compiled_rules == compiled
    st = oracle.initial_state(desc)
    k, ci, last_S = 0, 0, np.full(desc.q, -1, np.int32)
    while k < nsteps:
        n = min(chunks[ci % len(chunks)], nsteps - k)
        ci += 1
        done = gs.step(n)
        ex, S = oracle.run(desc, st, n, mode, seed, step0=k)
        assert done == ex, (k, done, ex)
        if ex:
            last_S = S
        C, D, P, kk = gs.get_state()
        assert kk == k + ex
        assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all(), f"state differs after {k + ex}"
        assert (gs.spiking() == last_S).all(), f"S differs after {k + ex}"
        k += ex
        if ex < n:
            break
    info = gs.info()
    gs.close()
    return k, info


@pytest.mark.parametrize("engine", ["launch", "resident", "tiled", "auto"])
@pytest.mark.parametrize("q", [1, 33, 1000, 4099])
def test_unions_every_engine(engine, q):
    d = union_system(q, 700 + q)
    for mode in (oracle.FIRST, oracle.PHILOX):
        k, _ = compare(d, 40, mode, 31 + q, engine=ENGINES[engine])
        assert k > 0 or q == 1


@pytest.mark.parametrize("form,prop", [("ell", "pull"), ("ell", "push"), ("dense", "pull"), ("opt", "push")])
def test_unions_every_form(form, prop):
    forms = {"opt": libsnp.SNP_FORM_OPT, "ell": libsnp.SNP_FORM_ELL, "dense": libsnp.SNP_FORM_DENSE}
    props = {"pull": libsnp.SNP_PROP_PULL, "push": libsnp.SNP_PROP_PUSH}
    d = union_system(600, 811)
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 30, mode, 5, form=forms[form], prop=props[prop])


def test_unions_tiled_several_tiles():
    """200,000 neurons on the tiled engine (several source partitions and a
    ragged last slice), Philox, four terms per rule at most."""
    d = union_system(200_003, 905, rules=(3, 4), terms=(1, 4), outdeg=(4, 20))
    k, info = compare(d, 12, oracle.PHILOX, 77, chunks=(1, 5, 6), engine=libsnp.SNP_ENGINE_TILED)
    assert k == 12 and info.engine == libsnp.SNP_ENGINE_TILED


def test_unions_counts_forced_and_branch_step():
    d = union_system(2500, 913)
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
    st = oracle.initial_state(d)
    gs.step(4)
    oracle.run(d, st, 4)
    assert (gs.count_choices() == oracle.count_choices(d, st)).all()
    counts = oracle.count_choices(d, st)
    rng = np.random.default_rng(9)
    ch = (rng.integers(0, 1 << 30, size=d.q) % np.maximum(counts, 1)).astype(np.int32)
    gs.set_choices(ch)
    assert gs.step(3) == 3
    oracle.step(d, st, 4, oracle.FORCED, forced=ch)
    oracle.run(d, st, 2, step0=5)
    C, D, P, k = gs.get_state()
    assert k == 7 and (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all()
    # branch step over 64 reachable configurations
    states, s_ = [], oracle.initial_state(d)
    for k in range(64):
        oracle.run(d, s_, 1, oracle.PHILOX, 3, step0=k)
        states.append(tuple(x.copy() for x in s_))
    C = np.stack([x[0] for x in states]); D = np.stack([x[1] for x in states]); P = np.stack([x[2] for x in states])
    cnt0 = np.stack([oracle.count_choices(d, x) for x in states])
    ch = (rng.integers(0, 1 << 30, size=cnt0.shape) % np.maximum(cnt0, 1)).astype(np.int32)
    C1, D1, P1, ex, bad, cnt = gs.branch_step(C, D, P, ch)
    assert bad.sum() == 0
    for b, x in enumerate(states):
        s2 = tuple(v.copy() for v in x)
        halted = oracle.is_halted(d, s2[0], s2[2])
        if not halted:
            oracle.step(d, s2, 0, oracle.FORCED, forced=ch[b])
        assert ex[b] == (0 if halted else 1)
        assert (C1[b] == s2[0]).all() and (D1[b] == s2[1]).all() and (P1[b] == s2[2]).all(), b
        assert (cnt[b] == oracle.count_choices(d, s2)).all(), b
    gs.close()


def test_unions_tree_equals_oracle_branches():
    base = synth.random_system(5, 17, outdeg=(1, 3), rules=(2, 3), d_range=(0, 2), spikes=(1, 6))
    d = synth.with_unions(base, 18, terms=(1, 3), k_max=4, j_max=3)
    for batched in (False, True):
        t = tree.explore(d, 4, max_branches=4096, batched=batched, chunk=5)
        children = {}
        for parent, child, _ in t.edges:
            children.setdefault(parent, set()).add(child)
        for node, st in enumerate(t.states):
            if t.depth[node] >= 4:
                continue
            if oracle.is_halted(d, st[0], st[2]):
                assert node in t.halted
                continue
            counts = oracle.count_choices(d, st)
            want = set()
            for combo in itertools.product(*[range(max(1, int(c))) for c in counts]):
                s2 = tuple(x.copy() for x in st)
                oracle.step(d, s2, t.depth[node], oracle.FORCED, forced=np.asarray(combo, np.int32))
                want.add(tuple(tuple(int(v) for v in x) for x in s2))
            got = {tuple(tuple(int(v) for v in x) for x in t.states[c]) for c in children.get(node, ())}
            assert got == want


def test_unions_in_a_batch():
    descs = [union_system(int(q), 930 + i) for i, q in enumerate([64, 500, 3000, 9000, 40000])]
    systems = [libsnp.System(x, select=libsnp.SNP_SELECT_PHILOX, seed=i) for i, x in enumerate(descs)]
    b = libsnp.Batch()
    done = b.wait(b.submit(systems, [60] * len(systems)))
    for i, x in enumerate(descs):
        st = oracle.initial_state(x)
        ex, S = oracle.run(x, st, 60, oracle.PHILOX, i)
        C, D, P, k = systems[i].get_state()
        assert done[i] == ex and k == ex
        assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all(), i
    b.close()
    for g in systems:
        g.close()


def beyond_record(kind, q, seed):
    """Unions outside what a 16-byte compiled record holds, one limit each:
    more than 4 rules; a neuron whose term periods have lcm 35; c >= 64;
    p >= 32; d >= 32; periods and offsets of a few hundred (the divisibility
    test's generic path)."""
    rng = np.random.default_rng(seed)
    if kind == "rules6":
        return union_system(q, seed, rules=(5, 7))
    if kind == "lcm35":
        d = union_system(q, seed, rules=(2, 4), terms=(2, 3))
        tj = np.asarray(d.term_j).copy()
        tj[:] = np.where(np.arange(tj.size) % 2 == 0, 5, 7)       # every rule mixes j = 5 and j = 7
        return dataclasses.replace(d, term_j=tj.astype(np.int32))
    if kind == "c64":
        base = synth.random_system(q, seed, outdeg=(1, 8), rules=(2, 4), k_range=(60, 90), d_range=(0, 3),
                                   spikes=(40, 200))
        return synth.with_unions(base, seed + 1, terms=(1, 3), k_max=90, j_max=6)
    if kind == "p32":
        base = synth.random_system(q, seed, outdeg=(1, 8), rules=(2, 4), p_range=(20, 60), d_range=(0, 3),
                                   spikes=(0, 10))
        return synth.with_unions(base, seed + 1, terms=(1, 3))
    if kind == "d32":
        base = synth.random_system(q, seed, outdeg=(1, 8), rules=(2, 4), d_range=(0, 45), spikes=(0, 10))
        return synth.with_unions(base, seed + 1, terms=(1, 3))
    if kind == "j300":
        d = union_system(q, seed, rules=(2, 4), terms=(1, 3))
        T = np.asarray(d.term_j).size
        tj = rng.integers(1, 4, size=T).astype(np.int32)      # small periods keep rules applying
        big = rng.random(T) < 0.5
        tj[big] = rng.integers(250, 400, size=int(big.sum()))
        tk = rng.integers(0, 6, size=T).astype(np.int32)
        bk = rng.random(T) < 0.3
        tk[bk] = rng.integers(200, 300, size=int(bk.sum()))
        return dataclasses.replace(d, term_j=tj, term_k=tk,
                                   init_spikes=rng.integers(0, 320, size=q).astype(np.int32))
    raise ValueError(kind)


LIMITS = ["rules6", "lcm35", "c64", "p32", "d32", "j300"]


@pytest.mark.parametrize("kind", LIMITS)
@pytest.mark.parametrize("engine", ["launch", "resident", "tiled", "auto"])
def test_unions_beyond_the_record_every_engine(kind, engine):
    """Unions no compiled record holds run through the rule table's union
    records on every engine, element by element equal to the oracle."""
    q = 3001
    d = beyond_record(kind, q, 1200 + LIMITS.index(kind))
    for mode in (oracle.FIRST, oracle.PHILOX):
        k, info = compare(d, 40, mode, 17, compiled=0, engine=ENGINES[engine])
        assert k > 0
        assert info.compact_rules == 0


@pytest.mark.parametrize("kind", LIMITS)
@pytest.mark.parametrize("form,prop", [("ell", "pull"), ("ell", "push"), ("dense", "pull"), ("opt", "push")])
def test_unions_beyond_the_record_every_form(kind, form, prop):
    forms = {"opt": libsnp.SNP_FORM_OPT, "ell": libsnp.SNP_FORM_ELL, "dense": libsnp.SNP_FORM_DENSE}
    props = {"pull": libsnp.SNP_PROP_PULL, "push": libsnp.SNP_PROP_PUSH}
    d = beyond_record(kind, 700, 1300 + LIMITS.index(kind))
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 30, mode, 5, compiled=0, form=forms[form], prop=props[prop])


@pytest.mark.parametrize("kind", ["rules6", "lcm35", "c64"])
def test_unions_beyond_the_record_counts_branch_and_batch(kind):
    d = beyond_record(kind, 2000, 1400 + LIMITS.index(kind))
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
    assert gs.info().compiled_rules == 0
    st = oracle.initial_state(d)
    gs.step(3)
    oracle.run(d, st, 3)
    assert (gs.count_choices() == oracle.count_choices(d, st)).all()
    states, s_ = [], oracle.initial_state(d)
    for k in range(24):
        oracle.run(d, s_, 1, oracle.PHILOX, 3, step0=k)
        states.append(tuple(x.copy() for x in s_))
    C = np.stack([x[0] for x in states]); D = np.stack([x[1] for x in states]); P = np.stack([x[2] for x in states])
    rng = np.random.default_rng(2)
    cnt0 = np.stack([oracle.count_choices(d, x) for x in states])
    ch = (rng.integers(0, 1 << 30, size=cnt0.shape) % np.maximum(cnt0, 1)).astype(np.int32)
    C1, D1, P1, ex, bad, cnt = gs.branch_step(C, D, P, ch)
    for b, x in enumerate(states):
        s2 = tuple(v.copy() for v in x)
        if not oracle.is_halted(d, s2[0], s2[2]):
            oracle.step(d, s2, 0, oracle.FORCED, forced=ch[b])
        assert (C1[b] == s2[0]).all() and (D1[b] == s2[1]).all() and (P1[b] == s2[2]).all(), b
        assert (cnt[b] == oracle.count_choices(d, s2)).all(), b
    gs.close()
    descs = [beyond_record(kind, int(qq), 1500 + i) for i, qq in enumerate([64, 900, 7000, 30000])]
    systems = [libsnp.System(x, select=libsnp.SNP_SELECT_PHILOX, seed=i) for i, x in enumerate(descs)]
    b = libsnp.Batch()
    done = b.wait(b.submit(systems, [50] * len(systems)))
    for i, x in enumerate(descs):
        st = oracle.initial_state(x)
        ex_, _ = oracle.run(x, st, 50, oracle.PHILOX, i)
        Cg, Dg, Pg, kg = systems[i].get_state()
        assert done[i] == ex_ and kg == ex_
        assert (Cg == st[0]).all() and (Dg == st[1]).all() and (Pg == st[2]).all(), i
    b.close()
    for g in systems:
        g.close()
