"""Computation-tree exploration on the GPU: snp_count_choices,
snp_set_choices and paper_2408_04343_gb300.tree.explore against the
oracle's forced-choice step (its FORCED mode) and its choice counts."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth, tree

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ENGINES = {"launch": libsnp.SNP_ENGINE_LAUNCH, "resident": libsnp.SNP_ENGINE_RESIDENT,
           "tiled": libsnp.SNP_ENGINE_TILED}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()


def tiny(seed, q):
    """A tiny random system with delays and overlapping rules (branching)."""
    rng = np.random.default_rng(seed)
    offs, ks, js, cs, ps, ds = [0], [], [], [], [], []
    for _ in range(q):
        for _ in range(int(rng.integers(1, 4))):
            k = int(rng.integers(1, 4)); j = int(rng.integers(0, 3))
            c = int(rng.integers(1, k + 1)); p = int(rng.integers(0, 3))
            ks.append(k); js.append(j); cs.append(c); ps.append(p)
            ds.append(int(rng.integers(0, 3)) if p > 0 else 0)
        offs.append(len(ks))
    out = [[b for b in range(q) if b != a and rng.random() < 0.5] for a in range(q)]
    so = np.zeros(q + 1, np.int64)
    so[1:] = np.cumsum([len(o) for o in out])
    a32 = lambda x: np.asarray(x, np.int32)
    return synth.SystemDesc(q=q, init_spikes=a32(rng.integers(1, 7, size=q)), rule_offsets=np.asarray(offs, np.int64),
                            rule_k=a32(ks), rule_j=a32(js), rule_c=a32(cs), rule_p=a32(ps), rule_d=a32(ds),
                            syn_offsets=so, syn_targets=a32([x for o in out for x in o]))


def oracle_children(d, st, k):
    """Every child of configuration st under the oracle's forced step."""
    counts = oracle.count_choices(d, st)
    if oracle.is_halted(d, st[0], st[2]):
        return None
    kids = set()
    for combo in itertools.product(*[range(max(1, int(c))) for c in counts]):
        s2 = tuple(x.copy() for x in st)
        oracle.step(d, s2, k, oracle.FORCED, forced=np.asarray(combo, np.int32))
        kids.add(tuple(tuple(int(v) for v in x) for x in s2))
    return kids


@pytest.mark.parametrize("mode", ["launch", "resident", "tiled", "batched"])
@pytest.mark.parametrize("seed", range(4))
def test_explored_tree_equals_oracle_branches(mode, seed):
    """Per-branch forced steps on each engine, and the batched branch step
    (one launch per level), give every configuration's children exactly as
    the oracle's forced step enumerates them."""
    d = tiny(300 + seed, q=4 + seed % 3)
    if mode == "batched":
        t = tree.explore(d, 4, max_branches=4096, batched=True, chunk=7)
    else:
        t = tree.explore(d, 4, max_branches=4096, engine=ENGINES[mode], batched=False)
    assert not t.truncated
    children = {}
    for parent, child, _ in t.edges:
        children.setdefault(parent, set()).add(child)
    for node, st in enumerate(t.states):
        if t.depth[node] >= 4:
            continue
        want = oracle_children(d, st, t.depth[node])
        if want is None:
            assert node in t.halted and node not in children
            continue
        got = {tuple(tuple(int(v) for v in x) for x in t.states[c]) for c in children.get(node, ())}
        assert got == want, (node, t.depth[node])


@pytest.mark.parametrize("engine", list(ENGINES))
def test_counts_forced_first_step_and_invalid_index(engine):
    d = synth.random_system(3000, 17, outdeg=(2, 8), rules=(3, 4), d_range=(0, 3), spikes=(0, 12))
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST, engine=ENGINES[engine])
    st = oracle.initial_state(d)
    gs.step(3)
    oracle.run(d, st, 3)
    assert (gs.count_choices() == oracle.count_choices(d, st)).all()
    # a forced first step, then first-applicable steps
    counts = oracle.count_choices(d, st)
    rng = np.random.default_rng(5)
    choice = (rng.integers(0, 1 << 30, size=d.q) % np.maximum(counts, 1)).astype(np.int32)
    gs.set_choices(choice)
    assert gs.step(6) == 6
    oracle.step(d, st, 3, oracle.FORCED, forced=choice)
    oracle.run(d, st, 5, step0=4)
    C, D, P, k = gs.get_state()
    assert k == 9 and (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all()
    # an index beyond a neuron's choices is refused after the step
    bad = np.zeros(d.q, np.int32)
    counts = gs.count_choices()
    i = int(np.nonzero(counts > 0)[0][0])
    bad[i] = counts[i]
    gs.set_choices(bad)
    with pytest.raises(libsnp.SnpError) as ei:
        gs.step(1)
    assert ei.value.status == libsnp.SNP_ERR_INVALID
    assert gs.step(1) == 1      # the next call selects as usual
    gs.close()


def test_branch_step_matches_oracle_on_many_configurations():
    """snp_branch_step on 300 configurations of a 2,000-neuron system with
    delays (random reachable states, random valid choices): every result,
    executed flag and next-level count equals the oracle's; an invalid index
    is reported per configuration; the system's own state is untouched."""
    d = synth.random_system(2000, 23, outdeg=(2, 10), rules=(2, 4), d_range=(0, 3), spikes=(0, 12))
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
    rng = np.random.default_rng(4)
    states = []
    st = oracle.initial_state(d)
    for k in range(300):
        oracle.run(d, st, 1, oracle.PHILOX, 9, step0=k)
        states.append(tuple(x.copy() for x in st))
    C = np.stack([s_[0] for s_ in states]); D = np.stack([s_[1] for s_ in states]); P = np.stack([s_[2] for s_ in states])
    counts = np.stack([oracle.count_choices(d, s_) for s_ in states])
    ch = (rng.integers(0, 1 << 30, size=counts.shape) % np.maximum(counts, 1)).astype(np.int32)
    ch[7, int(np.nonzero(counts[7] > 0)[0][0])] = 99     # one invalid index
    before = gs.get_state()
    C1, D1, P1, ex, bad, cnt = gs.branch_step(C, D, P, ch)
    after = gs.get_state()
    assert all((x == y).all() for x, y in zip(before[:3], after[:3])) and before[3] == after[3]
    assert bad[7] == 1 and bad.sum() == 1
    for b in range(len(states)):
        s2 = tuple(x.copy() for x in states[b])
        fc = ch[b].copy()
        if b == 7:
            fc[fc == 99] = 0
        halted = oracle.is_halted(d, s2[0], s2[2])
        if not halted:
            oracle.step(d, s2, 0, oracle.FORCED, forced=fc)
        assert ex[b] == (0 if halted else 1)
        assert (C1[b] == s2[0]).all() and (D1[b] == s2[1]).all() and (P1[b] == s2[2]).all(), b
        assert (cnt[b] == oracle.count_choices(d, s2)).all(), b
    gs.close()


@pytest.mark.parametrize("field", ["C", "D", "P_other", "P_high", "D_without_P"])
def test_branch_step_rejects_bad_configurations(field):
    """A configuration outside the state's ranges (C < 0, D outside
    0..65535, a pending rule of another neuron or beyond m, D > 0 with no
    pending rule) is refused with SNP_ERR_INVALID naming the configuration
    and neuron; the check runs before the step kernel, so nothing is
    written.  A good call afterwards still matches the oracle."""
    d = synth.random_system(1500, 41, outdeg=(2, 8), rules=(3, 4), d_range=(0, 3), spikes=(0, 12))
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
    st = oracle.initial_state(d)
    oracle.run(d, st, 3, oracle.PHILOX, 5)
    nb = 6
    C = np.stack([st[0]] * nb); D = np.stack([st[1]] * nb); P = np.stack([st[2]] * nb)
    ch = np.zeros_like(C)
    b, i = 4, 777
    Cb, Db, Pb = C.copy(), D.copy(), P.copy()
    if field == "C":
        Cb[b, i] = -3
    elif field == "D":
        Pb[b, i] = int(d.rule_offsets[i]); Db[b, i] = 70000
    elif field == "P_other":
        Pb[b, i] = int(d.rule_offsets[i + 1]); Db[b, i] = 1      # first rule of neuron i+1
    elif field == "P_high":
        Pb[b, i] = int(d.rule_offsets[-1]) + 5; Db[b, i] = 1
    else:
        Pb[b, i] = -1; Db[b, i] = 2
    sentinel = np.full_like(C, 12345)
    C1, D1, P1 = sentinel.copy(), sentinel.copy(), sentinel.copy()
    ex = np.full(nb, 7, np.int32); bad = np.full(nb, 7, np.int32)
    lib = libsnp.load()
    rc = lib.snp_branch_step(gs.handle, nb, libsnp._ptr(Cb), libsnp._ptr(Db), libsnp._ptr(Pb), libsnp._ptr(ch),
                             libsnp._ptr(C1), libsnp._ptr(D1), libsnp._ptr(P1), libsnp._ptr(ex), libsnp._ptr(bad),
                             None)
    assert rc == libsnp.SNP_ERR_INVALID
    msg = lib.snp_last_error().decode()
    assert f"configuration {b}" in msg and str(i) in msg, msg
    assert (C1 == 12345).all() and (D1 == 12345).all() and (P1 == 12345).all()
    assert (ex == 7).all() and (bad == 7).all()
    # a good call afterwards
    C1, D1, P1, ex, bad, cnt = gs.branch_step(C, D, P, ch)
    s2 = tuple(x.copy() for x in st)
    oracle.step(d, s2, 3, oracle.FORCED, forced=np.zeros(d.q, np.int32))
    assert (ex == 1).all() and (bad == 0).all()
    for k in range(nb):
        assert (C1[k] == s2[0]).all() and (D1[k] == s2[1]).all() and (P1[k] == s2[2]).all()
    gs.close()


def test_branch_step_stages_through_the_callers_allocator():
    """With a caller allocator, the host arrays of a branch step are staged
    in memory the allocator hands out (and returns), not in the library's."""
    import ctypes as ct
    d = synth.random_system(600, 43, outdeg=(2, 8), rules=(3, 4), d_range=(0, 3), spikes=(0, 12))
    live, calls = {}, {"alloc": 0, "release": 0}

    def alloc(ctx, nbytes, stream):
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        live[t.data_ptr()] = t
        calls["alloc"] += 1
        return t.data_ptr()

    def release(ctx, ptr, nbytes, stream):
        calls["release"] += 1
        live.pop(ptr, None)

    a = libsnp.snp_allocator(libsnp.ALLOC_FN(alloc), libsnp.RELEASE_FN(release), None)
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST, allocator=a)
    before = dict(calls)
    st = oracle.initial_state(d)
    C, D, P = (np.stack([x] * 3) for x in st)
    C1, D1, P1, ex, bad, cnt = gs.branch_step(C, D, P, np.zeros_like(C))
    assert calls["alloc"] == before["alloc"] + 1 and calls["release"] == before["release"] + 1
    s2 = tuple(x.copy() for x in st)
    oracle.step(d, s2, 0, oracle.FORCED, forced=np.zeros(d.q, np.int32))
    assert (C1[2] == s2[0]).all() and (P1[2] == s2[2]).all()
    gs.close()
    del a
