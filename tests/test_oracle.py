"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: the paper's
worked example (Tables 1-3, the sorting system of Sec. 6), the matrix
formula C_{k+1} = C_k + S_k . M_Pi of Sec. 2 on delay-free systems, spike
bookkeeping, hand-written delay traces, brute-force enumeration of every
spiking vector on tiny systems, and NVIDIA's host-side Philox generator.
"""
import ctypes as ct
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers

def load_table1():
    rows = []
    for line in open(os.path.join(GOLD, "sort3_table1_dense.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x) for x in line.split()[1:]])
    return np.array(rows, np.int64)


def dense_matrix(desc):
    """M_Pi by its definition (Sec. 2): row r has -c_r at its own neuron and
    +p_r at every neuron its neuron has a synapse to."""
    M = np.zeros((desc.m, desc.q), np.int64)
    for i in range(desc.q):
        for r in range(desc.rule_offsets[i], desc.rule_offsets[i + 1]):
            M[r, i] -= desc.rule_c[r]
            for e in range(desc.syn_offsets[i], desc.syn_offsets[i + 1]):
                M[r, desc.syn_targets[e]] += desc.rule_p[r]
    return M


def regex_ok(n, k, j, c):
    """a^k (a^j)*: n = k + t*j for some t >= 0 (j = 0: n = k); and n >= c."""
    if j == 0:
        return n == k and n >= c
    return n >= k and (n - k) % j == 0 and n >= c


def make_desc(q, rules, syn, init):
    """rules: list per neuron of (k, j, c, p, d); syn: list of (i, j)."""
    offs, ks, js, cs, ps, ds = [0], [], [], [], [], []
    for rl in rules:
        for (k, j, c, p, d) in rl:
            ks.append(k); js.append(j); cs.append(c); ps.append(p); ds.append(d)
        offs.append(len(ks))
    out = [[] for _ in range(q)]
    for (a, b) in syn:
        out[a].append(b)
    so, tg = [0], []
    for i in range(q):
        tg.extend(out[i]); so.append(len(tg))
    a32 = lambda x: np.asarray(x, np.int32)
    return synth.SystemDesc(q=q, init_spikes=a32(init), rule_offsets=np.asarray(offs, np.int64),
                            rule_k=a32(ks), rule_j=a32(js), rule_c=a32(cs), rule_p=a32(ps),
                            rule_d=a32(ds), syn_offsets=np.asarray(so, np.int64), syn_targets=a32(tg))


def tiny_random(seed, q=5, delays=True):
    rng = np.random.default_rng(seed)
    rules = []
    for i in range(q):
        rl = []
        for _ in range(int(rng.integers(0, 4))):
            k = int(rng.integers(1, 4)); j = int(rng.integers(0, 3))
            c = int(rng.integers(1, k + 1)); p = int(rng.integers(0, 3))
            d = int(rng.integers(0, 3)) if (delays and p > 0) else 0
            rl.append((k, j, c, p, d))
        rules.append(rl)
    syn = [(a, b) for a in range(q) for b in range(q) if a != b and rng.random() < 0.4]
    init = rng.integers(0, 6, size=q)
    return make_desc(q, rules, syn, init)


# ---------------------------------------------------------------- Philox

def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("", "/usr/local/cuda/lib64/", "/usr/local/cuda/lib/"):
            try:
                return ct.CDLL(d + name)
            except OSError:
                pass
    return None


def test_philox_matches_curand_host_generator():
    """NVIDIA's host Philox4_32_10 generator (libcurand, run on the CPU) emits
    block b of seed s as Philox4x32-10 at counter (b >> 16, 0, b & 0xffff, 0)
    and key (s mod 2^32, s >> 32); the oracle's Philox must give the same words."""
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ct.c_void_p()
    CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161
    assert lib.curandCreateGeneratorHost(ct.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        nblk = 70000  # spans the 65,536-block wrap, so counter word 0 moves too
        for seed in (0, 1, 0x9E3779B97F4A7C15, 0x0123456789ABCDEF, 2**64 - 1):
            assert lib.curandSetPseudoRandomGeneratorSeed(gen, ct.c_ulonglong(seed)) == 0
            assert lib.curandSetGeneratorOffset(gen, ct.c_ulonglong(0)) == 0
            out = np.zeros(nblk * 4, np.uint32)
            assert lib.curandGenerate(gen, out.ctypes.data_as(ct.c_void_p), ct.c_size_t(out.size)) == 0
            out = out.reshape(-1, 4)
            key = [seed & 0xFFFFFFFF, seed >> 32]
            for b in [0, 1, 2, 3, 17, 255, 4096, 65535, 65536, 65537, 69999]:
                got = oracle.philox4x32_10([b >> 16, 0, b & 0xFFFF, 0], key)
                assert (got == out[b]).all(), (seed, b)
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_choice_is_uniform():
    """The Philox-keyed pick over |A| = 3 rules is uniform (chi-square, 2 dof)."""
    # three always-applicable rules a*(k=1,j=1 with c=1 needs n>=1): give n large
    d = make_desc(1, [[(1, 1, 1, 0, 0), (1, 1, 1, 0, 0), (1, 1, 1, 0, 0)]], [], [10**6])
    counts = np.zeros(3)
    st = oracle.initial_state(d)
    for k in range(6000):
        S, _, h = oracle.step(d, st, k, oracle.PHILOX, seed=12345)
        counts[S[0]] += 1
    exp = counts.sum() / 3
    chi2 = ((counts - exp) ** 2 / exp).sum()
    assert chi2 < 13.8  # p = 0.001 for 2 dof


def test_philox_choice_every_word_position_is_uniform():
    """Neurons 0..7 draw words 0..3 of two Philox blocks (i mod 4 of the
    block at counter i / 4): each neuron's pick over |A| = 3 always
    applicable rules is uniform (chi-square, 2 dof, p = 0.001 each)."""
    q = 8
    d = make_desc(q, [[(1, 1, 1, 0, 0), (1, 1, 1, 0, 0), (1, 1, 1, 0, 0)] for _ in range(q)], [], [10**6] * q)
    counts = np.zeros((q, 3))
    st = oracle.initial_state(d)
    for k in range(6000):
        S, _, _ = oracle.step(d, st, k, oracle.PHILOX, seed=777)
        for i in range(q):
            counts[i, S[i] - 3 * i] += 1
    exp = 6000 / 3
    chi2 = ((counts - exp) ** 2 / exp).sum(axis=1)
    assert (chi2 < 13.8).all(), chi2


@pytest.mark.parametrize("pair", [(0, 1), (3, 4)])
def test_philox_choices_of_neighbours_are_independent(pair):
    """Two neurons sharing one Philox block (0, 1: words 0 and 1) or in
    adjacent blocks (3, 4) choose independently: their joint picks over 3 x 3
    cells are uniform (chi-square, 8 dof, p = 0.001).  Giving two neurons of
    a block the same word would put every draw on the diagonal."""
    q = 8
    d = make_desc(q, [[(1, 1, 1, 0, 0), (1, 1, 1, 0, 0), (1, 1, 1, 0, 0)] for _ in range(q)], [], [10**6] * q)
    a, b = pair
    joint = np.zeros((3, 3))
    st = oracle.initial_state(d)
    for k in range(9000):
        S, _, _ = oracle.step(d, st, k, oracle.PHILOX, seed=31337)
        joint[S[a] - 3 * a, S[b] - 3 * b] += 1
    exp = 9000 / 9
    chi2 = ((joint - exp) ** 2 / exp).sum()
    assert chi2 < 26.1, (chi2, joint)


# ---------------------------------------------------------------- worked example

def test_sort_system_reproduces_table1():
    """The sorting system's rules and synapses give Table 1 entry for entry."""
    d = synth.sort_system([3, 2, 1])
    assert (dense_matrix(d) == load_table1()).all()


def test_sort3_trace():
    """Hand-derived computation of the sorting system on v = (3, 2, 1)."""
    d = synth.sort_system([3, 2, 1])
    tr = oracle.run_trace(d, 20)
    assert len(tr) == 4                       # halts before step 4
    C = [t[0].tolist() for t in tr]
    S = [t[3].tolist() for t in tr]
    #           i1 i2 i3 s1 s2 s3 o1 o2 o3
    assert C[0] == [2, 1, 0, 3, 3, 3, 0, 0, 0]
    assert C[1] == [1, 0, 0, 2, 2, 2, 1, 1, 1]
    assert C[2] == [0, 0, 0, 1, 1, 1, 1, 2, 2]
    assert C[3] == [0, 0, 0, 0, 0, 0, 1, 2, 3]
    # rule ids: r1..r3 = 0..2, s1: r4 r5 r6 = 3 4 5, s2: r7 r8 r9 = 6 7 8, s3: 9 10 11
    assert S[0] == [0, 1, 2, -1, -1, -1, -1, -1, -1]
    assert S[1] == [0, 1, -1, 3, 7, 11, -1, -1, -1]
    assert S[2] == [0, -1, -1, 4, 6, 10, -1, -1, -1]
    assert S[3] == [-1, -1, -1, 5, 8, 9, -1, -1, -1]


@pytest.mark.parametrize("seed", range(12))
def test_sort_closed_form(seed):
    """o_k holds the k-th smallest input; the run takes max(v) + 1 steps."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 9))
    v = rng.integers(1, 13, size=n).tolist()
    d = synth.sort_system(v)
    st = oracle.initial_state(d)
    ex, _ = oracle.run(d, st, 1000)
    assert ex == max(v) + 1
    assert st[0][2 * n:].tolist() == sorted(v)


def test_dense_formula_on_table1():
    """Every step of the sorting system satisfies C_{k+1} = C_k + s_k . M_Pi
    with M_Pi read from Table 1 and s_k the 0/1 vector of selected rules."""
    M = load_table1()
    for v in ([3, 2, 1], [1, 2, 3], [2, 2, 3]):
        d = synth.sort_system(v)
        st = oracle.initial_state(d)
        for k in range(10):
            c0 = st[0].astype(np.int64).copy()
            S, _, halted = oracle.step(d, st, k)
            if halted:
                break
            s = np.zeros(d.m, np.int64)
            s[S[S >= 0]] = 1
            assert (st[0] == c0 + s @ M).all()


@pytest.mark.parametrize("seed", range(40))
def test_dense_formula_random_delay_free(seed):
    """Delay-free random systems: C_{k+1} = C_k + s_k . M_Pi every step,
    for first-applicable and Philox selection."""
    d = tiny_random(seed, q=6, delays=False)
    M = dense_matrix(d)
    for mode in (oracle.FIRST, oracle.PHILOX):
        st = oracle.initial_state(d)
        for k in range(8):
            c0 = st[0].astype(np.int64).copy()
            S, _, halted = oracle.step(d, st, k, mode, seed=seed + 7)
            if halted:
                break
            s = np.zeros(d.m, np.int64)
            s[S[S >= 0]] = 1
            assert (st[0] == c0 + s @ M).all()


# ---------------------------------------------------------------- delays

def test_delay_chain_traces():
    """Hand traces: a rule fired at t with delay d consumes at t, keeps its
    neuron closed for steps t..t+d-1 and emits at t+d."""
    for dl in (1, 2, 3):
        d = make_desc(2, [[(1, 0, 1, 1, dl)], []], [(0, 1)], [1, 0])
        tr = oracle.run_trace(d, 20)
        assert len(tr) == dl + 1
        C, D, P, S = tr[0]
        assert C.tolist() == [0, 0] and D.tolist() == [dl - 1, 0] and P.tolist() == [0, -1]
        assert S.tolist() == [0, -1]
        for t in range(1, dl):
            C, D, P, S = tr[t]
            assert C.tolist() == [0, 0] and D.tolist() == [dl - 1 - t, 0] and P.tolist() == [0, -1]
            assert S.tolist() == [-1, -1]
        C, D, P, S = tr[dl]
        assert C.tolist() == [0, 1] and D.tolist() == [0, 0] and P.tolist() == [-1, -1]


def test_spikes_to_closed_neuron_are_lost():
    # n0: a -> a; 2   n2: a -> a; 0   synapses 2 -> 0, 0 -> 1
    d = make_desc(3, [[(1, 0, 1, 1, 2)], [], [(1, 0, 1, 1, 0)]], [(2, 0), (0, 1)], [1, 0, 1])
    tr = oracle.run_trace(d, 20)
    assert len(tr) == 3
    assert [t[0].tolist() for t in tr] == [[0, 0, 0], [0, 0, 0], [0, 1, 0]]
    assert [t[1].tolist() for t in tr] == [[1, 0, 0], [0, 0, 0], [0, 0, 0]]
    assert [t[2].tolist() for t in tr] == [[0, -1, -1], [0, -1, -1], [-1, -1, -1]]
    assert [t[3].tolist() for t in tr] == [[0, -1, 1], [-1, -1, -1], [-1, -1, -1]]


def test_reopened_neuron_receives_and_refires():
    # n0: a -> a; 1   n1: sink   n2: a^2 -> a; 0   n3: a -> a; 0
    # synapses 0 -> 1, 2 -> 0, 3 -> 2
    d = make_desc(4, [[(1, 0, 1, 1, 1)], [], [(2, 0, 2, 1, 0)], [(1, 0, 1, 1, 0)]],
                  [(0, 1), (2, 0), (3, 2)], [1, 0, 1, 1])
    tr = oracle.run_trace(d, 20)
    assert len(tr) == 4
    assert [t[0].tolist() for t in tr] == [[0, 0, 2, 0], [1, 1, 0, 0], [0, 1, 0, 0], [0, 2, 0, 0]]
    assert [t[1].tolist() for t in tr] == [[0] * 4] * 4
    assert [t[2].tolist() for t in tr] == [[0, -1, -1, -1], [-1] * 4, [0, -1, -1, -1], [-1] * 4]
    assert [t[3].tolist() for t in tr] == [[0, -1, -1, 2], [-1, -1, 1, -1], [0, -1, -1, -1],
                                           [-1] * 4]


@pytest.mark.parametrize("seed", range(25))
def test_bookkeeping_with_delays(seed):
    """Per step: the spike total changes by what open senders emit times their
    out-degree, minus what is consumed, minus what lands on closed neurons;
    a closed neuron's count does not change; every selection is applicable
    and belongs to an idle open neuron; first-applicable picks the first."""
    d = synth.random_system(300, 100 + seed, outdeg=(1, 8), rules=(2, 4), d_range=(0, 3), spikes=(0, 10))
    outs = [d.syn_targets[d.syn_offsets[i]:d.syn_offsets[i + 1]] for i in range(d.q)]
    mode = oracle.PHILOX if seed % 2 else oracle.FIRST
    st = oracle.initial_state(d)
    for k in range(30):
        C0, D0, P0 = (x.copy() for x in st)
        S, E, halted = oracle.step(d, st, k, mode, seed=seed)
        if halted:
            break
        Ei = np.zeros(d.q, np.int64)
        recv = np.ones(d.q, bool)
        consumed = 0
        for i in range(d.q):
            if P0[i] != -1 and D0[i] == 0:
                Ei[i] = d.rule_p[P0[i]]
                assert S[i] == -1
            elif P0[i] != -1:
                recv[i] = False
                assert S[i] == -1 and st[0][i] == C0[i]
            elif S[i] != -1:
                r = S[i]
                assert d.rule_offsets[i] <= r < d.rule_offsets[i + 1]
                assert regex_ok(C0[i], d.rule_k[r], d.rule_j[r], d.rule_c[r])
                if mode == oracle.FIRST:
                    for r2 in range(d.rule_offsets[i], r):
                        assert not regex_ok(C0[i], d.rule_k[r2], d.rule_j[r2], d.rule_c[r2])
                consumed += d.rule_c[r]
                if d.rule_d[r] == 0:
                    Ei[i] = d.rule_p[r]
                else:
                    recv[i] = False
            else:
                for r2 in range(d.rule_offsets[i], d.rule_offsets[i + 1]):
                    assert not regex_ok(C0[i], d.rule_k[r2], d.rule_j[r2], d.rule_c[r2])
        assert (E == Ei).all()
        produced = sum(int(Ei[i]) * len(outs[i]) for i in range(d.q))
        lost = sum(int(Ei[i]) * int((~recv[outs[i]]).sum()) for i in range(d.q))
        assert int(st[0].astype(np.int64).sum() - C0.astype(np.int64).sum()) == produced - consumed - lost


# ---------------------------------------------------------------- brute force

def py_successors(d, C, D, P):
    """Independent enumerator: every spiking vector of SV_k (one applicable
    rule per idle open neuron, all combinations) and the state it leads to,
    computed by pulling from in-neighbours.  Returns None at a fixed point."""
    q = d.q
    inn = [[] for _ in range(q)]
    for i in range(q):
        for e in range(d.syn_offsets[i], d.syn_offsets[i + 1]):
            inn[d.syn_targets[e]].append(i)
    choices = []
    for i in range(q):
        if P[i] == -1:
            A = [r for r in range(d.rule_offsets[i], d.rule_offsets[i + 1])
                 if regex_ok(C[i], d.rule_k[r], d.rule_j[r], d.rule_c[r])]
            choices.append(A if A else [None])
        else:
            choices.append([None])
    if all(ch == [None] for ch in choices) and all(p == -1 for p in P):
        return None
    res = []
    for combo in itertools.product(*choices):
        emit = [0] * q
        recv = [True] * q
        Cn, Dn, Pn = list(map(int, C)), list(map(int, D)), list(map(int, P))
        for i in range(q):
            if P[i] != -1 and D[i] == 0:
                emit[i] = int(d.rule_p[P[i]]); Pn[i] = -1; Dn[i] = 0
            elif P[i] != -1:
                recv[i] = False; Dn[i] = D[i] - 1
            elif combo[i] is not None:
                r = combo[i]
                Cn[i] -= int(d.rule_c[r])
                if d.rule_d[r] == 0:
                    emit[i] = int(d.rule_p[r])
                else:
                    recv[i] = False; Pn[i] = r; Dn[i] = int(d.rule_d[r]) - 1
        for j in range(q):
            if recv[j]:
                Cn[j] += sum(emit[i] for i in inn[j])
        forced = [choices[i].index(combo[i]) if combo[i] is not None else 0 for i in range(q)]
        res.append((forced, (tuple(Cn), tuple(Dn), tuple(Pn))))
    return res


@pytest.mark.parametrize("seed", range(30))
def test_bruteforce_tree(seed):
    """On tiny systems the oracle's forced-choice step reproduces every branch
    of the independent enumerator, and the FIRST / PHILOX runs are paths of
    the computation tree."""
    d = tiny_random(1000 + seed, q=int(np.random.default_rng(seed).integers(2, 6)))
    frontier = [oracle.initial_state(d)]
    for k in range(5):
        nxt = []
        for st in frontier:
            succ = py_successors(d, *st)
            assert oracle.is_halted(d, st[0], st[2]) == (succ is None)
            if succ is None:
                continue
            for forced, expect in succ[:20]:
                s2 = tuple(x.copy() for x in st)
                oracle.step(d, s2, k, oracle.FORCED, forced=np.asarray(forced, np.int32))
                assert (tuple(map(int, s2[0])), tuple(map(int, s2[1])), tuple(map(int, s2[2]))) == expect
                nxt.append(s2)
        frontier = nxt[:30]
    # FIRST and PHILOX trajectories lie in the tree
    for mode in (oracle.FIRST, oracle.PHILOX):
        st = oracle.initial_state(d)
        for k in range(5):
            succ = py_successors(d, *st)
            S, _, halted = oracle.step(d, st, k, mode, seed=seed)
            if succ is None:
                assert halted
                break
            got = (tuple(map(int, st[0])), tuple(map(int, st[1])), tuple(map(int, st[2])))
            assert got in {e for _, e in succ}


# ---------------------------------------------------------------- edge cases

def test_fixed_point_and_empty_system():
    d = make_desc(3, [[], [(2, 0, 2, 1, 0)], []], [(1, 0)], [5, 1, 0])
    st = oracle.initial_state(d)
    ex, S = oracle.run(d, st, 10)
    assert ex == 0 and (S == -1).all() and st[0].tolist() == [5, 1, 0]
    d1 = make_desc(1, [[]], [], [0])
    ex, _ = oracle.run(d1, oracle.initial_state(d1), 3)
    assert ex == 0


def test_overflow_is_detected():
    d = make_desc(2, [[(1, 1, 1, 1000, 0)], []], [(0, 1)], [10, 2**31 - 600])
    st = oracle.initial_state(d)
    with pytest.raises(oracle.OracleOverflow):
        oracle.run(d, st, 5)


def test_forgetting_rule_needs_exact_count():
    # forgetting a^2 -> lambda stored as k=c=2, j=0, p=0
    d = make_desc(2, [[(2, 0, 2, 0, 0)], []], [(0, 1)], [3, 0])
    ex, _ = oracle.run(d, oracle.initial_state(d), 5)
    assert ex == 0
    d2 = make_desc(2, [[(2, 0, 2, 0, 0)], []], [(0, 1)], [2, 0])
    st = oracle.initial_state(d2)
    ex, S = oracle.run(d2, st, 5)
    assert ex == 1 and st[0].tolist() == [0, 0] and S.tolist() == [0, -1]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_parallel_pull_oracle_equals_definition_oracle(seed):
    """orc_run_pull (phase 2 pulled over in-lists, each phase split across
    threads) gives the state, spiking vector and executed step count of the
    neuron-by-neuron oracle, step by step, with FIRST and PHILOX, up to and
    past a fixed point."""
    d = synth.random_system(3000 + 500 * seed, 40 + seed, outdeg=(1, 12), rules=(2, 4), d_range=(0, 4),
                            spikes=(0, 15))
    for mode in (oracle.FIRST, oracle.PHILOX):
        a = oracle.initial_state(d)
        b = oracle.initial_state(d)
        pr = oracle.PullRunner(d)
        k = 0
        for n in (1, 1, 5, 20, 60):
            ea, Sa = oracle.run(d, a, n, mode, 99, step0=k)
            eb, Sb = pr.run(b, n, mode, 99, step0=k)
            assert ea == eb
            for x, y in zip(a, b):
                assert (x == y).all()
            if ea:
                assert (Sa == Sb).all()
            k += ea
    # a system that reaches a fixed point
    h = synth.sort_system([3, 2, 1])
    a, b = oracle.initial_state(h), oracle.initial_state(h)
    ea, _ = oracle.run(h, a, 50)
    eb, _ = oracle.PullRunner(h).run(b, 50)
    assert ea == eb == 4 and all((x == y).all() for x, y in zip(a, b))


def test_parallel_pull_oracle_reports_overflow():
    d = synth.random_system(50, 5, outdeg=(20, 40), rules=(2, 2), spikes=(2**31 - 100, 2**31 - 50))
    with pytest.raises(oracle.OracleOverflow):
        oracle.PullRunner(d).run(oracle.initial_state(d), 20, oracle.FIRST)


def test_subset_sum_shaped_stand_in_runs_and_branches():
    """The stand-in is a valid system with delays; its choice neurons each
    have two applicable rules on one spike (the computation tree branches),
    and with FIRST every value chain delivers sum(v) spikes to the output
    neuron over the run (one per chain step), besides the check neurons'."""
    import numpy as np
    v = [3, 0, 5, 2]
    d = synth.subset_sum_shaped(len(v), v=v)
    st = oracle.initial_state(d)
    S, E, halted = oracle.step(d, st, 0)
    assert not halted and S[0] == 0          # the source fires
    S, E, halted = oracle.step(d, st, 1)
    # each choice neuron (1..n) holds one spike and two applicable rules
    for i in range(1, 1 + len(v)):
        r0 = int(d.rule_offsets[i])
        assert S[i] == r0                     # FIRST takes a -> a;0
    ex, _ = oracle.run(d, st, 200, oracle.FIRST, 0, step0=2)
    assert ex < 200                           # reaches a fixed point


@pytest.mark.parametrize("seed", range(6))
def test_count_choices_is_the_branching_of_sv_k(seed):
    """orc_count_choices gives |A_i| per neuron: on tiny systems the product
    over neurons equals the number of spiking vectors the independent
    enumerator finds, level after level."""
    d = tiny_random(2000 + seed, q=int(np.random.default_rng(seed).integers(2, 6)))
    frontier = [oracle.initial_state(d)]
    for k in range(4):
        nxt = []
        for st in frontier:
            succ = py_successors(d, *st)
            counts = oracle.count_choices(d, st)
            if succ is None:
                assert counts.sum() == 0
                continue
            assert int(np.prod(np.maximum(counts, 1))) == len(succ)
            for forced, _ in succ[:6]:
                s2 = tuple(x.copy() for x in st)
                oracle.step(d, s2, k, oracle.FORCED, forced=np.asarray(forced, np.int32))
                nxt.append(s2)
        frontier = nxt[:12]


def test_branch_enumeration_order_and_cap():
    """paper_2408_04343_gb300.tree.branch_choices: every combination exactly
    once (the product of the counts), neurons with one choice fixed at 0,
    and the cap reported."""
    import itertools
    from paper_2408_04343_gb300.tree import branch_choices
    counts = np.array([0, 3, 1, 2, 4], np.int32)
    combos, cut = branch_choices(counts, 1000)
    assert not cut and len(combos) == 24
    want = {tuple(c) for c in itertools.product(*[range(max(1, int(x))) for x in counts])}
    assert {tuple(int(v) for v in c) for c in combos} == want
    combos, cut = branch_choices(counts, 10)
    assert cut and len(combos) == 10
    combos, cut = branch_choices(np.zeros(4, np.int32), 5)
    assert not cut and len(combos) == 1


# ---------------------------------------------------------------- finite unions

def _terms_of(d, r):
    return [(int(d.term_k[t]), int(d.term_j[t])) for t in range(d.rule_term_offsets[r], d.rule_term_offsets[r + 1])]


def _union_member(n, terms, c):
    """n in the union of the terms' languages, by listing each language's
    word lengths k, k+j, k+2j, ... up to n (not by the modular test)."""
    if n < c:
        return False
    for k, j in terms:
        lengths = [k] if j == 0 else range(k, n + 1, j)
        if n in lengths:
            return True
    return False


def _single_term_union(d, decoy=True):
    """d with every rule a^k(a^j)* written as a one-term union."""
    import dataclasses
    m = d.m
    return dataclasses.replace(d, rule_term_offsets=np.arange(m + 1, dtype=np.int64),
                               term_k=np.asarray(d.rule_k, np.int32).copy(), term_j=np.asarray(d.rule_j, np.int32).copy(),
                               rule_k=np.full(m, 1000, np.int32) if decoy else d.rule_k,
                               rule_j=np.zeros(m, np.int32) if decoy else d.rule_j)


@pytest.mark.parametrize("seed", range(8))
def test_one_term_unions_equal_plain_rules(seed):
    """A rule given as a one-term union behaves exactly as the plain rule
    (rule_k/rule_j hold decoys that would make nothing applicable)."""
    d = synth.random_system(300, 50 + seed, outdeg=(1, 6), rules=(1, 4), d_range=(0, 3), spikes=(0, 9))
    u = _single_term_union(d)
    for mode in (oracle.FIRST, oracle.PHILOX):
        a, b = oracle.initial_state(d), oracle.initial_state(u)
        for k in range(25):
            Sa, _, ha = oracle.step(d, a, k, mode, seed=seed)
            Sb, _, hb = oracle.step(u, b, k, mode, seed=seed)
            assert ha == hb and (Sa == Sb).all()
            assert all((x == y).all() for x, y in zip(a, b))
            if ha:
                break


def test_union_equal_to_one_expression():
    """a^2(a^2)* U a^3(a^2)* is a^2 a* (every n >= 2), and a^1(a^3)* U
    a^2(a^3)* U a^3(a^3)* is a+: systems written either way run identically."""
    rules = [[(2, 1, 1, 1, 0), (1, 0, 1, 0, 0)], [(1, 1, 1, 2, 1)], [(3, 2, 2, 1, 0), (1, 1, 1, 1, 0)]]
    syn = [(0, 1), (0, 2), (1, 0), (2, 1), (2, 0)]
    plain = make_desc(3, rules, syn, [5, 2, 4])
    import dataclasses
    # rule 0: a^2 a*  -> two terms; rule 2: a+ (k=1, j=1) -> three terms; others one term
    terms = [[(2, 2), (3, 2)], [(1, 0)], [(1, 3), (2, 3), (3, 3)], [(3, 2)], [(1, 1)]]
    off = np.zeros(plain.m + 1, np.int64)
    off[1:] = np.cumsum([len(t) for t in terms])
    u = dataclasses.replace(plain, rule_term_offsets=off,
                            term_k=np.asarray([k for t in terms for k, _ in t], np.int32),
                            term_j=np.asarray([j for t in terms for _, j in t], np.int32),
                            rule_k=np.full(plain.m, 1000, np.int32), rule_j=np.zeros(plain.m, np.int32))
    for mode in (oracle.FIRST, oracle.PHILOX):
        ta = oracle.run_trace(plain, 40, mode, seed=3)
        tb = oracle.run_trace(u, 40, mode, seed=3)
        assert len(ta) == len(tb) and len(ta) > 5
        for x, y in zip(ta, tb):
            assert all((p == r).all() for p, r in zip(x, y))


def test_union_hand_trace():
    """Neuron 0 holds 5 spikes and one rule (a^4 U a^1(a^3)*)/a^2 -> a;
    neuron 1 has (a^2 U a^5)/a -> a, neuron 2 forgets a^3.  By hand:
    step 0: n0 = 5 is neither 4 nor 1 mod 3 -> idle; n1 = 0 idle; halted.
    With 7 spikes instead (7 = 1 + 2*3): n0 fires, 7-2 = 5, sends 1 to n1 and
    n2; then n0 = 5 idle, n1 = 1 idle -- but n2 = 1 idle: halted after one
    step.  With 4 spikes: n0 fires (a^4), 4-2 = 2 -> n1 = 1, n2 = 1; step 1:
    n0 = 2 idle (2 != 4, 2-1 = 1 not a multiple of 3): halted."""
    import dataclasses
    base = make_desc(3, [[(9, 0, 2, 1, 0)], [(9, 0, 1, 1, 0)], [(3, 0, 3, 0, 0)]], [(0, 1), (0, 2), (1, 2)], [5, 0, 0])
    terms = [[(4, 0), (1, 3)], [(2, 0), (5, 0)], [(3, 0)]]
    off = np.zeros(4, np.int64)
    off[1:] = np.cumsum([len(t) for t in terms])
    mk = lambda init: dataclasses.replace(base, init_spikes=np.asarray(init, np.int32), rule_term_offsets=off,
                                          term_k=np.asarray([k for t in terms for k, _ in t], np.int32),
                                          term_j=np.asarray([j for t in terms for _, j in t], np.int32))
    st = oracle.initial_state(mk([5, 0, 0]))
    assert oracle.run(mk([5, 0, 0]), st, 5)[0] == 0
    d = mk([7, 0, 0]); st = oracle.initial_state(d)
    ex, S = oracle.run(d, st, 5)
    assert ex == 1 and S.tolist() == [0, -1, -1] and st[0].tolist() == [5, 1, 1]
    d = mk([4, 0, 0]); st = oracle.initial_state(d)
    ex, S = oracle.run(d, st, 5)
    assert ex == 1 and st[0].tolist() == [2, 1, 1]
    # n1 = 2 fires its a^2 term: send n1 two spikes as well
    d = mk([7, 1, 0]); st = oracle.initial_state(d)
    S, _, h = oracle.step(d, st, 0)
    assert S.tolist() == [0, -1, -1] and st[0].tolist() == [5, 2, 1]
    S, _, h = oracle.step(d, st, 1)
    assert S.tolist() == [-1, 1, -1] and st[0].tolist() == [5, 1, 2]


@pytest.mark.parametrize("seed", range(12))
def test_union_bruteforce_tree(seed):
    """Random unions on tiny systems: the oracle's choice counts equal the
    number of rules whose union lists n (by enumeration), and its forced
    steps give every branch the enumerator finds."""
    q = int(np.random.default_rng(seed).integers(2, 6))
    d = synth.with_unions(tiny_random(2000 + seed, q=q), seed, terms=(1, 3), k_max=4, j_max=3)
    frontier = [oracle.initial_state(d)]
    for k in range(4):
        nxt = []
        for st in frontier:
            C, D, P = st
            A = []
            for i in range(q):
                rs = [r for r in range(d.rule_offsets[i], d.rule_offsets[i + 1])
                      if _union_member(int(C[i]), _terms_of(d, r), int(d.rule_c[r]))]
                A.append(rs if P[i] == -1 else [])
            assert oracle.count_choices(d, st).tolist() == [len(a) for a in A]
            halted = all(not a for a in A) and all(p == -1 for p in P)
            assert oracle.is_halted(d, C, P) == halted
            if halted:
                continue
            for combo in itertools.islice(itertools.product(*[range(max(1, len(a))) for a in A]), 16):
                s2 = tuple(x.copy() for x in st)
                S, _, _ = oracle.step(d, s2, k, oracle.FORCED, forced=np.asarray(combo, np.int32))
                for i in range(q):
                    if A[i]:
                        assert S[i] == A[i][combo[i]]
                nxt.append(s2)
        frontier = nxt[:24]


@pytest.mark.parametrize("cuts", [(0, 3000), (0, 1100, 2050, 3000), (0, 1, 2999, 3000)])
@pytest.mark.parametrize("mode", [oracle.FIRST, oracle.PHILOX])
def test_range_phases_compose_to_the_step(cuts, mode):
    """The definition split at its exchange point (phase 1 per neuron range,
    the emissions of every range collected, then phase 2 and the delay update
    per range) composes, over ranges covering all neurons, to the whole step:
    the same states and executed step count as orc_run over 30 steps, and
    nothing executes once no range is active (the fixed point)."""
    d = synth.random_system(3000, 5, outdeg=(2, 10), rules=(3, 4), d_range=(0, 3), spikes=(0, 12))
    full = oracle.initial_state(d)
    ex, _ = oracle.run(d, full, 30, mode, 7)
    sh = [oracle.RangeShard(d, a, b) for a, b in zip(cuts[:-1], cuts[1:])]
    k = 0
    for _ in range(30):
        act = [x.select(k, mode, 7) for x in sh]
        if not any(act):
            break
        E = np.zeros(d.q, np.int32)
        for x in sh:
            E[x.lo:x.hi] = x.E[x.lo:x.hi]
        for x in sh:
            x.E[:] = E
            x.receive()
        k += 1
    assert k == ex
    for i, arr in enumerate(full):
        got = np.concatenate([(x.C, x.D, x.P)[i][x.lo:x.hi] for x in sh])
        assert (got == arr).all()
