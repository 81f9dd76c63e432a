"""Seeded synthetic SNP systems shaped like the evaluation workloads.

This module only draws random inputs: neuron counts, initial spikes, rule
fields and synapse lists.  It holds none of the method's arithmetic (no
applicability test, no selection, no propagation) and is the one piece of code
shared by the CUDA path's tests and bench and by the CPU oracle's tests.

A system is described exactly as the C-ABI's ``snp_desc`` takes it (Sec. 5,
"Initialization": initial spikes, rules with consumed/produced spikes, regular
expression and delay, then synapses):

* ``init_spikes[q]``      -- C_0 (Sec. 2, configuration vector)
* ``rule_offsets[q+1]``   -- N_Pi, rules of neuron i are offsets[i]..offsets[i+1]-1
* ``rule_k/j/c/p/d[m]``   -- regex a^k(a^j)* (j = 0 means exactly a^k),
                             consumed c, produced p (0 = forgetting), delay d
* ``syn_offsets[q+1]``, ``syn_targets[|syn|]`` -- out-lists of syn, no
                             self-loops, no duplicates (Sec. 2)
* optional ``rule_term_offsets[m+1]``, ``term_k/term_j[T]`` -- rule r's regex
                             is the finite union of a^term_k[t](a^term_j[t])*
                             over its terms; rule_k/rule_j are then unused

Rule recipe (the evaluation workloads): per neuron, R-1 firing rules followed
by one forgetting rule.  A firing rule draws k in [1,4], j in [0,3], c in [1,k],
p in [1,3] and d in the workload's delay range; the forgetting rule a^s -> lambda
draws s in [1,4] and is stored as k = c = s, j = 0, p = 0, d = 0.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass
class SystemDesc:
    q: int
    init_spikes: np.ndarray
    rule_offsets: np.ndarray
    rule_k: np.ndarray
    rule_j: np.ndarray
    rule_c: np.ndarray
    rule_p: np.ndarray
    rule_d: np.ndarray
    syn_offsets: np.ndarray
    syn_targets: np.ndarray
    out_neuron: int = 0
    seed: int = 0          # key of the nondeterministic choice (Philox)
    name: str = ""
    rule_term_offsets: np.ndarray | None = None   # [m+1]: union expressions (optional)
    term_k: np.ndarray | None = None
    term_j: np.ndarray | None = None

    @property
    def m(self) -> int:
        return int(self.rule_offsets[-1])

    @property
    def num_syn(self) -> int:
        return int(self.syn_offsets[-1])

    def arrays(self):
        """Contiguous arrays in the dtypes the C-ABI expects."""
        return dict(
            init_spikes=np.ascontiguousarray(self.init_spikes, np.int32),
            rule_offsets=np.ascontiguousarray(self.rule_offsets, np.int64),
            rule_k=np.ascontiguousarray(self.rule_k, np.int32),
            rule_j=np.ascontiguousarray(self.rule_j, np.int32),
            rule_c=np.ascontiguousarray(self.rule_c, np.int32),
            rule_p=np.ascontiguousarray(self.rule_p, np.int32),
            rule_d=np.ascontiguousarray(self.rule_d, np.int32),
            syn_offsets=np.ascontiguousarray(self.syn_offsets, np.int64),
            syn_targets=np.ascontiguousarray(self.syn_targets, np.int32),
            rule_term_offsets=(None if self.rule_term_offsets is None
                               else np.ascontiguousarray(self.rule_term_offsets, np.int64)),
            term_k=None if self.term_k is None else np.ascontiguousarray(self.term_k, np.int32),
            term_j=None if self.term_j is None else np.ascontiguousarray(self.term_j, np.int32),
        )


def _targets(rng: np.random.Generator, q: int, deg: np.ndarray) -> np.ndarray:
    """Targets drawn uniformly without replacement per row, never the source."""
    n = int(deg.sum())
    if n == 0:
        return np.zeros(0, np.int32)
    if int(deg.max()) > q - 1:
        raise ValueError("out-degree larger than q-1")
    src = np.repeat(np.arange(q, dtype=np.int64), deg)
    t = rng.integers(0, q - 1, size=n, dtype=np.int64)
    t += t >= src
    while True:
        key = src * q + t
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup_pos = order[1:][ks[1:] == ks[:-1]]
        if dup_pos.size == 0:
            break
        r = rng.integers(0, q - 1, size=dup_pos.size, dtype=np.int64)
        r += r >= src[dup_pos]
        t[dup_pos] = r
    return t.astype(np.int32)


def zipf_degrees(rng: np.random.Generator, n: int, alpha: float, lo: int, hi: int) -> np.ndarray:
    """Truncated discrete power law on [lo, hi]: P(x) proportional to x^-alpha."""
    x = np.arange(lo, hi + 1, dtype=np.float64)
    w = np.exp(-alpha * np.log(x))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(n)
    return (np.searchsorted(cdf, u, side="right") + lo).astype(np.int64).clip(lo, hi)


def random_system(q: int, seed: int, *, outdeg=(1, 8), zipf=None, rules=(3, 3),
                  k_range=(1, 4), j_range=(0, 3), p_range=(1, 3), d_range=(0, 3),
                  spikes=(0, 10), forget_s=(1, 4), name: str = "") -> SystemDesc:
    """One random SNP system with delays.

    ``rules`` is the inclusive range of the total rule count per neuron
    (R-1 firing rules, then one forgetting rule).  ``zipf`` = (alpha, lo, hi)
    replaces the uniform out-degree range.
    """
    rng = np.random.default_rng(seed)
    if q < 1:
        raise ValueError("q >= 1")
    init = rng.integers(spikes[0], spikes[1] + 1, size=q, dtype=np.int64).astype(np.int32)
    R = rng.integers(rules[0], rules[1] + 1, size=q, dtype=np.int64)
    rule_offsets = np.zeros(q + 1, np.int64)
    np.cumsum(R, out=rule_offsets[1:])
    m = int(rule_offsets[-1])
    # position of each rule inside its neuron; the last one is the forgetting rule
    owner = np.repeat(np.arange(q, dtype=np.int64), R)
    local = np.arange(m, dtype=np.int64) - rule_offsets[owner]
    is_forget = local == (R[owner] - 1)
    k = rng.integers(k_range[0], k_range[1] + 1, size=m, dtype=np.int64)
    j = rng.integers(j_range[0], j_range[1] + 1, size=m, dtype=np.int64)
    c = 1 + (rng.random(m) * k).astype(np.int64)          # c uniform in [1, k]
    c = np.minimum(c, k)
    p = rng.integers(p_range[0], p_range[1] + 1, size=m, dtype=np.int64)
    d = rng.integers(d_range[0], d_range[1] + 1, size=m, dtype=np.int64)
    s = rng.integers(forget_s[0], forget_s[1] + 1, size=m, dtype=np.int64)
    k = np.where(is_forget, s, k)
    c = np.where(is_forget, s, c)
    j = np.where(is_forget, 0, j)
    p = np.where(is_forget, 0, p)
    d = np.where(is_forget, 0, d)
    if q == 1:
        deg = np.zeros(1, np.int64)
    elif zipf is not None:
        deg = zipf_degrees(rng, q, zipf[0], zipf[1], min(zipf[2], q - 1))
    else:
        deg = rng.integers(min(outdeg[0], q - 1), min(outdeg[1], q - 1) + 1, size=q, dtype=np.int64)
    syn_offsets = np.zeros(q + 1, np.int64)
    np.cumsum(deg, out=syn_offsets[1:])
    tg = _targets(rng, q, deg)
    return SystemDesc(q=q, init_spikes=init, rule_offsets=rule_offsets,
                      rule_k=k.astype(np.int32), rule_j=j.astype(np.int32),
                      rule_c=c.astype(np.int32), rule_p=p.astype(np.int32),
                      rule_d=d.astype(np.int32), syn_offsets=syn_offsets,
                      syn_targets=tg, out_neuron=0, seed=seed, name=name)


# ---------------------------------------------------------------------------
# The evaluation workloads.  Each returns a SystemDesc (or a list) plus the
# step count and selection mode it is run with.

SEL_FIRST = 0
SEL_PHILOX = 1


def with_unions(desc: SystemDesc, seed: int, terms=(1, 3), k_max: int = 5, j_max: int = 3,
                decoy: bool = True) -> SystemDesc:
    """The same system with each rule's expression replaced by a union of
    ``terms`` random terms a^k(a^j)* (k in [0, k_max], j in [0, j_max]).
    With ``decoy`` the now unused rule_k/rule_j hold values that would make
    no rule applicable, so a path that still read them would show."""
    rng = np.random.default_rng(seed)
    m = desc.m
    cnt = rng.integers(terms[0], terms[1] + 1, size=m)
    off = np.zeros(m + 1, np.int64)
    off[1:] = np.cumsum(cnt)
    T = int(off[-1])
    tk = rng.integers(0, k_max + 1, size=T).astype(np.int32)
    tj = rng.integers(0, j_max + 1, size=T).astype(np.int32)
    rk = np.full(m, 1000, np.int32) if decoy else np.asarray(desc.rule_k, np.int32).copy()
    rj = np.zeros(m, np.int32) if decoy else np.asarray(desc.rule_j, np.int32).copy()
    return dataclasses.replace(desc, rule_k=rk, rule_j=rj, rule_term_offsets=off, term_k=tk, term_j=tj,
                               name=(desc.name + "+unions") if desc.name else "unions")


def small_1k(seed: int = 1001):
    """1,024 neurons, out-degree U{1..8}, 2 firing + 1 forgetting rule,
    d in [0,3], spikes U[0,10]; 100 steps, first-applicable selection."""
    s = random_system(1024, seed, outdeg=(1, 8), rules=(3, 3), d_range=(0, 3),
                      spikes=(0, 10), name="small-1k")
    return s, 100, SEL_FIRST


def large_1m(seed: int = 2002, q: int = 1 << 20):
    """1,048,576 neurons, out-degree U{8..24}, 3 firing + 1 forgetting rule,
    d in [0,5], spikes U[0,20]; 1,000 steps, Philox-keyed selection."""
    s = random_system(q, seed, outdeg=(8, 24), rules=(4, 4), d_range=(0, 5),
                      spikes=(0, 20), name=f"large-{q}")
    return s, 1000, SEL_PHILOX


def skewed_2m(seed: int = 3003, q: int = 1 << 21):
    """2,097,152 neurons, truncated Zipf(2.1) out-degree on [1, 4096],
    2 firing + 1 forgetting rule, d in [0,3], spikes U[0,20]; 256 steps, Philox."""
    s = random_system(q, seed, zipf=(2.1, 1, 4096), rules=(3, 3), d_range=(0, 3),
                      spikes=(0, 20), name=f"skewed-{q}")
    return s, 256, SEL_PHILOX


def skewed_dense_copy(seed: int = 3004):
    """The 16,384-neuron copy of the skewed workload, for the dense baseline."""
    return skewed_2m(seed, q=16384)


def batch_sizes(rng: np.random.Generator, count: int, lo: int = 64, hi: int = 65536) -> np.ndarray:
    """Neuron counts log-uniform in [lo, hi] (floor)."""
    x = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return np.floor(x).astype(np.int64).clip(lo, hi)


def _batch_member(args):
    i, qs, sd = args
    return random_system(int(qs), int(sd), outdeg=(4, 16), rules=(3, 3), d_range=(0, 4), spikes=(0, 10),
                         name=f"batch-{i}")


def batch_8k(seed: int = 4004, count: int = 8192, lo: int = 64, hi: int = 65536, processes: int = 0):
    """8,192 independent systems, q log-uniform in [64, 65536], out-degree
    U{4..16}, 2 firing + 1 forgetting rule, d in [0,4], spikes U[0,10];
    500 steps each, Philox with a per-system seed.  With processes > 1 the
    systems are drawn in a spawned process pool (same systems: each is
    seeded on its own)."""
    rng = np.random.default_rng(seed)
    sizes = batch_sizes(rng, count, lo, hi)
    seeds = rng.integers(1, 2**62, size=count, dtype=np.int64)
    work = [(i, int(qs), int(sd)) for i, (qs, sd) in enumerate(zip(sizes, seeds))]
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            systems = pool.map(_batch_member, work, chunksize=64)
    else:
        systems = [_batch_member(w) for w in work]
    return systems, 500, SEL_PHILOX


@dataclasses.dataclass
class Request:
    arrival_s: float
    q: int
    steps: int
    seed: int

    def system(self) -> SystemDesc:
        rng = np.random.default_rng(self.seed)
        lo, hi = 2, 32
        rules_n = int(rng.integers(2, 5))
        return random_system(self.q, self.seed + 1, outdeg=(lo, hi), rules=(rules_n, rules_n),
                             d_range=(0, 5), spikes=(0, 20), name=f"req-{self.seed}")


def serving_requests(rate_per_s: float, count: int, seed: int = 5005,
                     q_range=(1000, 1_000_000), steps_range=(10, 10_000)):
    """Poisson arrivals at ``rate_per_s``; each request a system of q
    log-uniform in q_range with a log-uniform step count."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    t = np.cumsum(gaps)
    qs = np.floor(np.exp(rng.uniform(math.log(q_range[0]), math.log(q_range[1]), size=count))).astype(np.int64)
    st = np.floor(np.exp(rng.uniform(math.log(steps_range[0]), math.log(steps_range[1]), size=count))).astype(np.int64)
    seeds = rng.integers(1, 2**62, size=count, dtype=np.int64)
    return [Request(float(a), int(qv), int(sv), int(sd)) for a, qv, sv, sd in zip(t, qs, st, seeds)]


def _request_member(req: Request) -> SystemDesc:
    return req.system()


def serving_systems(reqs, processes: int = 0):
    """The system of every request, drawn in a spawned process pool when
    processes > 1 (same systems: each is seeded on its own)."""
    if processes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_request_member, reqs, chunksize=1)
    return [_request_member(r) for r in reqs]


def subset_sum_shaped(n: int, seed: int = 6006, v=None) -> SystemDesc:
    """A stand-in with the sizes of Sec. 6's subset-sum family (the
    construction itself is not in the paper): for n numbers v_i drawn from
    U[0, 50] (or given), q = sum(v) + 2n + 2 neurons, m = sum(v) + 4n + 2
    rules and maximum out-degree z = n, with delays and a nondeterministic
    choice.  Neuron 0 (one spike, a -> a) feeds n "choice" neurons; each
    choice neuron holds a -> a;0 and a -> a;1 (both apply to one spike: the
    choice is the branch) and feeds its "check" neuron and the head of a
    chain of v_i neurons (a -> a;0 each, the last into the output neuron);
    each check neuron holds a -> a;0 and a^2 -> lambda and feeds the output
    neuron, the last neuron, which holds a -> a;0 with no synapses."""
    rng = np.random.default_rng(seed)
    vals = [int(x) for x in (v if v is not None else rng.integers(0, 51, size=n))]
    n = len(vals)
    total = sum(vals)
    q = total + 2 * n + 2
    ks, js, cs, ps, ds, offs = [], [], [], [], [], [0]
    def rule(k, j, c, p, d):
        ks.append(k); js.append(j); cs.append(c); ps.append(p); ds.append(d)
    src = 0
    choice0, check0, chain0, out = 1, 1 + n, 1 + 2 * n, q - 1
    targets = [[] for _ in range(q)]
    rule(1, 0, 1, 1, 0); offs.append(len(ks))                       # source
    targets[src] = list(range(choice0, choice0 + n))
    heads = []
    pos = chain0
    for i in range(n):
        heads.append(pos if vals[i] > 0 else -1)
        pos += vals[i]
    for i in range(n):                                               # choice neurons
        rule(1, 0, 1, 1, 0); rule(1, 0, 1, 1, 1); offs.append(len(ks))
        targets[choice0 + i] = [check0 + i] + ([heads[i]] if heads[i] >= 0 else [])
    for i in range(n):                                               # check neurons
        rule(1, 0, 1, 1, 0); rule(2, 0, 2, 0, 0); offs.append(len(ks))
        targets[check0 + i] = [out]
    pos = chain0
    for i in range(n):                                               # chains
        for t in range(vals[i]):
            rule(1, 0, 1, 1, 0); offs.append(len(ks))
            targets[pos + t] = [pos + t + 1] if t + 1 < vals[i] else [out]
        pos += vals[i]
    rule(1, 0, 1, 1, 0); offs.append(len(ks))                        # output
    init = np.zeros(q, np.int32)
    init[src] = 1
    so = np.zeros(q + 1, np.int64)
    so[1:] = np.cumsum([len(t) for t in targets])
    tg = np.asarray([x for t in targets for x in t], np.int32)
    a = lambda x: np.asarray(x, np.int32)
    return SystemDesc(q=q, init_spikes=init, rule_offsets=np.asarray(offs, np.int64),
                      rule_k=a(ks), rule_j=a(js), rule_c=a(cs), rule_p=a(ps), rule_d=a(ds),
                      syn_offsets=so, syn_targets=tg, out_neuron=out, seed=seed, name=f"subset-sum-shaped-{n}")


def sort_system(values) -> SystemDesc:
    """The sorting system of Sec. 6 for the given natural numbers (Table 1's
    layout): neurons i_1..i_n, s_1..s_n, o_1..o_n.

    i_k holds v_k spikes and the rule a+/a -> a (k=1, j=1, c=1, p=1) with
    synapses to every s_j.  s_j fires a^(n-j+1) -> a to o_j..o_n and forgets
    every other count in 1..n.  For n = 3 the rule order inside s_j is the one
    printed in Table 1 (r_4..r_12); for other n the firing rule comes first and
    the forgetting rules follow in ascending count.
    """
    v = [int(x) for x in values]
    n = len(v)
    q = 3 * n
    init = np.zeros(q, np.int32)
    init[:n] = v
    ks, js, cs, ps, ds, offs = [], [], [], [], [], [0]
    for _ in range(n):                          # i_k: a+/a -> a
        ks.append(1); js.append(1); cs.append(1); ps.append(1); ds.append(0)
        offs.append(offs[-1] + 1)
    table1_forget = {1: [2, 1], 2: [3, 1], 3: [2, 3]}
    for jn in range(1, n + 1):                   # s_j
        fire = n - jn + 1
        forget = table1_forget[jn] if n == 3 else [s for s in range(1, n + 1) if s != fire]
        ks.append(fire); js.append(0); cs.append(fire); ps.append(1); ds.append(0)
        for s in forget:
            ks.append(s); js.append(0); cs.append(s); ps.append(0); ds.append(0)
        offs.append(offs[-1] + 1 + len(forget))
    for _ in range(n):                          # o_k: no rules
        offs.append(offs[-1])
    so, tg = [0], []
    for _ in range(n):
        tg.extend(range(n, 2 * n)); so.append(len(tg))
    for jn in range(1, n + 1):
        tg.extend(range(2 * n + jn - 1, 3 * n)); so.append(len(tg))
    for _ in range(n):
        so.append(len(tg))
    a = lambda x: np.asarray(x, np.int32)
    return SystemDesc(q=q, init_spikes=init, rule_offsets=np.asarray(offs, np.int64),
                      rule_k=a(ks), rule_j=a(js), rule_c=a(cs), rule_p=a(ps), rule_d=a(ds),
                      syn_offsets=np.asarray(so, np.int64), syn_targets=a(tg),
                      out_neuron=2 * n, seed=0, name=f"sort-{n}")
