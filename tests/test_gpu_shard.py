"""The neuron-sharded step (snp_shard_*) on one GPU: a system split by
neuron range into 1, 2 or 3 CUDA shards that exchange their emission slices
by device copies (the protocol of paper_2408_04343_gb300.shard) equals the
whole system's oracle result step for step: C, D, P, the spiking vector of
the last executed step and the executed step count, with delays, both
selections, unions of terms, and a system that reaches a fixed point."""
import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, shard, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEL = {oracle.FIRST: libsnp.SNP_SELECT_FIRST, oracle.PHILOX: libsnp.SNP_SELECT_PHILOX}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()


def _dag(q, seed):
    """Forward synapses and exact-count rules: a fixed point within ~20 steps."""
    rng = np.random.default_rng(seed)
    offs, ks, js, cs, ps, ds = [0], [], [], [], [], []
    for _ in range(q):
        for _ in range(2):
            k = int(rng.integers(1, 4))
            ks.append(k); js.append(0); cs.append(int(rng.integers(1, k + 1)))
            ps.append(int(rng.integers(1, 3))); ds.append(int(rng.integers(0, 3)))
        s_ = int(rng.integers(1, 4))
        ks.append(s_); js.append(0); cs.append(s_); ps.append(0); ds.append(0)
        offs.append(len(ks))
    tg, so = [], [0]
    for i in range(q):
        cand = np.arange(i + 1, min(q - 1, i + 64) + 1)
        if len(cand):
            tg += sorted(int(x) for x in rng.choice(cand, size=min(len(cand), int(rng.integers(0, 4))), replace=False))
        so.append(len(tg))
    a32 = lambda x: np.asarray(x, np.int32)
    return synth.SystemDesc(q=q, init_spikes=a32(rng.integers(0, 6, size=q)), rule_offsets=np.asarray(offs, np.int64),
                            rule_k=a32(ks), rule_j=a32(js), rule_c=a32(cs), rule_p=a32(ps), rule_d=a32(ds),
                            syn_offsets=np.asarray(so, np.int64), syn_targets=a32(tg))


SYSTEMS = {
    "random": lambda: synth.random_system(5000, 11, outdeg=(2, 12), rules=(3, 4), d_range=(0, 4), spikes=(0, 15)),
    "unions": lambda: synth.with_unions(synth.random_system(3001, 12, outdeg=(2, 8), rules=(2, 4), d_range=(0, 3),
                                                            spikes=(0, 10)), 13, terms=(1, 3)),
    "wide": lambda: synth.random_system(2000, 14, outdeg=(2, 8), rules=(5, 6), p_range=(1, 40), d_range=(0, 20),
                                        spikes=(0, 10)),
    "halting": lambda: _dag(4000, 70),
}


@pytest.mark.parametrize("kind", list(SYSTEMS))
@pytest.mark.parametrize("world", [1, 2, 3])
@pytest.mark.parametrize("mode", [oracle.FIRST, oracle.PHILOX])
def test_sharded_step_equals_oracle(kind, world, mode):
    d = SYSTEMS[kind]()
    seed = 99
    ranges, chunk = shard.shard_ranges(d.q, world)
    Es = [torch.zeros(world * chunk + 1, dtype=torch.int16, device="cuda") for _ in ranges]
    shards = [libsnp.Shard(d, lo, hi, select=SEL[mode], seed=seed, E=E) for (lo, hi), E in zip(ranges, Es)]
    ex = shard.local_exchange([(E, lo, hi) for (lo, hi), E in zip(ranges, Es)])
    st = oracle.initial_state(d)
    k, last_S = 0, np.full(d.q, -1, np.int32)
    for n in (1, 4, 25, 40):
        done = shard.run(shards, n, k, ex, lambda a: a)
        ex_or, S = oracle.run(d, st, n, mode, seed, step0=k)
        assert done == ex_or, (k, done, ex_or)
        if ex_or:
            last_S = S
        k += done
        parts = [sh.get_state() for sh in shards]
        C, D, P, Sg = (np.concatenate([p[i] for p in parts]) for i in range(4))
        assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all(), k
        assert (Sg == last_S).all(), k
        if done < n:
            break
    if kind == "halting":
        assert k < 70
    for sh in shards:
        sh.close()


def test_shard_checks_its_arguments():
    d = SYSTEMS["random"]()
    for lo, hi in ((-1, 10), (10, 10), (4000, 5001)):
        with pytest.raises(libsnp.SnpError) as ei:
            libsnp.Shard(d, lo, hi)
        assert ei.value.status == libsnp.SNP_ERR_INVALID
    sh = libsnp.Shard(d, 0, 100)
    with pytest.raises(libsnp.SnpError) as ei:
        sh.receive()                      # phase 2 before phase 1
    assert ei.value.status == libsnp.SNP_ERR_INVALID
    sh.close()
