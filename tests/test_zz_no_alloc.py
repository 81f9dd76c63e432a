"""snp_step_noalloc against snp_step.

snp_step_noalloc is the entry point for callers that cannot allocate device
memory (for example a plugin inside a framework that owns the whole device
memory pool, or a latency-critical loop that must not risk an allocation's
device synchronization).  It must give exactly the results of the ordinary
entry point, which allocates its working buffers per system: this test runs
both on the same seeded systems, calls the non-allocating one twice in a row
(so the second call starts from the static scratch the first call left
behind), and compares configuration, delay status, pending rules, spiking
vector and executed step counts bit for bit after each call.
"""
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


def device_tables(d):
    """The caller-side device arrays: rules as int32 columns and the
    in-neighbour lists (transpose of the synapse lists) as CSR."""
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
    src = np.repeat(np.arange(d.q, dtype=np.int64), np.diff(d.syn_offsets))
    tgt = d.syn_targets.astype(np.int64)
    order = np.argsort(tgt, kind="stable")
    in_off = np.zeros(d.q + 1, np.int64)
    np.cumsum(np.bincount(tgt, minlength=d.q), out=in_off[1:])
    return dict(rule_offsets=dev(d.rule_offsets), rule_k=dev(d.rule_k), rule_j=dev(d.rule_j),
                rule_c=dev(d.rule_c), rule_p=dev(d.rule_p), rule_d=dev(d.rule_d),
                in_offsets=dev(in_off), in_sources=dev(src[order]))


@pytest.mark.parametrize("q,select", [(20000, libsnp.SNP_SELECT_PHILOX), (20000, libsnp.SNP_SELECT_FIRST),
                                      (libsnp.SNP_NOALLOC_MAX_Q, libsnp.SNP_SELECT_PHILOX)])
def test_noalloc_matches_snp_step_on_two_calls(q, select):
    d = synth.random_system(q, 900 + q, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    seed = 12345
    ref = libsnp.System(d, select=select, seed=seed, engine=libsnp.SNP_ENGINE_LAUNCH)
    tabs = device_tables(d)
    C = torch.from_numpy(d.init_spikes.astype(np.int32)).cuda()
    D = torch.zeros(q, dtype=torch.int32, device="cuda")
    P = torch.full((q,), -1, dtype=torch.int32, device="cuda")
    S = torch.full((q,), -1, dtype=torch.int32, device="cuda")
    k = 0
    for n in (23, 31):
        done = libsnp.snp_step_noalloc(q, d.m, C=C, D=D, P=P, S=S, select=select, seed=seed, step=k, n=n,
                                       **tabs)
        ref_done = ref.step(n)
        assert done == ref_done
        k += done
        rC, rD, rP, rk = ref.get_state()
        assert rk == k
        assert (C.cpu().numpy() == rC).all()
        assert (D.cpu().numpy() == rD).all()
        assert (P.cpu().numpy() == rP).all()
        assert (S.cpu().numpy() == ref.spiking()).all()
    ref.close()


def test_noalloc_rejects_too_large_systems():
    q = libsnp.SNP_NOALLOC_MAX_Q + 1
    x = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.snp_step_noalloc(q, 1, x, x, x, x, x, x, x, x, x, x, x, x, n=1)
    assert ei.value.status == libsnp.SNP_ERR_INVALID
    assert "SNP_NOALLOC_MAX_Q" in str(ei.value)


@pytest.mark.parametrize("field,value", [("rule_p", 70000), ("rule_d", 70000), ("rule_c", -1)])
def test_noalloc_rejects_fired_rules_out_of_range(field, value):
    # The device arrays bypass snp_create's validation, so the kernels check
    # the fields of every rule they fire; a step that fires one out of range
    # must report SNP_ERR_INVALID rather than pack a wrapped value.  A valid
    # call afterwards still matches snp_step.
    q, select, seed = 4096, libsnp.SNP_SELECT_FIRST, 7
    d = synth.random_system(q, 31, outdeg=(2, 8), rules=(3, 3), d_range=(0, 3), spikes=(0, 10))
    tabs = device_tables(d)
    bad = dict(tabs)
    col = tabs[field].clone()
    firing = torch.from_numpy(d.rule_p > 0).cuda()
    col[firing] = value
    bad[field] = col

    def fresh():
        return (torch.from_numpy(d.init_spikes.astype(np.int32)).cuda(),
                torch.zeros(q, dtype=torch.int32, device="cuda"),
                torch.full((q,), -1, dtype=torch.int32, device="cuda"),
                torch.full((q,), -1, dtype=torch.int32, device="cuda"))

    C, D, P, S = fresh()
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.snp_step_noalloc(q, d.m, C=C, D=D, P=P, S=S, select=select, seed=seed, step=0, n=5, **bad)
    assert ei.value.status == libsnp.SNP_ERR_INVALID

    C, D, P, S = fresh()
    ref = libsnp.System(d, select=select, seed=seed, engine=libsnp.SNP_ENGINE_LAUNCH)
    done = libsnp.snp_step_noalloc(q, d.m, C=C, D=D, P=P, S=S, select=select, seed=seed, step=0, n=9, **tabs)
    assert done == ref.step(9)
    rC, rD, rP, _ = ref.get_state()
    assert (C.cpu().numpy() == rC).all() and (D.cpu().numpy() == rD).all() and (P.cpu().numpy() == rP).all()
    assert (S.cpu().numpy() == ref.spiking()).all()
    ref.close()


def dag_system(q, seed):
    """A system whose synapses only go forward (i -> i+1 .. i+64) and whose
    firing rules need an exact spike count: spikes drain towards the last
    neurons and stop where no count matches, so it reaches a fixed point in
    about twenty steps."""
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
            tg += sorted(int(x) for x in rng.choice(cand, size=min(len(cand), int(rng.integers(0, 4))),
                                                    replace=False))
        so.append(len(tg))
    a32 = lambda x: np.asarray(x, np.int32)
    return synth.SystemDesc(q=q, init_spikes=a32(rng.integers(0, 6, size=q)), rule_offsets=np.asarray(offs, np.int64),
                            rule_k=a32(ks), rule_j=a32(js), rule_c=a32(cs), rule_p=a32(ps), rule_d=a32(ds),
                            syn_offsets=np.asarray(so, np.int64), syn_targets=a32(tg))


def fresh_state(d):
    return (torch.from_numpy(d.init_spikes.astype(np.int32)).cuda(),
            torch.zeros(d.q, dtype=torch.int32, device="cuda"),
            torch.full((d.q,), -1, dtype=torch.int32, device="cuda"),
            torch.full((d.q,), -1, dtype=torch.int32, device="cuda"))


@pytest.mark.parametrize("select", [libsnp.SNP_SELECT_FIRST, libsnp.SNP_SELECT_PHILOX])
def test_noalloc_halts_partway_like_snp_step_and_the_oracle(select):
    """A call that reaches a fixed point partway reports the steps it
    executed, leaves S holding the last executed step's spiking vector, and
    a later call at the fixed point executes nothing and leaves S alone --
    exactly as snp_step and the CPU oracle do.  The buffers are passed as
    raw device pointers (data_ptr integers) with num_in given."""
    d = dag_system(5000, 70)
    seed = 12345
    omode = oracle.FIRST if select == libsnp.SNP_SELECT_FIRST else oracle.PHILOX
    ref = libsnp.System(d, select=select, seed=seed, engine=libsnp.SNP_ENGINE_LAUNCH)
    tabs = device_tables(d)
    raw = {k: v.data_ptr() for k, v in tabs.items()}
    C, D, P, S = fresh_state(d)
    st = oracle.initial_state(d)
    k, halted_seen = 0, False
    for n in (9, 40, 10):
        done = libsnp.snp_step_noalloc(d.q, d.m, C=C.data_ptr(), D=D.data_ptr(), P=P.data_ptr(), S=S.data_ptr(),
                                       num_in=tabs["in_sources"].numel(), select=select, seed=seed, step=k, n=n,
                                       **raw)
        ex, S_or = oracle.run(d, st, n, omode, seed, step0=k)
        assert done == ref.step(n) == ex
        halted_seen |= done < n
        k += done
        rC, rD, rP, rk = ref.get_state()
        assert rk == k
        for got, want in ((C, rC), (D, rD), (P, rP)):
            assert (got.cpu().numpy() == want).all()
        assert (C.cpu().numpy() == st[0]).all() and (D.cpu().numpy() == st[1]).all()
        assert (P.cpu().numpy() == st[2]).all()
        if done:
            assert (S.cpu().numpy() == ref.spiking()).all() and (S.cpu().numpy() == S_or).all()
        else:
            assert (S.cpu().numpy() == ref.spiking()).all()   # untouched by a call that ran no step
    assert halted_seen and done == 0
    ref.close()


def test_noalloc_raw_pointer_without_num_in_is_refused():
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(TypeError):
        libsnp.snp_step_noalloc(4, 1, x, x, x, x, x, x, x, x.data_ptr(), x, x, x, x, n=1)


@pytest.mark.parametrize("case", ["src_high", "src_negative", "offsets", "P_other", "D_without_P", "C_negative"])
def test_noalloc_rejects_out_of_range_inputs(case):
    """An in-neighbour index outside 0..q-1, in_offsets beyond num_in, a
    pending rule that is not its neuron's, D > 0 with no pending rule or a
    negative spike count return SNP_ERR_INVALID; a valid call afterwards on
    fresh buffers matches snp_step."""
    d = synth.random_system(3000, 33, outdeg=(2, 8), rules=(3, 3), d_range=(0, 3), spikes=(0, 10))
    tabs = device_tables(d)
    bad = dict(tabs)
    C, D, P, S = fresh_state(d)
    i = 1234
    if case == "src_high":
        col = tabs["in_sources"].clone(); col[17] = d.q; bad["in_sources"] = col
    elif case == "src_negative":
        col = tabs["in_sources"].clone(); col[17] = -5; bad["in_sources"] = col
    elif case == "offsets":
        col = tabs["in_offsets"].clone(); col[-1] = tabs["in_sources"].numel() + 3; bad["in_offsets"] = col
    elif case == "P_other":
        P[i] = int(d.rule_offsets[i + 1]); D[i] = 1
    elif case == "D_without_P":
        D[i] = 2
    else:
        C[i] = -1
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.snp_step_noalloc(d.q, d.m, C=C, D=D, P=P, S=S, step=0, n=3, **bad)
    assert ei.value.status == libsnp.SNP_ERR_INVALID
    C, D, P, S = fresh_state(d)
    ref = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST, engine=libsnp.SNP_ENGINE_LAUNCH)
    assert libsnp.snp_step_noalloc(d.q, d.m, C=C, D=D, P=P, S=S, step=0, n=6, **tabs) == ref.step(6)
    rC, rD, rP, _ = ref.get_state()
    assert (C.cpu().numpy() == rC).all() and (D.cpu().numpy() == rD).all() and (P.cpu().numpy() == rP).all()
    ref.close()


def test_noalloc_rejects_more_than_2_31_steps():
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.snp_step_noalloc(4, 1, x, x, x, x, x, x, x, x, x, x, x, x, n=2**31)
    assert ei.value.status == libsnp.SNP_ERR_INVALID
