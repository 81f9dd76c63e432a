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
