"""GPU parity of the ELL form (pull and push) and of the uncompressed
("Sparse", dense M_Pi) form against the CPU oracle, bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2408_04343_gb300 import libsnp, synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SEL = {oracle.FIRST: libsnp.SNP_SELECT_FIRST, oracle.PHILOX: libsnp.SNP_SELECT_PHILOX}
FORMS = {"ell-pull": (libsnp.SNP_FORM_ELL, libsnp.SNP_PROP_PULL),
         "ell-push": (libsnp.SNP_FORM_ELL, libsnp.SNP_PROP_PUSH),
         "dense": (libsnp.SNP_FORM_DENSE, libsnp.SNP_PROP_PULL)}


@pytest.fixture(scope="module", autouse=True)
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2408_04343_gb300 import build
    build.build()
    libsnp.load()


def compare(desc, nsteps, mode, seed, form, chunks=(1,)):
    f, p = FORMS[form]
    gs = libsnp.System(desc, form=f, prop=p, select=SEL[mode], seed=seed)
    st = oracle.initial_state(desc)
    k, ci = 0, 0
    last_S = np.full(desc.q, -1, np.int32)
    while k < nsteps:
        n = min(chunks[ci % len(chunks)], nsteps - k)
        ci += 1
        done = gs.step(n)
        ex, S = oracle.run(desc, st, n, mode, seed, step0=k)
        assert done == ex, (form, k, done, ex)
        if ex:
            last_S = S
        C, D, P, kk = gs.get_state()
        assert kk == k + ex
        assert (C == st[0]).all(), f"{form}: C differs after step {k + ex}"
        assert (D == st[1]).all() and (P == st[2]).all(), f"{form}: D/P differ after step {k + ex}"
        assert (gs.spiking() == last_S).all(), f"{form}: S differs after step {k + ex}"
        k += ex
        if ex < n:
            break
    gs.close()
    return k


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("q", [1, 31, 33, 200, 3001])
def test_forms_ragged_sizes(form, q):
    d = synth.random_system(q, 300 + q, outdeg=(1, 8), rules=(2, 4), d_range=(0, 3), spikes=(0, 10))
    for mode in (oracle.FIRST, oracle.PHILOX):
        compare(d, 30, mode, 11 + q, form, chunks=(1, 5, 13))


@pytest.mark.parametrize("form", list(FORMS))
def test_forms_small_1k_workload(form):
    d, nsteps, mode = synth.small_1k()
    compare(d, nsteps, mode, d.seed, form, chunks=(1, 9, 40))


@pytest.mark.parametrize("form", list(FORMS))
def test_forms_sort_system(form):
    for v in ([3, 2, 1], [7, 3, 3, 9, 1]):
        d = synth.sort_system(v)
        assert compare(d, 100, oracle.FIRST, 0, form, chunks=(1, 50)) == max(v) + 1


def test_forms_hand_delay_traces():
    from tests.test_oracle import make_desc
    cases = [
        make_desc(2, [[(1, 0, 1, 1, 3)], []], [(0, 1)], [1, 0]),
        make_desc(3, [[(1, 0, 1, 1, 2)], [], [(1, 0, 1, 1, 0)]], [(2, 0), (0, 1)], [1, 0, 1]),
        make_desc(4, [[(1, 0, 1, 1, 1)], [], [(2, 0, 2, 1, 0)], [(1, 0, 1, 1, 0)]],
                  [(0, 1), (2, 0), (3, 2)], [1, 0, 1, 1]),
    ]
    for d in cases:
        for form in FORMS:
            compare(d, 20, oracle.FIRST, 0, form)


@pytest.mark.parametrize("form", ["ell-pull", "ell-push"])
def test_ell_skewed_degrees(form):
    d = synth.random_system(30000, 9, zipf=(2.1, 1, 4096), rules=(3, 3), d_range=(0, 3), spikes=(0, 20))
    compare(d, 40, oracle.PHILOX, 17, form, chunks=(1, 19, 20))


def test_dense_skewed_16k_copy_sampled():
    """The 16,384-neuron copy of the skewed workload through the dense
    transition matrix (49,152 x 16,384 int32, 3.2 GB), compared after steps
    1, 2 and 12."""
    d, _, mode = synth.skewed_dense_copy()
    compare(d, 12, mode, d.seed, "dense", chunks=(1, 1, 10))


def test_overflow_is_reported_in_every_form():
    from tests.test_oracle import make_desc
    d = make_desc(2, [[(1, 1, 1, 1000, 0)], []], [(0, 1)], [10, 2**31 - 600])
    for form, (f, p) in FORMS.items():
        g = libsnp.System(d, form=f, prop=p)
        with pytest.raises(libsnp.SnpError) as ei:
            g.step(5)
        assert ei.value.status == libsnp.SNP_ERR_OVERFLOW, form


@pytest.mark.parametrize("form", list(FORMS) + ["opt"])
def test_paper_families_sort_and_subset_sum_shaped(form):
    """Sec. 6's families on every form: the sort system on a worst-case
    input (n, n-1, ..., 1) halts after n + 1 steps with o_k = k (the closed
    form) and matches the oracle step for step; the subset-sum-shaped
    stand-in (delays, a branching choice per number) matches it under
    Philox."""
    n = 40
    d = synth.sort_system(list(range(n, 0, -1)))
    if form == "opt":
        gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
        done = gs.step(4 * n)
        C = gs.get_state()[0]
        gs.close()
    else:
        done = compare(d, 4 * n, oracle.FIRST, 0, form, chunks=(5, 13))
        st = oracle.initial_state(d)
        oracle.run(d, st, 4 * n)
        C = st[0]
    assert done == n + 1
    assert (C[2 * n:] == np.arange(1, n + 1)).all()
    s = synth.subset_sum_shaped(12, seed=3)
    if form == "opt":
        gs = libsnp.System(s, select=libsnp.SNP_SELECT_PHILOX, seed=8)
        done = gs.step(100)
        st = oracle.initial_state(s)
        ex, S = oracle.run(s, st, 100, oracle.PHILOX, 8)
        C, D, P, _ = gs.get_state()
        assert done == ex and (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all()
        gs.close()
    else:
        compare(s, 100, oracle.PHILOX, 8, form, chunks=(7,))
