"""Host-side checks of libsnp that need no GPU: the library loads and exports
every call include/snp.h declares; the paper-format exporters reproduce
Tables 1-3; the element-count formulas reproduce Sec. 6's printed values;
malformed systems are rejected before any device work."""
import os
import re

import numpy as np
import pytest

from paper_2408_04343_gb300 import libsnp, synth
from paper_2408_04343_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def header_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\**\s*(snp_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_call():
    import ctypes as ct
    lib = ct.CDLL(libsnp.library_path())
    names = header_functions()
    assert "snp_create" in names and "snp_step" in names and "snp_batch_submit" in names
    for n in names:
        assert hasattr(lib, n), n


def load_table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        if line.startswith("#") or not line.strip():
            continue
        rows.append(line.split()[1:])
    return rows


def test_export_dense_is_table1():
    M = libsnp.export_dense(synth.sort_system([3, 2, 1]))
    T = np.array([[int(x) for x in r] for r in load_table("sort3_table1_dense.txt")])
    assert (M == T).all()


def test_export_ell_is_table2():
    vals, nrn = libsnp.export_ell(synth.sort_system([3, 2, 1]))
    rows = load_table("sort3_table2_ell.txt")   # one line per rule (column)
    assert vals.shape == (4, 12)
    for r, entries in enumerate(rows):
        for row, e in enumerate(entries):
            if e == "-":
                assert nrn[row, r] == -1 and vals[row, r] == 0
            else:
                v, n = (int(x) for x in e.split(","))
                assert (vals[row, r], nrn[row, r]) == (v, n)


def test_export_compressed_is_table3():
    sy = libsnp.export_compressed(synth.sort_system([3, 2, 1]))
    rows = load_table("sort3_table3_compressed.txt")   # one line per neuron (column)
    assert sy.shape == (3, 9)
    for col, entries in enumerate(rows):
        for row, e in enumerate(entries):
            assert sy[row, col] == (-1 if e == "-" else int(e))


def test_paper_size_formulas():
    forms = {"sparse": libsnp.SNP_FORM_DENSE, "ell": libsnp.SNP_FORM_ELL, "compressed": libsnp.SNP_FORM_OPT}
    for line in open(os.path.join(GOLD, "paper_size_formulas.txt")):
        if line.startswith("#") or not line.strip():
            continue
        fam, q, m, z, fmt, printed, agrees = line.split()
        got = libsnp.paper_format_elements(forms[fmt], int(q), int(m), int(z))
        if agrees == "yes":
            assert got == int(printed), (fam, fmt)
        else:
            assert got != int(printed) and got == 3060901  # the printed value has a typo


def _bad(desc):
    with pytest.raises(libsnp.SnpError) as ei:
        libsnp.System(desc)
    assert ei.value.status == libsnp.SNP_ERR_INVALID


def test_rejects_malformed_systems():
    base = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d.syn_targets = d.syn_targets.copy()
    d.syn_targets[d.syn_offsets[3]] = 3          # self-loop
    _bad(d)
    d = synth.random_system(40, 7, outdeg=(2, 5), rules=(2, 3))
    d.syn_targets = d.syn_targets.copy()
    d.syn_targets[d.syn_offsets[5] + 1] = d.syn_targets[d.syn_offsets[5]]   # duplicate
    _bad(d)
    d = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d.syn_targets = d.syn_targets.copy()
    d.syn_targets[0] = 40                        # out of range
    _bad(d)
    d = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d.rule_d = d.rule_d.copy()
    d.rule_p = d.rule_p.copy()
    d.rule_p[0] = 0
    d.rule_d[0] = 2                              # forgetting rule with a delay
    _bad(d)
    d = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d.rule_p = d.rule_p.copy()
    d.rule_p[1] = 70000                          # p out of range
    _bad(d)
    d = synth.random_system(40, 7, outdeg=(1, 5), rules=(2, 3))
    d.init_spikes = d.init_spikes.copy()
    d.init_spikes[2] = -1
    _bad(d)
    assert base.q == 40


def test_union_descriptions_are_checked():
    """Union expressions: malformed term arrays are SNP_ERR_INVALID, refused
    on the host before any device work.  Unions the compiled applicability
    table cannot hold (K + L > 14, more than 4 rules) are packed as union
    records of the general rule table: 4 words per rule plus 2 per term."""
    import dataclasses
    base = synth.random_system(40, 9, outdeg=(1, 5), rules=(2, 3))
    u = synth.with_unions(base, 3)
    off = u.rule_term_offsets.copy(); off[5] = off[4]                  # rule 4 without a term
    _bad(dataclasses.replace(u, rule_term_offsets=off, term_k=u.term_k, term_j=u.term_j))
    tk = u.term_k.copy(); tk[2] = -1                                 # negative term
    _bad(dataclasses.replace(u, term_k=tk))
    _bad(dataclasses.replace(u, rule_term_offsets=None))             # terms without offsets
    for tk_big, tj_big in ((20, 0), (2, 13)):                        # K + L > 14 (K >= 2)
        tk = u.term_k.copy(); tj = u.term_j.copy(); tk[0] = tk_big; tj[0] = tj_big
        g = libsnp.System(dataclasses.replace(u, term_k=tk, term_j=tj), deferred=True)
        inf = g.info()
        assert inf.compiled_rules == 0 and inf.compact_rules == 0
        assert inf.rule_words == 4 * u.m + 2 * int(u.rule_term_offsets[-1])
        g.close()
    five = synth.with_unions(synth.random_system(40, 9, outdeg=(1, 5), rules=(5, 5)), 3)   # 5 rules per neuron
    g = libsnp.System(five, deferred=True)
    assert g.info().compiled_rules == 0 and g.info().rule_words == 4 * five.m + 2 * int(five.rule_term_offsets[-1])
    g.close()
    small = libsnp.System(u, deferred=True)                          # fits the record: compiled
    assert small.info().compiled_rules == 1
    small.close()


def test_strerror_names_every_status():
    lib = libsnp.load()
    for st in range(8):
        assert lib.snp_strerror(st)
    assert lib.snp_strerror(99) == b"unknown status"


def test_family_generators_have_the_papers_sizes():
    """The sort family (q = 3n, m = n + n^2, z = n) and the subset-sum-shaped
    stand-in (V = {1..100}: q = 5,252, m = 5,452, z = 100) have the sizes
    Sec. 6 states, so the size formulas give its printed element counts."""
    import numpy as np
    for n in (3, 10, 100):
        d = synth.sort_system(list(range(n, 0, -1)))
        z = int(np.diff(d.syn_offsets).max())
        assert (d.q, d.m, z) == (3 * n, n + n * n, n)
    d = synth.subset_sum_shaped(100, v=list(range(1, 101)))
    z = int(np.diff(d.syn_offsets).max())
    assert (d.q, d.m, z) == (5252, 5452, 100)
    assert libsnp.paper_format_elements(libsnp.SNP_FORM_OPT, d.q, d.m, z) == 562765
    assert libsnp.paper_format_elements(libsnp.SNP_FORM_ELL, d.q, d.m, z) == 1128165
    assert libsnp.paper_format_elements(libsnp.SNP_FORM_DENSE, d.q, d.m, z) == 28660765
    r = synth.subset_sum_shaped(30, seed=5)           # v drawn from U[0, 50]
    assert r.m - r.q == 2 * 30 and r.q >= 2 * 30 + 2
