"""The tiled engine's packed layout, checked on the CPU (no GPU).

`tiled_layout_check.cpp` links the library's packer (csrc/pack.cpp), packs
a seeded random system for a 152-SM device with the cluster counts per wave
that a GB300 reports at about 225 KB of shared memory per CTA, decodes
every CTA's entries back into in-edges and checks that each in-edge appears
exactly once in its (target range, source partition) CTA, that a target's
in-edges from one partition lie in one thread's run (run-length layout:
that thread alone writes the accumulator), that the entry buffer has its
two rows of slack, and that shared memory fits.  The cases span the
layouts: the 1M-neuron and 2M-neuron skewed workloads' shapes (byte
accumulators, run-length entries, clusters of 2 and 4), 32-bit
accumulators with paired and plain target words, more partitions than a
cluster holds (the two-launch form), and tiny and ragged systems.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2408_04343_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("tiled") / "tiled_layout_check")
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        os.path.join(ROOT, "tests", "tiled_layout_check.cpp"), os.path.join(CSRC, "pack.cpp"),
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, q, deg_lo, deg_hi, p_max, zipf, seed):
    r = subprocess.run([exe, str(q), str(deg_lo), str(deg_hi), str(p_max), str(int(zipf)), str(seed)],
                       capture_output=True, text=True, timeout=300)
    line = r.stdout.strip().splitlines()[-1] if r.stdout.strip() else ""
    assert r.returncode == 0, (r.returncode, line, r.stderr[-2000:])
    return {k: int(v) for k, v in (kv.split("=") for kv in line.split())}


CASES = {
    # (q, out-degree lo, hi, largest p, Zipf out-degree, seed), expected shape
    "1m_uniform": ((1 << 20, 8, 24, 3, False, 5), dict(P=2, G=152, rle=1, acc8=1)),
    "2m_skewed": ((1 << 21, 1, 1, 3, True, 6), dict(rle=1, acc8=1, rin_esm=1)),
    "paired_32bit": ((65536, 8, 24, 100, False, 3), dict(pairs=1, acc8=0, rle=0)),
    "words_32bit": ((300000, 2, 6, 1000, False, 8), dict(pairs=0, acc8=0, rle=0, e_bits=16)),
    "two_launch": ((1 << 20, 2, 4, 1000, False, 7), dict(acc8=0, rle=0)),
    "q33": ((33, 1, 4, 3, False, 9), dict(rle=1)),
    "q1": ((1, 0, 0, 3, False, 10), dict(edges=0)),
    "sparse_ragged": ((5000, 0, 3, 3, False, 11), dict(rle=1)),
}


@pytest.mark.parametrize("name", list(CASES))
def test_tiled_layout_decodes_to_the_in_lists(checker, name):
    args, want = CASES[name]
    got = _run(checker, *args)
    assert got["mismatched"] == 0 and got["split_targets"] == 0
    assert got["slack"] == 1 and got["smem_ok"] == 1
    assert got["edges"] == got["num_syn"]
    for k, v in want.items():
        assert got[k] == v, (k, got)
    if name == "2m_skewed":
        assert got["G"] <= 152          # one wave of clusters
    if name == "two_launch":
        assert got["P"] > 8             # more partitions than one cluster holds
    if got["rle"]:
        # padding of the run-length layout: runs cut at target boundaries
        # stay within a few percent of the in-edges on the large workloads
        if args[0] >= 1 << 20:
            assert got["positions"] <= 1.10 * got["edges"], got
