"""Computation-tree exploration on the GPU library (host orchestration only).

The paper's systems are nondeterministic (Sec. 2): at step k every idle
open neuron with applicable rules picks one, and each combination -- a
spiking vector of SV_k -- is one branch.  explore() walks that tree
breadth first with the library's own step: for each configuration it reads
how many rules each neuron may choose (snp_count_choices), enumerates the
combinations in a fixed order (mixed radix over the neurons with more than
one choice, lowest neuron id the fastest digit), and runs each as one
forced step (snp_set_choices + snp_step).  Children equal as configurations
(C, D, P) are merged.  Every step runs in the CUDA library; this module
only marshals states and choices.
"""
from __future__ import annotations

import dataclasses
import hashlib

import numpy as np

from . import libsnp


@dataclasses.dataclass
class Tree:
    states: list        # (C, D, P) per node, caller's neuron order
    depth: list         # level of each node
    edges: list         # (parent, child, choice index vector) per executed branch
    halted: set         # nodes at a fixed point (no branch)
    truncated: set      # nodes whose branches were cut at max_branches


def _key(C, D, P) -> bytes:
    h = hashlib.blake2b(digest_size=16)
    for a in (C, D, P):
        h.update(np.ascontiguousarray(a, np.int32).tobytes())
    return h.digest()


def branch_choices(counts: np.ndarray, limit: int):
    """The choice vectors of one configuration, in the fixed order, at most
    `limit` of them: neurons with one choice take 0; the others run through
    their choices as digits of a mixed-radix counter."""
    counts = np.asarray(counts, np.int64)
    free = np.nonzero(counts > 1)[0]
    idx = np.zeros(len(counts), np.int32)
    out = [idx.copy()]
    while len(out) < limit:
        for pos in free:                  # increment the counter
            idx[pos] += 1
            if idx[pos] < counts[pos]:
                break
            idx[pos] = 0
        else:
            return out, False             # wrapped around: all enumerated
        out.append(idx.copy())
    total = int(np.prod(counts[free], dtype=object)) if len(free) else 1
    return out, total > limit


def explore(desc, depth: int, *, max_branches: int = 1024, max_nodes: int = 100000,
            engine: int = libsnp.SNP_ENGINE_AUTO, batched: bool = None, chunk: int = 8192) -> Tree:
    """Breadth-first computation tree of `desc` from its initial
    configuration, `depth` levels deep (level = step).

    batched (default: when the system has at most 8,192 neurons): each level
    runs as snp_branch_step launches of up to `chunk` configurations, which
    also return the next level's choice counts; otherwise every branch is
    one forced snp_step."""
    if batched is None:
        batched = desc.q <= 8192 and engine in (libsnp.SNP_ENGINE_AUTO, libsnp.SNP_ENGINE_LAUNCH,
                                                libsnp.SNP_ENGINE_RESIDENT)
    sys_ = libsnp.System(desc, select=libsnp.SNP_SELECT_FIRST, engine=engine)
    try:
        if batched:
            return _explore_batched(sys_, desc, depth, max_branches, max_nodes, chunk)
        C0 = np.array(desc.init_spikes, np.int32)
        D0 = np.zeros(desc.q, np.int32)
        P0 = np.full(desc.q, -1, np.int32)
        tree = Tree(states=[(C0, D0, P0)], depth=[0], edges=[], halted=set(), truncated=set())
        seen = {_key(C0, D0, P0): 0}
        frontier = [0]
        for level in range(depth):
            nxt = []
            for node in frontier:
                C, D, P = tree.states[node]
                sys_.set_state(C, D, P, level)
                counts = sys_.count_choices()
                combos, cut = branch_choices(counts, max_branches)
                if cut:
                    tree.truncated.add(node)
                for choice in combos:
                    sys_.set_state(C, D, P, level)
                    sys_.set_choices(choice)
                    if sys_.step(1) == 0:     # a fixed point: no branch
                        tree.halted.add(node)
                        break
                    Cc, Dc, Pc, _ = sys_.get_state()
                    key = _key(Cc, Dc, Pc)
                    child = seen.get(key)
                    if child is None:
                        if len(tree.states) >= max_nodes:
                            return tree
                        child = len(tree.states)
                        seen[key] = child
                        tree.states.append((Cc, Dc, Pc))
                        tree.depth.append(level + 1)
                        nxt.append(child)
                    tree.edges.append((node, child, choice))
            frontier = nxt
        return tree
    finally:
        sys_.close()


def _explore_batched(sys_, desc, depth, max_branches, max_nodes, chunk):
    C0 = np.array(desc.init_spikes, np.int32)
    D0 = np.zeros(desc.q, np.int32)
    P0 = np.full(desc.q, -1, np.int32)
    sys_.set_state(C0, D0, P0, 0)
    tree = Tree(states=[(C0, D0, P0)], depth=[0], edges=[], halted=set(), truncated=set())
    seen = {_key(C0, D0, P0): 0}
    counts = {0: sys_.count_choices()}
    frontier = [0]
    for level in range(depth):
        work = []  # (parent, choice vector)
        for node in frontier:
            combos, cut = branch_choices(counts[node], max_branches)
            if cut:
                tree.truncated.add(node)
            work.extend((node, c) for c in combos)
        nxt = []
        for a in range(0, len(work), chunk):
            part = work[a:a + chunk]
            Cs = np.stack([tree.states[p][0] for p, _ in part])
            Ds = np.stack([tree.states[p][1] for p, _ in part])
            Ps = np.stack([tree.states[p][2] for p, _ in part])
            ch = np.stack([c for _, c in part])
            C1, D1, P1, ex, bad, cnt = sys_.branch_step(Cs, Ds, Ps, ch)
            if bad.any():
                raise RuntimeError("a choice index was out of range")
            for r, (parent, choice) in enumerate(part):
                if not ex[r]:
                    tree.halted.add(parent)
                    continue
                key = _key(C1[r], D1[r], P1[r])
                child = seen.get(key)
                if child is None:
                    if len(tree.states) >= max_nodes:
                        return tree
                    child = len(tree.states)
                    seen[key] = child
                    tree.states.append((C1[r].copy(), D1[r].copy(), P1[r].copy()))
                    tree.depth.append(level + 1)
                    counts[child] = cnt[r].copy()
                    nxt.append(child)
                tree.edges.append((parent, child, choice))
        frontier = nxt
    return tree
