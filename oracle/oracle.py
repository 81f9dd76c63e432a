"""ctypes front end of the C oracle (``snp_oracle.c``) -- test infrastructure.

Builds ``_build/liboracle.so`` with plain gcc on first use.  The state of a
system is (C, D, P): spikes, steps until reopening, pending rule id or -1.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

FIRST, PHILOX, FORCED = 0, 1, 2
_OK, _INVALID, _OOM, _OVERFLOW = 0, 1, 2, 5

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "snp_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


class OracleError(RuntimeError):
    pass


class OracleOverflow(OracleError):
    pass


class _Sys(ct.Structure):
    _fields_ = [("q", ct.c_int32),
                ("rule_off", ct.c_void_p), ("rk", ct.c_void_p), ("rj", ct.c_void_p),
                ("rc", ct.c_void_p), ("rp", ct.c_void_p), ("rd", ct.c_void_p),
                ("syn_off", ct.c_void_p), ("syn_tgt", ct.c_void_p),
                ("term_off", ct.c_void_p), ("tk", ct.c_void_p), ("tj", ct.c_void_p)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vendor code); with OpenMP when
    the compiler has it (only orc_run_pull's loops use it)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".{os.getpid()}.tmp"
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC]
        try:
            subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _OUT)
    return _OUT


def load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ct.CDLL(build())
            lib.orc_philox4x32_10.argtypes = [ct.c_void_p, ct.c_void_p, ct.c_void_p]
            lib.orc_philox4x32_10.restype = None
            lib.orc_step.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                     ct.c_uint64, ct.c_int, ct.c_uint64, ct.c_void_p, ct.c_void_p,
                                     ct.c_void_p, ct.POINTER(ct.c_int)]
            lib.orc_step.restype = ct.c_int
            lib.orc_run.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                    ct.c_uint64, ct.c_int64, ct.c_int, ct.c_uint64, ct.c_void_p,
                                    ct.POINTER(ct.c_int64)]
            lib.orc_run.restype = ct.c_int
            lib.orc_is_halted.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p]
            lib.orc_is_halted.restype = ct.c_int
            lib.orc_count_choices.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p, ct.c_void_p]
            lib.orc_count_choices.restype = None
            lib.orc_threads.argtypes = []
            lib.orc_threads.restype = ct.c_int
            lib.orc_in_lists.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p]
            lib.orc_in_lists.restype = ct.c_int
            lib.orc_run_pull.argtypes = [ct.POINTER(_Sys), ct.c_void_p, ct.c_void_p, ct.c_void_p, ct.c_void_p,
                                         ct.c_void_p, ct.c_uint64, ct.c_int64, ct.c_int, ct.c_uint64,
                                         ct.c_void_p, ct.POINTER(ct.c_int64)]
            lib.orc_run_pull.restype = ct.c_int
            lib.orc_range_select.argtypes = [ct.POINTER(_Sys), ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p,
                                             ct.c_void_p, ct.c_uint64, ct.c_int, ct.c_uint64, ct.c_void_p,
                                             ct.c_void_p, ct.c_void_p, ct.POINTER(ct.c_int)]
            lib.orc_range_select.restype = ct.c_int
            lib.orc_range_receive.argtypes = [ct.POINTER(_Sys), ct.c_int32, ct.c_int32, ct.c_void_p, ct.c_void_p,
                                              ct.c_void_p, ct.c_void_p, ct.c_void_p]
            lib.orc_range_receive.restype = ct.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _Bound:
    """Keeps the numpy arrays of a system alive while C holds pointers to them."""

    def __init__(self, desc):
        a = desc.arrays()
        self.arrays = a
        self.s = _Sys(desc.q, _ptr(a["rule_offsets"]), _ptr(a["rule_k"]), _ptr(a["rule_j"]),
                      _ptr(a["rule_c"]), _ptr(a["rule_p"]), _ptr(a["rule_d"]),
                      _ptr(a["syn_offsets"]), _ptr(a["syn_targets"]),
                      *(None if a.get(n) is None else _ptr(a[n]) for n in ("rule_term_offsets", "term_k", "term_j")))


def _check(rc: int):
    if rc == _OVERFLOW:
        raise OracleOverflow("spike count left the int32 range")
    if rc != _OK:
        raise OracleError(f"oracle error {rc}")


def initial_state(desc):
    """(C_0, D_0 = 0, P_0 = -1): Alg. 1 initialises D with zeroes."""
    return (np.array(desc.init_spikes, np.int32, copy=True),
            np.zeros(desc.q, np.int32), np.full(desc.q, -1, np.int32))


def philox4x32_10(ctr, key) -> np.ndarray:
    lib = load()
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib.orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def is_halted(desc, C, P) -> bool:
    b = _Bound(desc)
    return bool(load().orc_is_halted(ct.byref(b.s), _ptr(C), _ptr(P)))


def step(desc, state, k: int, mode: int = FIRST, seed: int = 0, forced=None, bound=None):
    """One step in place on state=(C, D, P).  Returns (S, E, halted)."""
    lib = load()
    b = bound or _Bound(desc)
    C, D, P = state
    S = np.empty(desc.q, np.int32)
    E = np.empty(desc.q, np.int32)
    h = ct.c_int(0)
    f = None
    if forced is not None:
        f = np.ascontiguousarray(forced, np.int32)
    rc = lib.orc_step(ct.byref(b.s), _ptr(C), _ptr(D), _ptr(P), ct.c_uint64(k), mode,
                      ct.c_uint64(seed), _ptr(f) if f is not None else None, _ptr(S), _ptr(E),
                      ct.byref(h))
    _check(rc)
    return S, E, bool(h.value)


def run(desc, state, nsteps: int, mode: int = FIRST, seed: int = 0, step0: int = 0):
    """Up to nsteps steps in place.  Returns (executed, S of the last executed step)."""
    lib = load()
    b = _Bound(desc)
    C, D, P = state
    S = np.full(desc.q, -1, np.int32)
    ex = ct.c_int64(0)
    rc = lib.orc_run(ct.byref(b.s), _ptr(C), _ptr(D), _ptr(P), ct.c_uint64(step0),
                     ct.c_int64(nsteps), mode, ct.c_uint64(seed), _ptr(S), ct.byref(ex))
    _check(rc)
    return int(ex.value), S


def run_trace(desc, nsteps: int, mode: int = FIRST, seed: int = 0):
    """Every configuration from C_0 on: list of (C, D, P, S) after each executed step."""
    b = _Bound(desc)
    state = initial_state(desc)
    out = []
    for k in range(nsteps):
        S, E, halted = step(desc, state, k, mode, seed, bound=b)
        if halted:
            break
        out.append(tuple(x.copy() for x in state) + (S,))
    return out


def threads() -> int:
    """Threads orc_run_pull uses (1 without OpenMP)."""
    return int(load().orc_threads())


class PullRunner:
    """The same definition with phase 2 as a pull over in-lists, each phase
    split across threads (orc_run_pull).  Builds the in-lists once."""

    def __init__(self, desc):
        self.desc = desc
        self.b = _Bound(desc)
        self.in_off = np.zeros(desc.q + 1, np.int64)
        self.in_src = np.zeros(max(1, int(desc.num_syn)), np.int32)
        _check(load().orc_in_lists(ct.byref(self.b.s), _ptr(self.in_off), _ptr(self.in_src)))

    def run(self, state, nsteps: int, mode: int = FIRST, seed: int = 0, step0: int = 0):
        """Up to nsteps steps in place.  Returns (executed, S of the last executed step)."""
        if mode not in (FIRST, PHILOX):
            raise ValueError("orc_run_pull takes FIRST or PHILOX")
        C, D, P = state
        S = np.full(self.desc.q, -1, np.int32)
        ex = ct.c_int64(0)
        rc = load().orc_run_pull(ct.byref(self.b.s), _ptr(self.in_off), _ptr(self.in_src), _ptr(C), _ptr(D),
                                 _ptr(P), ct.c_uint64(step0), ct.c_int64(nsteps), mode, ct.c_uint64(seed),
                                 _ptr(S), ct.byref(ex))
        _check(rc)
        return int(ex.value), S


def count_choices(desc, state) -> np.ndarray:
    """Per neuron, how many rules it may choose at the next step (|A_i|, 0 while pending)."""
    b = _Bound(desc)
    C, D, P = state
    out = np.zeros(desc.q, np.int32)
    load().orc_count_choices(ct.byref(b.s), _ptr(C), _ptr(P), _ptr(out))
    return out


class RangeShard:
    """The definition's step split at its exchange point for the neurons
    lo..hi-1 (orc_range_select / orc_range_receive): a shard of a system
    partitioned by neuron range, holding the whole state arrays but changing
    only its own neurons.  E is the whole emission vector (int32, q); the
    caller fills the other shards' entries between the two phases."""

    def __init__(self, desc, lo: int, hi: int, state=None):
        self.desc = desc
        self.b = _Bound(desc)
        self.lo, self.hi = int(lo), int(hi)
        self.C, self.D, self.P = (x.copy() for x in (state or initial_state(desc)))
        self.S = np.full(desc.q, -1, np.int32)
        self.E = np.zeros(desc.q, np.int32)
        self.recv = np.ones(desc.q, np.int8)

    def select(self, k: int, mode: int = FIRST, seed: int = 0) -> bool:
        act = ct.c_int(0)
        _check(load().orc_range_select(ct.byref(self.b.s), self.lo, self.hi, _ptr(self.C), _ptr(self.D),
                                       _ptr(self.P), ct.c_uint64(k), mode, ct.c_uint64(seed), _ptr(self.S),
                                       _ptr(self.E), _ptr(self.recv), ct.byref(act)))
        return bool(act.value)

    def receive(self):
        _check(load().orc_range_receive(ct.byref(self.b.s), self.lo, self.hi, _ptr(self.C), _ptr(self.D),
                                        _ptr(self.P), _ptr(self.E), _ptr(self.recv)))
