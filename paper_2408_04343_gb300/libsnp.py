"""Thin ctypes binding of libsnp (include/snp.h), same names as the C-ABI.

Argument marshalling only: every step of the simulation runs in the CUDA
library.  There is no CPU fallback; if ``_build/libsnp.so`` is missing the
import of a function raises.  Device buffers may be passed as torch CUDA
tensors (their data_ptr is handed over) or as raw integer pointers.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

import numpy as np

from . import build as _build

SNP_OK, SNP_ERR_INVALID, SNP_ERR_OOM, SNP_ERR_CUDA, SNP_ERR_TIMEOUT, SNP_ERR_OVERFLOW, \
    SNP_ERR_BUSY, SNP_ERR_UNSUPPORTED = range(8)
SNP_FORM_OPT, SNP_FORM_ELL, SNP_FORM_DENSE = 0, 1, 2
SNP_PROP_PULL, SNP_PROP_PUSH = 0, 1
SNP_SELECT_FIRST, SNP_SELECT_PHILOX = 0, 1
SNP_ENGINE_AUTO, SNP_ENGINE_LAUNCH, SNP_ENGINE_RESIDENT, SNP_ENGINE_TILED = 0, 1, 2, 3


class SnpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{msg} (status {status})")
        self.status = status


ALLOC_FN = ct.CFUNCTYPE(ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p)
RELEASE_FN = ct.CFUNCTYPE(None, ct.c_void_p, ct.c_void_p, ct.c_size_t, ct.c_void_p)


class snp_allocator(ct.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", ct.c_void_p)]


class snp_options(ct.Structure):
    _fields_ = [("form", ct.c_int32), ("prop", ct.c_int32), ("select", ct.c_int32), ("engine", ct.c_int32),
                ("seed", ct.c_uint64), ("stream", ct.c_void_p), ("alloc", ct.POINTER(snp_allocator)),
                ("threads", ct.c_int32), ("flags", ct.c_int32)]


class snp_desc(ct.Structure):
    _fields_ = [("q", ct.c_int32), ("init_spikes", ct.c_void_p), ("rule_offsets", ct.c_void_p),
                ("rule_k", ct.c_void_p), ("rule_j", ct.c_void_p), ("rule_c", ct.c_void_p),
                ("rule_p", ct.c_void_p), ("rule_d", ct.c_void_p), ("num_syn", ct.c_int64),
                ("syn_offsets", ct.c_void_p), ("syn_targets", ct.c_void_p), ("out_neuron", ct.c_int32),
                ("rule_term_offsets", ct.c_void_p), ("term_k", ct.c_void_p), ("term_j", ct.c_void_p)]


class snp_info(ct.Structure):
    _fields_ = [("q", ct.c_int32), ("form", ct.c_int32), ("prop", ct.c_int32), ("select", ct.c_int32),
                ("engine", ct.c_int32), ("m", ct.c_int64), ("num_syn", ct.c_int64),
                ("in_entries", ct.c_int64), ("out_entries", ct.c_int64), ("rule_words", ct.c_int64),
                ("device_bytes", ct.c_int64), ("max_rules", ct.c_int32), ("max_p", ct.c_int32),
                ("compact_rules", ct.c_int32), ("e_bits", ct.c_int32), ("step", ct.c_uint64),
                ("compiled_rules", ct.c_int32), ("tiled_partitions", ct.c_int32), ("tiled_ctas", ct.c_int32),
                ("tiled_layout", ct.c_int32), ("tiled_acc_bits", ct.c_int32), ("tiled_smem_bytes", ct.c_int64)]


class snp_device_system(ct.Structure):
    _fields_ = [("q", ct.c_int32), ("m", ct.c_int64), ("num_in", ct.c_int64),
                ("rule_offsets", ct.c_void_p), ("rule_k", ct.c_void_p), ("rule_j", ct.c_void_p),
                ("rule_c", ct.c_void_p), ("rule_p", ct.c_void_p), ("rule_d", ct.c_void_p),
                ("in_offsets", ct.c_void_p), ("in_sources", ct.c_void_p),
                ("C", ct.c_void_p), ("D", ct.c_void_p), ("P", ct.c_void_p), ("S", ct.c_void_p)]


class snp_batch_info(ct.Structure):
    _fields_ = [("budget_bytes", ct.c_uint64), ("resident_bytes", ct.c_uint64),
                ("peak_resident_bytes", ct.c_uint64), ("rounds", ct.c_int64), ("admitted", ct.c_int64),
                ("finished", ct.c_int64), ("waiting", ct.c_int64), ("running", ct.c_int64),
                ("admit_seconds", ct.c_double), ("launch_seconds", ct.c_double),
                ("resident_seconds", ct.c_double), ("resident_device_seconds", ct.c_double),
                ("large_tail_seconds", ct.c_double), ("idle_seconds", ct.c_double),
                ("round_seconds", ct.c_double)]


SNP_NOALLOC_MAX_Q = 262144
SNP_FLAG_DEFER_UPLOAD = 1

_P = ct.c_void_p
_SIGS = {
    "snp_create": (ct.c_int, [ct.POINTER(snp_desc), ct.POINTER(snp_options), ct.POINTER(ct.c_void_p)]),
    "snp_destroy": (ct.c_int, [_P]),
    "snp_step": (ct.c_int, [_P, ct.c_int64, ct.POINTER(ct.c_int64)]),
    "snp_get_config": (ct.c_int, [_P, _P, ct.c_int64]),
    "snp_get_spiking": (ct.c_int, [_P, _P, ct.c_int64]),
    "snp_get_status": (ct.c_int, [_P, _P, ct.c_int64]),
    "snp_get_pending": (ct.c_int, [_P, _P, ct.c_int64]),
    "snp_get_state": (ct.c_int, [_P, _P, _P, _P, ct.c_int64, ct.POINTER(ct.c_uint64)]),
    "snp_set_state": (ct.c_int, [_P, _P, _P, _P, ct.c_int64, ct.c_uint64]),
    "snp_get_info": (ct.c_int, [_P, ct.POINTER(snp_info)]),
    "snp_batch_create": (ct.c_int, [ct.POINTER(snp_options), ct.c_size_t, ct.POINTER(ct.c_void_p)]),
    "snp_batch_destroy": (ct.c_int, [_P]),
    "snp_batch_submit": (ct.c_int, [_P, _P, _P, ct.c_int32, ct.POINTER(ct.c_int64)]),
    "snp_batch_poll": (ct.c_int, [_P, ct.c_int64, ct.POINTER(ct.c_int)]),
    "snp_batch_wait": (ct.c_int, [_P, ct.c_int64]),
    "snp_batch_steps_done": (ct.c_int, [_P, ct.c_int64, ct.c_int32, ct.POINTER(ct.c_int64)]),
    "snp_batch_get_info": (ct.c_int, [_P, ct.POINTER(snp_batch_info)]),
    "snp_export_dense": (ct.c_int, [ct.POINTER(snp_desc), _P, ct.c_int64]),
    "snp_export_ell": (ct.c_int, [ct.POINTER(snp_desc), _P, _P, ct.c_int64, ct.POINTER(ct.c_int64)]),
    "snp_export_compressed": (ct.c_int, [ct.POINTER(snp_desc), _P, ct.c_int64, ct.POINTER(ct.c_int64)]),
    "snp_paper_format_elements": (ct.c_int64, [ct.c_int32, ct.c_int64, ct.c_int64, ct.c_int64]),
    "snp_step_noalloc": (ct.c_int, [ct.POINTER(snp_device_system), ct.c_int32, ct.c_uint64, ct.c_uint64,
                                     ct.c_int64, _P, ct.POINTER(ct.c_int64)]),
    "snp_check_bounded_wait": (ct.c_int, [ct.c_int32]),
    "snp_count_choices": (ct.c_int, [_P, ct.c_void_p, ct.c_int64]),
    "snp_set_choices": (ct.c_int, [_P, ct.c_void_p, ct.c_int64]),
    "snp_branch_step": (ct.c_int, [_P, ct.c_int32] + [ct.c_void_p] * 10),
    "snp_shard_create": (ct.c_int, [ct.POINTER(snp_desc), ct.c_int32, ct.c_int32, ct.POINTER(snp_options), _P,
                                     ct.POINTER(ct.c_void_p)]),
    "snp_shard_destroy": (ct.c_int, [_P]),
    "snp_shard_emissions": (ct.c_int, [_P, ct.POINTER(ct.c_void_p)]),
    "snp_shard_select": (ct.c_int, [_P, ct.c_uint64, ct.POINTER(ct.c_int32)]),
    "snp_shard_gather": (ct.c_int, [_P]),
    "snp_shard_get_state": (ct.c_int, [_P, _P, _P, _P, _P, ct.c_int64]),
    "snp_strerror": (ct.c_char_p, [ct.c_int]),
    "snp_last_error": (ct.c_char_p, []),
}

_lib = None
_lock = threading.Lock()


def library_path() -> str:
    """The library this process loads: the bounds-checked debug build when
    SNP_CHECK_BOUNDS=1 is set, else the release build."""
    return _build.CHECK_LIB if os.environ.get("SNP_CHECK_BOUNDS") == "1" else _build.LIB


def load():
    """Loads libsnp.so.  Raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libsnp is not built ({path} missing); run "
                                   "paper_2408_04343_gb300.build.build() first")
            lib = ct.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(rc: int):
    if rc != SNP_OK:
        lib = load()
        raise SnpError(rc, lib.snp_last_error().decode(errors="replace") or lib.snp_strerror(rc).decode())


def _ptr(x) -> int:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _stream_handle(stream) -> int:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class _DescHolder:
    """Builds an snp_desc over numpy arrays and keeps them alive."""

    def __init__(self, desc):
        a = desc.arrays()
        self.a = a
        self.d = snp_desc(desc.q, _ptr(a["init_spikes"]), _ptr(a["rule_offsets"]), _ptr(a["rule_k"]),
                          _ptr(a["rule_j"]), _ptr(a["rule_c"]), _ptr(a["rule_p"]), _ptr(a["rule_d"]),
                          int(a["syn_offsets"][-1]), _ptr(a["syn_offsets"]), _ptr(a["syn_targets"]),
                          int(getattr(desc, "out_neuron", 0)), _ptr(a.get("rule_term_offsets")),
                          _ptr(a.get("term_k")), _ptr(a.get("term_j")))


def make_options(form=SNP_FORM_OPT, prop=SNP_PROP_PULL, select=SNP_SELECT_FIRST, engine=SNP_ENGINE_AUTO,
                 seed=0, stream=None, threads=0, allocator=None, flags=0) -> snp_options:
    o = snp_options(form, prop, select, engine, seed & (2**64 - 1), _stream_handle(stream), None, threads, flags)
    if allocator is not None:
        o.alloc = ct.pointer(allocator)
    return o


class System:
    """One SNP system on the GPU (snp_create .. snp_destroy)."""

    def __init__(self, desc, *, form=SNP_FORM_OPT, prop=SNP_PROP_PULL, select=SNP_SELECT_FIRST,
                 engine=SNP_ENGINE_AUTO, seed=None, stream=None, threads=0, allocator=None, deferred=False):
        lib = load()
        self._lib = lib
        self.q = int(desc.q)
        self.m = int(desc.rule_offsets[-1])
        self.num_syn = int(desc.syn_offsets[-1])
        h = _DescHolder(desc)
        seed = getattr(desc, "seed", 0) if seed is None else seed
        self._alloc = allocator
        opts = make_options(form, prop, select, engine, int(seed), stream, threads, allocator,
                            SNP_FLAG_DEFER_UPLOAD if deferred else 0)
        out = ct.c_void_p()
        check(lib.snp_create(ct.byref(h.d), ct.byref(opts), ct.byref(out)))
        self.handle = out.value

    # -- life cycle
    def close(self):
        if getattr(self, "handle", None):
            check(self._lib.snp_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping
    def step(self, n: int, wait: bool = True):
        """snp_step: returns executed steps when wait, else None (queued)."""
        if wait:
            done = ct.c_int64(0)
            check(self._lib.snp_step(self.handle, int(n), ct.byref(done)))
            return int(done.value)
        check(self._lib.snp_step(self.handle, int(n), None))
        return None

    # -- state
    def _get(self, fn, out=None):
        if out is None:
            out = np.empty(self.q, np.int32)
        n = out.numel() if hasattr(out, "numel") else out.size
        check(fn(self.handle, _ptr(out), int(n)))
        return out

    def config(self, out=None):
        return self._get(self._lib.snp_get_config, out)

    def spiking(self, out=None):
        return self._get(self._lib.snp_get_spiking, out)

    def status(self, out=None):
        return self._get(self._lib.snp_get_status, out)

    def pending(self, out=None):
        return self._get(self._lib.snp_get_pending, out)

    def get_state(self):
        C = np.empty(self.q, np.int32)
        D = np.empty(self.q, np.int32)
        P = np.empty(self.q, np.int32)
        k = ct.c_uint64(0)
        check(self._lib.snp_get_state(self.handle, _ptr(C), _ptr(D), _ptr(P), self.q, ct.byref(k)))
        return C, D, P, int(k.value)

    def count_choices(self, out=None):
        """snp_count_choices: per neuron, how many rules it may choose next."""
        return self._get(self._lib.snp_count_choices, out)

    def set_choices(self, idx):
        """snp_set_choices: the choice index of every neuron for the first step
        of the next step() call."""
        if not hasattr(idx, "data_ptr"):
            idx = np.ascontiguousarray(idx, np.int32)
        n = idx.numel() if hasattr(idx, "numel") else idx.size
        check(self._lib.snp_set_choices(self.handle, _ptr(idx), int(n)))

    def branch_step(self, C, D, P, choices):
        """snp_branch_step over [nb][q] numpy arrays: one forced step of each
        configuration.  Returns (C1, D1, P1, executed, bad, counts), counts
        being the choices of each new configuration."""
        C, D, P, ch = (np.ascontiguousarray(x, np.int32) for x in (C, D, P, choices))
        nb = C.shape[0]
        C1, D1, P1, cnt = (np.empty_like(C) for _ in range(4))
        ex = np.empty(nb, np.int32)
        bad = np.empty(nb, np.int32)
        check(self._lib.snp_branch_step(self.handle, nb, _ptr(C), _ptr(D), _ptr(P), _ptr(ch), _ptr(C1), _ptr(D1),
                                        _ptr(P1), _ptr(ex), _ptr(bad), _ptr(cnt)))
        return C1, D1, P1, ex, bad, cnt

    def set_state(self, C, D, P, step: int):
        n = C.numel() if hasattr(C, "numel") else np.asarray(C).size
        if isinstance(C, np.ndarray):
            C, D, P = (np.ascontiguousarray(x, np.int32) for x in (C, D, P))
        check(self._lib.snp_set_state(self.handle, _ptr(C), _ptr(D), _ptr(P), int(n), int(step)))

    def info(self) -> snp_info:
        inf = snp_info()
        check(self._lib.snp_get_info(self.handle, ct.byref(inf)))
        return inf


class Batch:
    """snp_batch_*: many systems advanced by persistent launches."""

    def __init__(self, *, mem_budget: int = 0, stream=None, threads=0):
        lib = load()
        self._lib = lib
        opts = make_options(stream=stream, threads=threads)
        out = ct.c_void_p()
        check(lib.snp_batch_create(ct.byref(opts), int(mem_budget), ct.byref(out)))
        self.handle = out.value
        self._keep = {}

    def submit(self, systems, steps) -> int:
        handles = (ct.c_void_p * len(systems))(*[s.handle for s in systems])
        st = np.ascontiguousarray(np.broadcast_to(np.asarray(steps, np.int64), (len(systems),)))
        t = ct.c_int64(0)
        check(self._lib.snp_batch_submit(self.handle, ct.cast(handles, ct.c_void_p), _ptr(st), len(systems),
                                         ct.byref(t)))
        self._keep[t.value] = (handles, st, len(systems))
        return int(t.value)

    def poll(self, ticket: int) -> bool:
        d = ct.c_int(0)
        check(self._lib.snp_batch_poll(self.handle, int(ticket), ct.byref(d)))
        return bool(d.value)

    def wait(self, ticket: int):
        check(self._lib.snp_batch_wait(self.handle, int(ticket)))
        n = self._keep[ticket][2]
        out = []
        for i in range(n):
            v = ct.c_int64(0)
            check(self._lib.snp_batch_steps_done(self.handle, int(ticket), i, ct.byref(v)))
            out.append(int(v.value))
        return out

    def steps_done(self, ticket: int, index: int) -> int:
        v = ct.c_int64(0)
        check(self._lib.snp_batch_steps_done(self.handle, int(ticket), int(index), ct.byref(v)))
        return int(v.value)

    def info(self) -> snp_batch_info:
        inf = snp_batch_info()
        check(self._lib.snp_batch_get_info(self.handle, ct.byref(inf)))
        return inf

    def close(self):
        if getattr(self, "handle", None):
            check(self._lib.snp_batch_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- paper formats (host only) --------------------------------------------

def export_dense(desc) -> np.ndarray:
    h = _DescHolder(desc)
    m, q = int(desc.rule_offsets[-1]), int(desc.q)
    M = np.zeros((m, q), np.int32)
    check(load().snp_export_dense(ct.byref(h.d), _ptr(M), M.size))
    return M


def export_ell(desc):
    h = _DescHolder(desc)
    rows = ct.c_int64(0)
    lib = load()
    check(lib.snp_export_ell(ct.byref(h.d), None, None, 0, ct.byref(rows)))
    m = int(desc.rule_offsets[-1])
    vals = np.zeros((rows.value, m), np.int32)
    nrn = np.zeros((rows.value, m), np.int32)
    check(lib.snp_export_ell(ct.byref(h.d), _ptr(vals), _ptr(nrn), vals.size, ct.byref(rows)))
    return vals, nrn


def export_compressed(desc) -> np.ndarray:
    h = _DescHolder(desc)
    rows = ct.c_int64(0)
    lib = load()
    check(lib.snp_export_compressed(ct.byref(h.d), None, 0, ct.byref(rows)))
    sy = np.zeros((rows.value, int(desc.q)), np.int32)
    check(lib.snp_export_compressed(ct.byref(h.d), _ptr(sy), sy.size, ct.byref(rows)))
    return sy


def paper_format_elements(form: int, q: int, m: int, z: int) -> int:
    return int(load().snp_paper_format_elements(form, q, m, z))


# ---- stepping without allocation -------------------------------------------

def snp_step_noalloc(q, m, rule_offsets, rule_k, rule_j, rule_c, rule_p, rule_d, in_offsets, in_sources,
                     C, D, P, S, *, num_in=None, select=SNP_SELECT_FIRST, seed=0, step=0, n=1, stream=None,
                     wait=True):
    """snp_step_noalloc over caller-owned device buffers (torch CUDA tensors
    or raw pointers, int32).  For callers that cannot allocate device memory:
    the library uses its fixed static scratch (q <= SNP_NOALLOC_MAX_Q).
    num_in is the length of in_sources; it is taken from a tensor and must be
    given when in_sources is a raw pointer.  Returns the executed step count
    when wait, else None."""
    if num_in is None:
        if not hasattr(in_sources, "numel"):
            raise TypeError("num_in must be given when in_sources is not a tensor")
        num_in = in_sources.numel()
    d = snp_device_system(int(q), int(m), int(num_in), _ptr(rule_offsets), _ptr(rule_k), _ptr(rule_j),
                          _ptr(rule_c), _ptr(rule_p), _ptr(rule_d), _ptr(in_offsets), _ptr(in_sources),
                          _ptr(C), _ptr(D), _ptr(P), _ptr(S))
    done = ct.c_int64(0)
    check(load().snp_step_noalloc(ct.byref(d), int(select), int(seed) & (2**64 - 1), int(step), int(n),
                                  _stream_handle(stream), ct.byref(done) if wait else None))
    return int(done.value) if wait else None


# ---- the neuron-sharded step ------------------------------------------------

class Shard:
    """snp_shard_*: neurons lo..hi-1 of one system (see shard.py for the step
    protocol).  E: the emission vector, a device tensor (int16/uint16, at
    least q + 1 entries) or raw device pointer the caller owns, or None."""

    def __init__(self, desc, lo, hi, *, select=SNP_SELECT_FIRST, seed=None, stream=None, E=None):
        lib = load()
        self._lib = lib
        self.lo, self.hi, self.q = int(lo), int(hi), int(desc.q)
        h = _DescHolder(desc)
        seed = getattr(desc, "seed", 0) if seed is None else seed
        opts = make_options(select=select, seed=int(seed), stream=stream)
        out = ct.c_void_p()
        check(lib.snp_shard_create(ct.byref(h.d), self.lo, self.hi, ct.byref(opts), _ptr(E), ct.byref(out)))
        self.handle = out.value

    def emissions_ptr(self) -> int:
        p = ct.c_void_p()
        check(self._lib.snp_shard_emissions(self.handle, ct.byref(p)))
        return int(p.value)

    def select(self, k: int) -> bool:
        a = ct.c_int32(0)
        check(self._lib.snp_shard_select(self.handle, int(k), ct.byref(a)))
        return bool(a.value)

    def receive(self):
        check(self._lib.snp_shard_gather(self.handle))

    def get_state(self):
        n = self.hi - self.lo
        C, D, P, S = (np.empty(n, np.int32) for _ in range(4))
        check(self._lib.snp_shard_get_state(self.handle, _ptr(C), _ptr(D), _ptr(P), _ptr(S), n))
        return C, D, P, S

    def close(self):
        if getattr(self, "handle", None):
            check(self._lib.snp_shard_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
