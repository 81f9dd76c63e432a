"""Failure paths of the library, made on the host or with a wait that nothing
completes -- never with a GPU fault.

(1) A caller-supplied allocator is used for every device allocation, and an
allocator that returns NULL surfaces as SNP_ERR_OOM; (2) a bounded device
wait that runs out reports SNP_ERR_TIMEOUT and leaves the context usable.
"""
import ctypes as ct

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


class TorchAllocator:
    """snp_allocator callbacks over torch's caching allocator, with counters
    and an optional failure after `fail_after` successful allocations."""

    def __init__(self, fail_after=None):
        self.fail_after = fail_after
        self.allocs = 0
        self.releases = 0
        self.live = {}

        def alloc(ctx, nbytes, stream):
            if self.fail_after is not None and self.allocs >= self.fail_after:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), stream=torch.cuda.current_stream())
            self.allocs += 1
            self.live[p] = nbytes
            return p

        def release(ctx, ptr, nbytes, stream):
            self.releases += 1
            self.live.pop(ptr, None)
            torch.cuda.caching_allocator_delete(ptr)

        self._alloc = libsnp.ALLOC_FN(alloc)
        self._release = libsnp.RELEASE_FN(release)
        self.struct = libsnp.snp_allocator(self._alloc, self._release, None)


@pytest.mark.parametrize("engine", ["launch", "tiled"])
def test_allocator_callbacks_hold_every_device_buffer(engine):
    d = synth.random_system(5000, 41, outdeg=(4, 16), rules=(3, 4), d_range=(0, 5), spikes=(0, 20))
    a = TorchAllocator()
    eng = {"launch": libsnp.SNP_ENGINE_LAUNCH, "tiled": libsnp.SNP_ENGINE_TILED}[engine]
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, engine=eng, seed=9, allocator=a.struct)
    done = gs.step(30)
    C, D, P, k = gs.get_state()
    st = oracle.initial_state(d)
    ex, _ = oracle.run(d, st, 30, oracle.PHILOX, 9)
    assert done == ex and k == ex
    assert (C == st[0]).all() and (D == st[1]).all() and (P == st[2]).all()
    assert a.allocs >= 1 and a.live
    assert gs.info().device_bytes <= sum(a.live.values())
    gs.close()
    assert a.releases == a.allocs and not a.live


def test_allocator_returning_null_is_out_of_memory():
    d = synth.random_system(3000, 42, outdeg=(4, 16), rules=(3, 3), d_range=(0, 3), spikes=(0, 10))
    a = TorchAllocator(fail_after=0)
    with pytest.raises(libsnp.SnpError) as ei:
        gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST, allocator=a.struct)
        gs.step(5)
    assert ei.value.status == libsnp.SNP_ERR_OOM
    assert a.allocs == 0 and not a.live
    # nothing leaked and the library still works without the failing allocator
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST)
    assert gs.step(5) >= 0
    gs.close()


def test_bounded_wait_that_runs_out_reports_timeout():
    lib = libsnp.load()
    assert lib.snp_check_bounded_wait(0) == libsnp.SNP_ERR_INVALID
    for polls in (1, 64, 2000):
        assert lib.snp_check_bounded_wait(polls) == libsnp.SNP_ERR_TIMEOUT
        assert b"gave up" in lib.snp_last_error()
    # the context is still usable: a system steps and matches the oracle
    d, nsteps, mode = synth.small_1k()
    gs = libsnp.System(d, select=libsnp.SNP_SELECT_FIRST, engine=libsnp.SNP_ENGINE_TILED, seed=d.seed)
    done = gs.step(20)
    st = oracle.initial_state(d)
    ex, _ = oracle.run(d, st, 20, mode, d.seed)
    C, _, _, _ = gs.get_state()
    assert done == ex and (C == st[0]).all()
    gs.close()
    torch.cuda.synchronize()
