"""CPU oracle for the SNP transition step -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg
use this package.  The simulator never imports it.
"""
from .oracle import (FIRST, PHILOX, FORCED, OracleError, OracleOverflow, build, load,
                     philox4x32_10, step, run, run_trace, is_halted, initial_state, threads,
                     PullRunner, RangeShard, count_choices)

__all__ = ["FIRST", "PHILOX", "FORCED", "OracleError", "OracleOverflow", "build", "load",
           "philox4x32_10", "step", "run", "run_trace", "is_halted", "initial_state", "threads",
           "PullRunner", "RangeShard", "count_choices"]
