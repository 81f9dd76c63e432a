"""Bench: synaptic updates/s of the SNP-with-delays step on one GB300.

Workload (the headline): a random SNP system with delays of 1,048,576 neurons,
out-degree uniform in 8..24 (mean 16, |syn| = 16.8M), 3 firing rules
a^k(a^j)*/a^c -> a^p;d plus one forgetting rule per neuron, d in [0,5],
initial spikes uniform in 0..20, Philox-keyed nondeterministic selection.

One bench step = one snp_step call advancing one system by `--call-steps`
SNP steps (default 48) on the tiled pull engine (emissions in shared
memory, one fused launch per SNP step).  To keep the inputs of
consecutive timed iterations out of L2 (129 MB), R replicas of the system
(same graph, different Philox seeds; 4 x ~126 MB on the device) are stepped
round-robin, so a system's data has been evicted by the time it is stepped
again.  value = |syn| x executed SNP steps / device time of the K timed
steps (CUDA events on the systems' stream, max over ranks, summed work).

--impl reference times the CPU oracle (test infrastructure, plain C) in its
parallel pull form, one OpenMP thread per host core, on the same workload:
each step is one SNP step of the same system.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np

WORKLOAD = ("1,048,576-neuron SNP system with delays: out-degree U{8..24}, 3 firing + 1 forgetting rule "
            "per neuron, d in [0,5], spikes U[0,20], Philox selection")
PEAK_FALLBACK_GBS = 6800.0
L2_BYTES = 129 * 2**20


def algorithmic_bytes_per_step(desc) -> int:
    """Bytes one SNP step must move at stored width, read or written once:
    in-list 4/in-edge; per neuron: E read 4, C read+write 8, status
    read+write 8, rule offset 4, rules 4 each (one word per rule), E write 4,
    S write 4."""
    R = np.diff(desc.rule_offsets)
    return int(4 * desc.num_syn + desc.q * 32 + 4 * int(R.sum()))


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    except Exception:
        return PEAK_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(ws, x: float) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def oracle_cpu_baseline(desc, mode, seed, budget_s=12.0):
    """The oracle as it stands on a bounded sample (the first steps of the same
    system): its parallel pull form on every host core (the figure reported),
    and its neuron-by-neuron form on one thread beside it."""
    import oracle
    oracle.build()
    pr = oracle.PullRunner(desc)                       # in-lists: built once, not timed
    st = oracle.initial_state(desc)
    t0 = time.perf_counter()
    ex, _ = pr.run(st, 1, mode, seed)
    one = time.perf_counter() - t0
    n = max(1, min(2000, int(budget_s / max(one, 1e-6)) - 1))
    t0 = time.perf_counter()
    ex2, _ = pr.run(st, n, mode, seed, step0=ex)
    dt = time.perf_counter() - t0
    threads = oracle.threads()
    st1 = oracle.initial_state(desc)
    t0 = time.perf_counter()
    e1, _ = oracle.run(desc, st1, 1, mode, seed)
    one1 = time.perf_counter() - t0
    n1 = max(1, min(400, int(budget_s / max(one1, 1e-6)) - 1))
    t0 = time.perf_counter()
    e2, _ = oracle.run(desc, st1, n1, mode, seed, step0=e1)
    dt1 = time.perf_counter() - t0
    return {"value": desc.num_syn * ex2 / dt, "unit": "synaptic updates/s", "cores": threads, "kind": "oracle",
            "sample": f"steps {ex}..{ex + ex2 - 1} of the 1,048,576-neuron workload, {dt:.1f} s, "
                      f"the oracle's parallel pull form on {threads} threads",
            "single_thread_value": desc.num_syn * e2 / dt1,
            "single_thread_sample": f"steps {e1}..{e1 + e2 - 1}, {dt1:.1f} s, neuron-by-neuron form, 1 thread"}


def run_reference(args, ws, rank):
    """The oracle arm: each bench step is one SNP step of the workload, run by
    the oracle's parallel pull form on the host cores."""
    if rank != 0:
        return
    import oracle
    from paper_2408_04343_gb300 import synth
    oracle.build()
    desc, _, mode = synth.large_1m()
    pr = oracle.PullRunner(desc)
    st = oracle.initial_state(desc)
    k = 0
    for _ in range(args.warmup):
        ex, _ = pr.run(st, 1, mode, desc.seed, step0=k)
        k += ex
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        ex, _ = pr.run(st, 1, mode, desc.seed, step0=k)
        k += ex
        done += ex
    dt = time.perf_counter() - t0
    v = desc.num_syn * done / dt
    threads = oracle.threads()
    line = {"impl": "reference", "metric": "synaptic updates/s", "value": v, "unit": "synaptic updates/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / max(1, args.steps) * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "engine": f"CPU oracle (parallel pull form, {threads} threads), "
                                                       "one SNP step per bench step"},
            "cpu_baseline": {"value": v, "unit": "synaptic updates/s", "cores": threads, "kind": "oracle",
                             "sample": f"{done} SNP steps of the 1,048,576-neuron workload"},
            "e2e": {"value": v, "unit": "synaptic updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--call-steps", type=int, default=48)
    ap.add_argument("--replicas", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--engine", default="tiled", choices=["tiled", "launch"],
                    help="tiled: emissions in shared memory (default); launch: emissions gathered from L2")
    ap.add_argument("--workload", default="large", choices=["large", "batch", "serve", "skewed", "families", "tree", "engines", "shards"],
                    help="large: the 1M-neuron headline (default); batch: 8,192 systems in one persistent "
                         "launch vs the plain per-system loop; serve: Poisson request loop; skewed: the "
                         "2M-neuron power-law system and its 16,384-neuron dense copy")
    ap.add_argument("--batch-count", type=int, default=8192)
    ap.add_argument("--skewed-engines", default="all",
                    help="skewed workload: comma list of auto,tiled,l2_gather,push,ell_pull,ell_push,dense")
    ap.add_argument("--rates", default="10,30,100,300,1000,3000,10000")
    ap.add_argument("--requests", type=int, default=1000)
    args = ap.parse_args()
    ws, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        barrier(ws)
        return
    if args.workload != "large":
        import bench_workloads
        bench_workloads.run(args, ws, rank, local)
        barrier(ws)
        return

    import torch
    from paper_2408_04343_gb300 import build as B, libsnp, synth
    if rank == 0:
        B.build()
    barrier(ws)
    torch.cuda.set_device(local)
    desc, _, mode = synth.large_1m()
    stream = torch.cuda.Stream()
    T = args.call_steps
    engine = {"tiled": libsnp.SNP_ENGINE_TILED, "launch": libsnp.SNP_ENGINE_LAUNCH}[args.engine]
    t_pack = time.perf_counter()  # load + pack + upload, outside the timed steps
    systems = [libsnp.System(desc, select=libsnp.SNP_SELECT_PHILOX, seed=desc.seed + 7919 * r + 104729 * rank,
                             engine=engine, stream=stream) for r in range(args.replicas)]
    stream.synchronize()
    t_pack = (time.perf_counter() - t_pack) / max(1, args.replicas)
    foot = sum(s.info().device_bytes for s in systems)
    inf0 = systems[0].info()
    shape = ({"clusters": inf0.tiled_ctas // max(1, inf0.tiled_partitions),
              "ctas_per_cluster": inf0.tiled_partitions, "threads_per_cta": 1024,
              "entry_layout": ["target words", "paired target words", "run-length"][inf0.tiled_layout],
              "accumulator_bits": inf0.tiled_acc_bits, "smem_bytes_per_cta": inf0.tiled_smem_bytes,
              "emission_bits": inf0.e_bits, "entry_bytes": inf0.in_entries * 4}
             if inf0.engine == libsnp.SNP_ENGINE_TILED else None)
    for i in range(args.warmup):
        systems[i % len(systems)].step(T, wait=False)
    stream.synchronize()
    k0 = [s.get_state()[3] for s in systems]

    clocks = ClockSampler(local)
    if rank == 0:
        clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(stream)
    for i in range(args.steps):
        systems[i % len(systems)].step(T, wait=False)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clk = clocks.stop() if rank == 0 else None
    dev_s = e0.elapsed_time(e1) / 1e3
    executed = sum(s.get_state()[3] - k for s, k in zip(systems, k0))
    t_max = max_over_ranks(ws, dev_s)
    work = sum_over_ranks(ws, float(executed) * desc.num_syn)
    value = work / t_max
    # launches of this library per call on this workload: begin, select,
    # T-1 fused steps (plus one advance per captured chunk of 48), gather,
    # finish -- the tiled engine's one-launch step (clusters of P <= 8 CTAs)
    per_call = 4 + (T - 1) + (T - 1) // 48
    launches = per_call * args.steps

    # end to end through the C-ABI with host buffers: every step uploads its
    # input state from pinned host memory and reads the configuration back
    q = desc.q
    hC = torch.empty(q, dtype=torch.int32).pin_memory()
    hD = torch.empty(q, dtype=torch.int32).pin_memory()
    hP = torch.empty(q, dtype=torch.int32).pin_memory()
    hOut = torch.empty(q, dtype=torch.int32).pin_memory()
    s0 = systems[0]
    C, D, P, k = s0.get_state()
    hC.numpy()[:] = C
    hD.numpy()[:] = D
    hP.numpy()[:] = P
    e2e_steps = max(3, min(args.steps, 20))
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_exec = 0
    for i in range(e2e_steps):
        s0.set_state(hC, hD, hP, k)
        e2e_exec += s0.step(T)
        s0.config(hOut)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(ws, time.perf_counter() - t0)
    e2e_value = sum_over_ranks(ws, float(e2e_exec) * desc.num_syn) / e2e_s

    peak, peak_kind = measured_peak()
    alg = algorithmic_bytes_per_step(desc)
    achieved = alg * executed / dev_s / 1e9
    traffic = None
    prof = os.path.join(ROOT, "profiles", f"{args.engine}_1m_traffic.txt")
    if os.path.exists(prof):
        try:
            with open(prof) as f:
                pj = json.load(f)
            from paper_2408_04343_gb300 import build as B2
            if pj.get("kernel_sources_hash") == B2.engine_sources_hash(args.engine):
                traffic = pj.get("dram_bytes_per_launch")
        except Exception:
            traffic = None

    if rank == 0:
        line = {
            "metric": "synaptic updates/s", "value": value, "unit": "synaptic updates/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "engine": {"tiled": "tiled pull (emissions bit-packed in shared memory): one clustered launch per SNP step, programmatic dependent launches replayed from CUDA graphs",
                                                     "launch": "grid-wide pull, emissions gathered from L2, one fused launch per SNP step"}[args.engine],
                       "snp_steps_per_bench_step": T, "replicas_round_robin": len(systems),
                       "l2": f"inputs larger than L2: {len(systems)} replicas, {foot / 1e6:.0f} MB on the device, "
                             f"stepped round-robin", "parallelism": f"replicas x{ws}",
                       "q": desc.q, "num_syn": desc.num_syn, "snp_steps_timed": int(executed),
                       "snp_steps_per_s": work / desc.num_syn / t_max if t_max > 0 else None,
                       "create_seconds_per_system": round(t_pack, 3), "launch_shape": shape},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                         "kernel": {"tiled": "k_tiled_step (one launch per SNP step: gather, then select in thread-block clusters; achieved = a step's algorithmic bytes / its live device time)",
                                    "launch": "k_step_pull (fused gather + select, one launch per SNP step)"}[args.engine],
                         "algorithmic_bytes_per_snp_step": alg},
            "e2e": {"value": e2e_value, "unit": "synaptic updates/s", "h2d_bytes_per_step": 3 * 4 * q,
                    "d2h_bytes_per_step": 4 * q,
                    "note": "per bench step: snp_set_state from pinned host C/D/P, snp_step, snp_get_config to pinned host"},
            "gpu_launches": launches,
        }
        if clk is not None:
            line["clocks"] = clk
        if ws == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_cpu_baseline(desc, mode, desc.seed)
        print(json.dumps(line), flush=True)
    for s in systems:
        s.close()
    barrier(ws)


if __name__ == "__main__":
    main()
