"""Secondary bench workloads (selected with bench.py --workload ...).

batch  -- 8,192 independent systems (q log-uniform in 64..65,536, out-degree
          U{4..16}, 3 rules, d in [0,4], 500 steps each, Philox) advanced by
          the batched form (one persistent launch per round, CTA per system)
          against the plain per-system loop (each system alone on the
          grid-wide engine, one launch per step, one system after another);
          the plain loop is timed on every 16th system and compared bit for
          bit with the batched result.
serve  -- Poisson request loop: each request a system of q log-uniform in
          1e3..1e6 with a log-uniform step count in 10..1e4, out-degree
          U{2..32}, 2-4 rules, d in [0,5]; admitted by a 150 GB device-memory
          budget; p50/p99 latency (arrival to completion) and aggregate
          synaptic updates/s per arrival rate.
skewed -- the 2,097,152-neuron system with truncated Zipf(2.1) out-degree on
          [1, 4096], 256 steps, on the engine AUTO picks (the headline value),
          the tiled, L2-gather and push engines and the ELL form; and its
          16,384-neuron copy on the dense M_Pi.
families -- Sec. 6's families: the sort system on worst-case inputs
          (n, ..., 1) for n up to 2,000 and the subset-sum-shaped stand-in
          (q = sum(v) + 2n + 2, m = sum(v) + 4n + 2, z = n) for n up to
          20,000: per n the device memory of each form against the paper's
          element-count formulas, and the time of a run (sort: to its fixed
          point, checked sorted; subset-sum-shaped: 200 Philox steps).
engines -- the 1,048,576-neuron workload of the headline bench on every
          engine and form (tiled, L2 gather, push, ELL pull, ELL push): one
          system each, 8 untimed steps, then one timed snp_step(192) call;
          the final configurations must agree.
shards -- the 1,048,576-neuron workload split by neuron range into 1, 2
          and 4 shards on one GPU (snp_shard_*, the step protocol of
          paper_2408_04343_gb300/shard.py with the emission slices exchanged
          by device copies): 64 timed steps after 4 untimed; the final
          configuration must equal the unsharded system's.
tree   -- computation-tree exploration of the subset-sum-shaped stand-in
          (n = 14: 2^14 branches when the choice neurons fire): branches per
          second explored breadth first with the batched branch step (one
          launch per level) and with one forced step per branch.
All inputs are seeded synthetic systems (paper_2408_04343_gb300/synth.py).
"""
from __future__ import annotations

import os
import threading
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np


def run(args, ws, rank, local):
    import json
    import torch
    from paper_2408_04343_gb300 import build as B, libsnp, synth
    if rank == 0:
        B.build()
    torch.cuda.set_device(local)
    fn = {"batch": batch, "serve": serve, "skewed": skewed, "families": families, "tree": tree_workload,
          "engines": engines, "shards": shards}[args.workload]
    line = fn(args, libsnp, synth)
    line.update({"n_gpus": ws, "data": "synthetic", "dtype": "int32", "higher_is_better": True})
    if rank == 0:
        print(json.dumps(line), flush=True)


def _threads():
    return max(1, min(16, os.cpu_count() or 1))


def batch(args, libsnp, synth):
    import torch
    descs, nsteps, _ = synth.batch_8k(count=args.batch_count, processes=_threads())
    sel = libsnp.SNP_SELECT_PHILOX
    with ThreadPoolExecutor(_threads()) as ex:
        gs = list(ex.map(lambda d: libsnp.System(d, select=sel, seed=d.seed), descs))
    torch.cuda.synchronize()
    b = libsnp.Batch()
    # warm-up pass: the batch's autotuner tries its candidates on real rounds;
    # then every system is reset to its initial state and the pass is timed
    b.wait(b.submit(gs, [nsteps] * len(gs)))
    for d, g in zip(descs, gs):
        g.set_state(d.init_spikes.astype(np.int32), np.zeros(d.q, np.int32), np.full(d.q, -1, np.int32), 0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = b.submit(gs, [nsteps] * len(gs))
    done = b.wait(t)
    t1 = time.perf_counter()
    work = sum(d.num_syn * n for d, n in zip(descs, done))
    batched = work / (t1 - t0)
    info = b.info()
    sample = list(range(0, len(descs), 16))
    plain = [libsnp.System(descs[i], select=sel, seed=descs[i].seed, engine=libsnp.SNP_ENGINE_LAUNCH)
             for i in sample]
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    pdone = [g.step(nsteps, wait=False) for g in plain]
    torch.cuda.synchronize()
    t3 = time.perf_counter()
    pdone = [g.get_state()[3] for g in plain]
    pwork = sum(descs[i].num_syn * n for i, n in zip(sample, pdone))
    plain_v = pwork / (t3 - t2)
    same = all((plain[j].config() == gs[i].config()).all() and pdone[j] == done[i] for j, i in enumerate(sample))
    return {"metric": "synaptic updates/s", "workload": "batch", "value": batched, "unit": "synaptic updates/s",
            "plain_loop_value": plain_v, "speedup_vs_plain_loop": batched / plain_v,
            "identical_to_plain_loop": bool(same),
            "config": {"systems": len(descs), "neurons": int(sum(d.q for d in descs)),
                       "synapses": int(sum(d.num_syn for d in descs)), "steps_each": nsteps,
                       "rounds": int(info.rounds), "batched_seconds": t1 - t0,
                       "autotune": "a warm-up pass of the same batch first (then every system reset)",
                       "plain_loop_sample": f"every 16th system ({len(sample)}), one after another, "
                                            f"{t3 - t2:.2f} s"}}


def serve(args, libsnp, synth):
    """The served form at each arrival rate, and the plain loop beside it.

    Every request is its own system (synth.serving_requests: q log-uniform in
    1e3..1e6, steps log-uniform in 10..1e4, its own seed); the same requests
    are replayed at every rate, each rate on freshly created (deferred)
    systems submitted at the request's Poisson arrival time to one batch
    under a 150 GB budget.  Latency is arrival to completion (ticket polled
    by the host).  The plain loop steps the same systems one after another,
    each alone on the grid-wide L2-gather engine (one launch per step)."""
    import torch
    rates = [float(x) for x in args.rates.split(",")]
    n = args.requests
    base = synth.serving_requests(1.0, n, seed=5005)       # sizes, steps, seeds (arrivals rescaled per rate)
    descs = synth.serving_systems(base, processes=_threads())
    sel = libsnp.SNP_SELECT_PHILOX
    per_rate = []
    for lam in rates:
        with ThreadPoolExecutor(_threads()) as ex:
            gs = list(ex.map(lambda i: libsnp.System(descs[i], select=sel, seed=base[i].seed, deferred=True),
                             range(n)))
        b = libsnp.Batch(mem_budget=150 << 30)
        arr = np.array([r.arrival_s for r in base]) / lam     # Poisson at rate lam (same order of requests)
        arr -= arr[0]
        tickets = [None] * n
        start = time.perf_counter()

        def submitter():
            for i in range(n):
                dt = start + arr[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[i] = b.submit([gs[i]], [base[i].steps])

        th = threading.Thread(target=submitter)
        th.start()
        lat, work, left = [0.0] * n, 0, set(range(n))
        last = start
        while left:
            for i in list(left):
                if tickets[i] is not None and b.poll(tickets[i]):
                    now = time.perf_counter()
                    lat[i] = now - (start + arr[i])
                    work += descs[i].num_syn * b.steps_done(tickets[i], 0)
                    gs[i].close()
                    left.discard(i)
                    last = now
            time.sleep(0.0005)
        th.join()
        inf = b.info()
        b.close()
        wall = last - start
        per_rate.append({"rate_per_s": lam, "requests": n, "p50_latency_s": float(np.percentile(lat, 50)),
                         "p99_latency_s": float(np.percentile(lat, 99)), "syn_updates_per_s": work / wall,
                         "wall_s": wall, "arrivals_span_s": float(arr[-1]), "rounds": int(inf.rounds),
                         "peak_device_gb": inf.peak_resident_bytes / 1e9,
                         "time_split_s": {"admission_uploads": inf.admit_seconds,
                                          "queue_grid_wide_steps": inf.launch_seconds,
                                          "resident_launches_host": inf.resident_seconds,
                                          "resident_launches_device": inf.resident_device_seconds,
                                          "wait_grid_wide_after_resident": inf.large_tail_seconds,
                                          "idle": inf.idle_seconds, "rounds_total": inf.round_seconds}})
    # the plain loop: one system after another on the grid-wide engine
    plain = [libsnp.System(descs[i], select=sel, seed=base[i].seed, engine=libsnp.SNP_ENGINE_LAUNCH)
             for i in range(n)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, g in enumerate(plain):
        g.step(base[i].steps, wait=False)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    pwork = sum(descs[i].num_syn * plain[i].get_state()[3] for i in range(n))
    for g in plain:
        g.close()
    plain_v = pwork / (t1 - t0)
    best = max(r["syn_updates_per_s"] for r in per_rate)
    return {"metric": "synaptic updates/s", "workload": "serve", "value": best, "unit": "synaptic updates/s",
            "plain_loop_value": plain_v, "served_vs_plain_loop": best / plain_v, "plain_loop_seconds": t1 - t0,
            "per_rate": per_rate,
            "config": {"requests_per_rate": n, "distinct_systems": n,
                       "neurons": int(sum(d.q for d in descs)), "synapses": int(sum(d.num_syn for d in descs)),
                       "q": "log-uniform 1e3..1e6", "steps": "log-uniform 10..1e4", "out_degree": "U{2..32}",
                       "budget_gb": 150}}


def skewed(args, libsnp, synth):
    import torch
    d, nsteps, mode = synth.skewed_2m()
    res = {}
    chosen = None if args.skewed_engines in (None, "all") else set(args.skewed_engines.split(","))
    for name, kw in [("auto", dict(engine=libsnp.SNP_ENGINE_AUTO)),
                     ("tiled", dict(engine=libsnp.SNP_ENGINE_TILED)),
                     ("l2_gather", dict(engine=libsnp.SNP_ENGINE_LAUNCH)),
                     ("push", dict(prop=libsnp.SNP_PROP_PUSH)),
                     ("ell_pull", dict(form=libsnp.SNP_FORM_ELL)),
                     ("ell_push", dict(form=libsnp.SNP_FORM_ELL, prop=libsnp.SNP_PROP_PUSH))]:
        if chosen is not None and name not in chosen:
            continue
        try:
            g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=d.seed, **kw)
        except libsnp.SnpError as e:
            res[name] = {"unavailable": str(e)}
            continue
        g.step(8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = g.step(nsteps)
        dt = time.perf_counter() - t0
        inf = g.info()
        res[name] = {"syn_updates_per_s": d.num_syn * done / dt, "us_per_step": dt / max(done, 1) * 1e6,
                     "device_mb": inf.device_bytes / 1e6,
                     "engine": {1: "l2_gather", 2: "resident", 3: "tiled"}.get(inf.engine, "?")}
        if inf.engine == libsnp.SNP_ENGINE_TILED:
            res[name]["launch_shape"] = {"clusters": inf.tiled_ctas // max(1, inf.tiled_partitions),
                                         "ctas_per_cluster": inf.tiled_partitions,
                                         "accumulator_bits": inf.tiled_acc_bits,
                                         "smem_bytes_per_cta": inf.tiled_smem_bytes}
        g.close()
    if chosen is not None and "dense" not in chosen:
        return {"metric": "synaptic updates/s", "workload": "skewed", "value": next(
                    (r.get("syn_updates_per_s") for r in res.values() if "syn_updates_per_s" in r), None),
                "unit": "synaptic updates/s", "engines": res,
                "config": {"q": d.q, "num_syn": d.num_syn, "steps": nsteps, "engines_run": sorted(chosen)}}
    dd, _, _ = synth.skewed_dense_copy()
    g = libsnp.System(dd, form=libsnp.SNP_FORM_DENSE, select=libsnp.SNP_SELECT_PHILOX, seed=dd.seed)
    g.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = g.step(10)
    dt = time.perf_counter() - t0
    dense_bytes = dd.m * dd.q * 4
    res["dense_16k"] = {"us_per_step": dt / max(done, 1) * 1e6, "matrix_gb": dense_bytes / 1e9,
                        "matrix_gbs": dense_bytes * done / dt / 1e9}
    g.close()
    gt = libsnp.System(dd, engine=libsnp.SNP_ENGINE_TILED, select=libsnp.SNP_SELECT_PHILOX, seed=dd.seed)
    gt.step(2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done = gt.step(10)
    res["tiled_16k_us_per_step"] = (time.perf_counter() - t0) / max(done, 1) * 1e6
    gt.close()
    return {"metric": "synaptic updates/s", "workload": "skewed", "value": res["auto"].get("syn_updates_per_s"),
            "unit": "synaptic updates/s", "engines": res,
            "config": {"q": d.q, "num_syn": d.num_syn, "steps": nsteps, "dense_copy_q": dd.q, "dense_copy_m": dd.m}}


def engines(args, libsnp, synth):
    import hashlib
    import torch
    d, _, _ = synth.large_1m()
    res, digests = {}, set()
    for name, kw in [("tiled", dict(engine=libsnp.SNP_ENGINE_TILED)),
                     ("l2_gather", dict(engine=libsnp.SNP_ENGINE_LAUNCH)),
                     ("push", dict(prop=libsnp.SNP_PROP_PUSH)),
                     ("ell_pull", dict(form=libsnp.SNP_FORM_ELL)),
                     ("ell_push", dict(form=libsnp.SNP_FORM_ELL, prop=libsnp.SNP_PROP_PUSH))]:
        g = libsnp.System(d, select=libsnp.SNP_SELECT_PHILOX, seed=d.seed, **kw)
        g.step(8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = g.step(192)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        digests.add(hashlib.sha256(g.config().tobytes()).hexdigest())
        res[name] = {"us_per_step": dt / max(done, 1) * 1e6, "syn_updates_per_s": d.num_syn * done / dt,
                     "device_mb": g.info().device_bytes / 1e6}
        g.close()
    return {"metric": "synaptic updates/s", "workload": "engines", "value": res["tiled"]["syn_updates_per_s"],
            "unit": "synaptic updates/s", "engines": res, "same_final_configuration": len(digests) == 1,
            "config": {"q": d.q, "num_syn": d.num_syn, "timed_steps": 192}}


def shards(args, libsnp, synth):
    """The sharded step of one system (one shard per device in a multi-GPU
    run) with all shards on this GPU: per step every shard's phase 1 (its
    activity read back to the host), the slices copied into every shard's
    emission vector, every shard's phase 2.  Timed on the host around a
    device synchronize; checked against the unsharded system."""
    import torch
    from paper_2408_04343_gb300 import shard as SH
    d, _, _ = synth.large_1m()
    warm, n = 4, 64
    sel = libsnp.SNP_SELECT_PHILOX
    ref = libsnp.System(d, select=sel, seed=d.seed, engine=libsnp.SNP_ENGINE_TILED)
    ref.step(warm)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    done_ref = ref.step(n)
    torch.cuda.synchronize()
    ref_dt = time.perf_counter() - t0
    C_ref = ref.config().copy()
    ref.close()
    res = {"unsharded_tiled": {"us_per_step": ref_dt / max(done_ref, 1) * 1e6,
                               "syn_updates_per_s": d.num_syn * done_ref / ref_dt}}
    for world in (1, 2, 4):
        ranges, chunk = SH.shard_ranges(d.q, world)
        Es = [torch.zeros(world * chunk + 1, dtype=torch.int16, device="cuda") for _ in range(world)]
        shs = [libsnp.Shard(d, lo, hi, select=sel, seed=d.seed, E=Es[r]) for r, (lo, hi) in enumerate(ranges)]
        ex = SH.local_exchange([(Es[r], lo, hi) for r, (lo, hi) in enumerate(ranges)])
        k = SH.run(shs, warm, 0, ex, lambda a: a)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = SH.run(shs, n, k, ex, lambda a: a)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        C = np.concatenate([sh.get_state()[0] for sh in shs])
        res[f"shards_{world}"] = {"us_per_step": dt / max(done, 1) * 1e6, "syn_updates_per_s": d.num_syn * done / dt,
                                  "identical_to_unsharded": bool(done == done_ref and (C == C_ref).all())}
        for sh in shs:
            sh.close()
    return {"metric": "synaptic updates/s", "workload": "shards", "value": res["shards_2"]["syn_updates_per_s"],
            "unit": "synaptic updates/s", "shards": res,
            "config": {"q": d.q, "num_syn": d.num_syn, "timed_steps": n, "exchange": "device copies, one GPU"}}


def families(args, libsnp, synth):
    import torch
    import numpy as np
    forms = {"compressed": dict(form=libsnp.SNP_FORM_OPT), "ell": dict(form=libsnp.SNP_FORM_ELL),
             "sparse": dict(form=libsnp.SNP_FORM_DENSE)}
    paper_form = {"compressed": libsnp.SNP_FORM_OPT, "ell": libsnp.SNP_FORM_ELL, "sparse": libsnp.SNP_FORM_DENSE}
    out = {"sort": [], "subset_sum_shaped": []}
    dense_cap = 24 << 30   # the dense form is built on the host too: keep it to 24 GB

    def run_one(d, fam, n, nsteps, select, check=None):
        z = int(np.diff(d.syn_offsets).max()) if d.q else 0
        row = {"n": n, "q": d.q, "m": d.m, "z": z, "forms": {}}
        for name, kw in forms.items():
            elems = libsnp.paper_format_elements(paper_form[name], d.q, d.m, z)
            ent = {"paper_elements": elems, "paper_mb_at_2_bytes": elems * 2 / 1e6}
            if name == "sparse" and d.m * d.q * 4 > dense_cap:
                ent["unavailable"] = "dense m x q matrix above 24 GB"
                row["forms"][name] = ent
                continue
            try:
                g = libsnp.System(d, select=select, seed=d.seed, **kw)
            except libsnp.SnpError as e:
                ent["unavailable"] = str(e)
                row["forms"][name] = ent
                continue
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            done = g.step(nsteps)
            dt = time.perf_counter() - t0
            ent.update({"device_mb": g.info().device_bytes / 1e6, "steps": done, "run_ms": dt * 1e3,
                        "us_per_step": dt / max(done, 1) * 1e6})
            if check is not None:
                ent["correct"] = bool(check(g.get_state()[0], done))
            g.close()
            row["forms"][name] = ent
        out[fam].append(row)

    for n in (10, 50, 100, 250, 500, 1000, 2000):
        d = synth.sort_system(list(range(n, 0, -1)))
        run_one(d, "sort", n, 4 * n + 10, libsnp.SNP_SELECT_FIRST,
                check=lambda C, done, n=n: done == n + 1 and bool((C[2 * n:] == np.arange(1, n + 1)).all()))
    for n in (100, 1000, 5000, 20000):
        d = synth.subset_sum_shaped(n)
        run_one(d, "subset_sum_shaped", n, 200, libsnp.SNP_SELECT_PHILOX)
    return {"metric": "device memory and run time per instance size", "workload": "families", "value": None,
            "unit": "MB / ms", **out}


def tree_workload(args, libsnp, synth):
    import torch
    from paper_2408_04343_gb300 import tree
    d = synth.subset_sum_shaped(14, seed=7007)
    res = {}
    for name, kw, depth in [("batched", dict(batched=True), 12), ("per_branch", dict(batched=False), 3)]:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        t = tree.explore(d, depth, max_branches=1 << 16, max_nodes=1 << 20, **kw)
        dt = time.perf_counter() - t0
        res[name] = {"depth": depth, "nodes": len(t.states), "branches": len(t.edges), "seconds": dt,
                     "branches_per_s": len(t.edges) / dt, "truncated": len(t.truncated)}
    return {"metric": "computation-tree branches explored per second", "workload": "tree",
            "value": res["batched"]["branches_per_s"], "unit": "branches/s",
            "config": {"system": "subset-sum-shaped stand-in, n = 14", "q": d.q, "m": d.m}, **res}
