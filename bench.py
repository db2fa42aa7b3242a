#!/usr/bin/env python
"""Benchmark of the B300 DFTT noisy-statevector engine.

Workload (default): the 28-qubit QAOA-style circuit on a seeded random
3-regular graph, 4 layers of RZZ(gamma) + RX(beta), 2q depolarizing 5e-3
and 1q 5e-4, 1e6 shots, alpha = 0.01, beta = 100, complex64 state (2 GiB)
with an FP64 output distribution (2 GiB).

A step is one traversal of the whole instance tree on the device: every
fused pass, Pauli injection, leaf accumulation, drift check and snapshot
restore (the plan -- ER sampling, tally, commutation, pruning, DFS order --
is built and its device program uploaded before the timed region; the
end-to-end number below includes them).  ``value`` = kept instances
(leaves) per second over all ranks.

Also reported: gate-amplitude updates/s (executed, and the from-scratch
equivalent N_l * G * 2^n), the HBM roofline of the fused pass kernel
measured live with CUDA events around each pass launch, the end-to-end
rate through the C ABI from host buffers (plan + compile + upload +
traversal + copy of the distribution back), the paper's uncompute DFTT and
the plain from-scratch GPU form timed beside the headline traversal, the
error of each against the oracle on an instance subset the oracle plans
itself, p50/p99 job latency of a short served run, the oracle on all host
cores and on one core as the CPU baseline, and SM clocks sampled during the
timed region.

``--impl reference`` times the CPU oracle (the reference arm): each step
simulates a bounded prefix of the first instance of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import tusq_workloads as W  # noqa: E402

WORKLOAD_DESC = {
    "qaoa_28q": "28-qubit QAOA on a seeded random 3-regular graph, p=4 layers RZZ(gamma)+RX(beta), "
                "2q depolarizing 5e-3, 1q 5e-4, 1e6 shots, alpha=0.01 beta=100",
    "brickwork_20q": "20-qubit brickwork depth 40, Haar SU(2) + CZ, depolarizing 1e-3/1e-2, 1e6 shots",
    "random_layers_6q": "6-qubit random layers depth 20, depolarizing 1e-3/1e-2, 1e4 shots",
    "qaoa_26q": "26-qubit QAOA on a seeded random 3-regular graph, p=4 layers RZZ(gamma)+RX(beta), "
                "2q depolarizing 5e-3, 1q 5e-4, 1e6 shots, alpha=0.01 beta=100 (profiling case)",
    "brickwork_24q": "24-qubit brickwork depth 40, Haar SU(2) + CZ, depolarizing 1e-3/1e-2, 1e6 shots "
                     "(state above L2)",
}
SHOTS = {"qaoa_28q": 1_000_000, "brickwork_20q": 1_000_000, "random_layers_6q": 10_000,
         "qaoa_26q": 1_000_000, "brickwork_24q": 1_000_000}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0}, "fallback"


def plan_admitted(T, circuits, shots_of, max_work, max_instances):
    """Plan every job on host threads (the planner releases the GIL) and keep
    those whose pruned tree costs at most max_work gate-amplitude updates
    (tree edges x 2^n) and has at most max_instances leaves (the compiled
    device program grows with the leaves).  A job whose shots are nearly all
    distinct keeps ~shots instances after pruning (alpha * c_max <= 1 marks
    every realization significant); such a job is rejected before its
    schedule is compiled.  Returns (kept indices, plans by index, rejected
    list, seconds)."""
    from concurrent.futures import ThreadPoolExecutor
    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=max(1, (os.cpu_count() or 2) // 2)) as pool:
        plans = list(pool.map(lambda jc: T.plan(jc[1], shots_of(jc[0]), jc[0]), enumerate(circuits)))
    kept, rejected = [], []
    for j, (c, p) in enumerate(zip(circuits, plans)):
        st = p.stats()
        work = float(st["tree_gate_edges"]) * float(1 << c.n_qubits)
        if work <= max_work and st["n_instances"] <= max_instances:
            kept.append(j)
        else:
            rejected.append({"job": j, "qubits": c.n_qubits, "gates": c.n_gates,
                             "instances": int(st["n_instances"]), "work": work})
    return kept, plans, rejected, time.perf_counter() - t0


class ClockSampler:
    """nvidia-smi SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.idx = device_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # nvidia-smi needs a moment to start: wait (at most 3 s) for its
            # first sample so that short regions are sampled too
            t_end = time.time() + 3.0
            while not self.rows and time.time() < t_end:
                time.sleep(0.02)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for k, name in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profile(kernel_src: str):
    """Per-launch DRAM traffic of the pass kernel from the committed ncu
    summary (profiles/pass_kernel_ncu.json), as DRAM bytes per algorithmic
    byte; None when the kernel source changed since the capture."""
    path = os.path.join(ROOT, "profiles", "pass_kernel_ncu.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    digest = hashlib.sha256(open(kernel_src, "rb").read()).hexdigest()[:16]
    if rec.get("kernels_cu_sha256_16") != digest:
        return None
    try:
        return float(rec["dram_bytes_per_algorithmic_byte"])
    except (KeyError, TypeError, ValueError):
        return None


def _omp_threads(k: int) -> None:
    """Set the OpenMP team size of later parallel regions in this process
    (the oracle's OpenMP runtime is the process's libgomp)."""
    import ctypes
    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(k))
    except OSError:
        pass


def cpu_baseline(circ, plan_inst, budget_s: float = 15.0, threads: int = 0):
    """The oracle as it stands, timed on a bounded sample: a prefix of the
    first kept instance's gates (with its Pauli events), sized to about
    budget_s of host work; the rate is scaled to instances/s.  threads = 0:
    every host core; otherwise the OpenMP team is limited to that many."""
    import oracle
    oracle.lib()
    all_cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    cores = threads if threads > 0 else all_cores
    _omp_threads(cores)
    G = circ.n_gates
    ev = list(plan_inst[0])
    k = 2
    try:
        while True:
            sub = W.Circuit(circ.n_qubits, circ.gates[:k], circ.channels[:k])
            t0 = time.perf_counter()
            oracle.simulate(sub, [e for e in ev if e[0] < k])
            dt = time.perf_counter() - t0
            if dt > budget_s / 3 or k >= G:
                break
            k = min(G, max(k + 1, int(k * min(8.0, budget_s / max(dt, 1e-3)))))
    finally:
        _omp_threads(all_cores)
    rate = (k / G) / dt
    return {"value": rate, "unit": "instances/s", "cores": cores, "kind": "oracle",
            "sample": f"first {k} of {G} gates of one instance ({circ.n_qubits} qubits, complex128), "
                      f"{dt:.2f} s, scaled by {G}/{k}"}


def error_vs_oracle(T, torch, circ, shots, seed, arms, sp):
    """Error of the engine against the oracle (complex128, every instance
    simulated from |0..0> with no tree) on an instance subset of the
    workload that the oracle plans itself: the first leaf in DFS order and
    the ideal instance (the last leaf), with their weights.  The subset
    runs through the engine as one plan under each arm's options; max-abs
    and total variation over all 2^n outcomes."""
    import oracle
    t0 = time.perf_counter()
    opl = oracle.plan(circ, shots, seed)
    idx = [0, len(opl.inst) - 1]
    subset = [[tuple(int(v) for v in e) for e in opl.inst[i]] for i in idx]
    w = np.array([opl.weights[i] for i in idx])
    ref = oracle.run_instances(circ, subset, w)
    oracle_s = time.perf_counter() - t0
    pl = T.tusq_plan_from_instances(T.circuit_from(circ), subset, w)
    refd = torch.from_numpy(ref).to("cuda")
    del ref
    probs = torch.empty_like(refd)
    per = {}
    for name, o in arms:
        ex = T.Exec(pl, o, sp)
        ex.launch(probs.data_ptr(), sp)
        ex.finish()
        d = (probs - refd).abs()
        per[name] = {"max_abs": float(d.max()), "tv": float(d.sum())}
        del ex, d
    del probs, refd
    torch.cuda.empty_cache()
    return {"instances_compared": len(idx), "subset": "first DFS leaf + ideal leaf, planned by the oracle",
            "subset_weight": float(w.sum()), "tolerance": {"max_abs": 1e-5, "tv": 1e-4},
            "max_abs": max(v["max_abs"] for v in per.values()), "tv": max(v["tv"] for v in per.values()),
            "per_arm": per, "oracle_seconds": oracle_s}


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on bounded samples of the workload."""
    if rank != 0:
        return
    import oracle
    oracle.build()
    circ = W.WORKLOADS[args.workload]()
    G = circ.n_gates
    k = max(1, min(G, args.ref_gates))
    sub = W.Circuit(circ.n_qubits, circ.gates[:k], circ.channels[:k])
    for _ in range(args.warmup):
        oracle.simulate(sub, [])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.simulate(sub, [])
    dt = (time.perf_counter() - t0) / args.steps
    value = (k / G) / dt
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {
        "impl": "reference", "metric": "noisy instances/s", "value": value, "unit": "instances/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": {"workload": WORKLOAD_DESC[args.workload], "sample_gates": k},
        "cpu_baseline": {"value": value, "unit": "instances/s", "cores": cores, "kind": "oracle",
                         "sample": f"first {k} of {G} gates of one instance, scaled by {G}/{k}"},
        "e2e": {"value": value, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_batch(args, T, torch):
    """Config 4: many noisy jobs of uneven size and depth in one persistent
    launch replayed from a CUDA graph.  Jobs that fit a CTA's shared memory
    (<= 13 qubits, complex64) run whole in one CTA; larger ones run on CTA
    groups with their state in global memory, scheduled onto the grid by the
    host.  Options (traversal, fusion schedule, CTAs per group) autotuned on
    a sample of the jobs.  One step = every job once."""
    all_jobs = W.job_mix(args.jobs, seed=0, n_lo=12, n_hi=18, d_lo=20, d_hi=80)
    kept, all_plans, rejected, plan_s = plan_admitted(T, all_jobs, lambda j: args.batch_shots, args.max_job_work,
                                                      args.max_job_instances)
    jobs = [all_jobs[j] for j in kept]
    plans = [all_plans[j] for j in kept]
    del all_plans
    n_inst = sum(p.stats()["n_instances"] for p in plans)
    outs = [torch.empty(1 << c.n_qubits, dtype=torch.float64, device="cuda") for c in jobs]
    stream = torch.cuda.Stream()
    base = T.run_opts(precision=T.C64, tc_mode=args.tc_mode)
    sample = list(range(0, len(jobs), max(1, len(jobs) // 256)))[:256]
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        best, tune_ms = T.tusq_batch_autotune([plans[i] for i in sample], [outs[i].data_ptr() for i in sample],
                                              base, stream.cuda_stream)
    tune_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        b = T.Batch(plans, [o.data_ptr() for o in outs], best, use_graph=True, stream=stream.cuda_stream)
    create_s = time.perf_counter() - t0

    def step():
        b.launch(stream.cuda_stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(torch.cuda.current_device()) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    secs = ev0.elapsed_time(ev1) / 1e3 / args.steps
    info = b.finish()
    # error against the oracle (complex128, every instance from |0..0>) of the
    # cheapest jobs of each kind (instances x gates x 2^n), so that the check
    # stays within seconds of host time
    import oracle
    errs = []
    cost = {i: plans[i].stats()["n_instances"] * jobs[i].n_gates * (1 << jobs[i].n_qubits) for i in range(len(jobs))}
    small = [i for i, c in enumerate(jobs) if c.n_qubits <= 13]
    group = [i for i, c in enumerate(jobs) if c.n_qubits > 13]
    for i in sorted(small, key=cost.get)[:2] + sorted(group, key=cost.get)[:2]:
        ref, _ = oracle.run(jobs[i], args.batch_shots, kept[i])
        d = np.abs(outs[i].cpu().numpy() - ref)
        errs.append({"job": kept[i], "qubits": jobs[i].n_qubits, "max_abs": float(d.max()), "tv": float(d.sum())})
    return {
        "metric": "noisy instances/s (batched jobs)", "value": n_inst / secs, "unit": "instances/s",
        "jobs_per_s": len(jobs) / secs, "ms_per_step": secs * 1e3, "steps": args.steps, "warmup": args.warmup,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"{args.jobs} jobs, 12-18 qubits, brickwork/QAOA mix, depth 20-80, "
                               f"{args.batch_shots} shots each", "jobs_run": len(jobs),
                   "rejected_over_work_budget": rejected, "max_job_work": args.max_job_work,
                   "max_job_instances": args.max_job_instances,
                   "tc_mode": ["none", "tf32x3", "bf16x3", "tf32"][args.tc_mode],
                   "one_launch": {"single_cta_jobs": len(small), "group_jobs": b.group_jobs(),
                                  "graph_replay": True},
                   "instances": n_inst,
                   "autotuned": {"traversal": best.traversal, "schedule": best.schedule,
                                 "group_ctas": best.group_ctas or 16, "ms_on_sample": tune_ms,
                                 "sample_jobs": len(sample), "seconds": tune_s}},
        "plan_seconds": plan_s, "create_seconds": create_s, "error_vs_oracle": errs,
        "run_info": {k: info[k] for k in ("passes", "gate_apps", "leaf_passes", "restores", "unrecovered",
                                          "dense_ops")},
        "clocks": clk.summary(),
    }


def hellinger_fidelity(p, q, torch):
    """Classical fidelity (sum_x sqrt(p_x q_x))^2 of two distributions."""
    return float(torch.sqrt(p.clamp(min=0) * q.clamp(min=0)).sum() ** 2)


def run_fidelity(args, T, torch):
    """Pruning study (Sec. IV-C metric delta, Sec. V-D ablation): for seeded
    circuits shaped like the paper's workloads, the output with pruning
    (alpha = 0.01, beta = 100) and without it, each against the noiseless
    output.  delta = |f_A - f_B| / (f_A + f_B) with f the classical fidelity
    to the noiseless distribution; gamma = time without / time with pruning;
    the ablation gives the matrix-vector products each stage leaves (shots x
    gates without tally; unique ERs x gates after tally and after
    commutation; kept instances x gates after pruning; DFTT edge traversals).
    Both arms simulate every instance from |0..0>."""
    cases = [("qaoa_12q_p2", lambda p1, p2: W.qaoa_3regular(12, 2, 3, p1, p2)),
             ("qaoa_16q_p3", lambda p1, p2: W.qaoa_3regular(16, 3, 4, p1, p2)),
             ("brickwork_12q_d20", lambda p1, p2: W.brickwork(12, 20, 5, p1, p2)),
             ("brickwork_16q_d30", lambda p1, p2: W.brickwork(16, 30, 6, p1, p2)),
             ("random_layers_8q_d30", lambda p1, p2: W.random_layers(8, 30, 7, p1, p2)),
             ("qaoa_20q_p2", lambda p1, p2: W.qaoa_3regular(20, 2, 8, p1, p2))]
    shots = args.fidelity_shots
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    out = []
    for name, make in cases:
        noisy, ideal_c = make(1e-3, 1e-2), make(0.0, 0.0)
        ideal, _ = T.run_torch(T.plan(ideal_c, 1, 0), T.run_opts(precision=T.C64))
        row = {"case": name, "qubits": noisy.n_qubits, "gates": noisy.n_gates}
        res = {}
        for prune in (True, False):
            pl = T.plan(noisy, shots, 0, prune=prune)
            st = pl.stats()
            if st["n_instances"] > 10_000:      # the unpruned program would take gigabytes
                res[prune] = None
                row["unpruned_instances"] = st["n_instances"]
                continue
            # both arms from scratch (no uncompute: the unpruned trees are deeper
            # than the snapshot LIFO), so the comparison isolates pruning
            ex = T.Exec(pl, T.run_opts(precision=T.C64, traversal=T.FROM_SCRATCH), sp)
            probs = torch.empty(1 << noisy.n_qubits, dtype=torch.float64, device="cuda")
            ex.launch(probs.data_ptr(), sp)
            ex.finish()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ex.launch(probs.data_ptr(), sp)
            b.record(stream)
            ex.finish()
            res[prune] = (probs, a.elapsed_time(b), st)
        p_st = res[True][2]
        G = noisy.n_gates
        row["ablation_matvecs"] = {"no_tally": shots * G, "tally": p_st["n_raw_unique"] * G,
                                   "commutation": p_st["n_commuted_unique"] * G,
                                   "pruning": p_st["n_instances"] * G, "dftt": p_st["dftt_gate_apps"]}
        row["pruned_instances"] = p_st["n_instances"]
        f_a = hellinger_fidelity(res[True][0], ideal, torch)
        row["fidelity_pruned"] = f_a
        row["ms_pruned"] = res[True][1]
        if res[False] is not None:
            f_b = hellinger_fidelity(res[False][0], ideal, torch)
            row.update({"fidelity_unpruned": f_b, "delta": abs(f_a - f_b) / (f_a + f_b),
                        "unpruned_instances": res[False][2]["n_instances"], "ms_unpruned": res[False][1],
                        "gamma_prune": res[False][1] / res[True][1]})
        out.append(row)
    deltas = [r["delta"] for r in out if "delta" in r]
    return {"metric": "pruning relative fidelity difference delta (alpha=0.01, beta=100)",
            "value": float(np.mean(deltas)) if deltas else None, "max": float(np.max(deltas)) if deltas else None,
            "unit": "fraction", "shots": shots, "dtype": "c64", "data": "synthetic", "cases": out}


def run_caching(args, T, torch):
    """DFTT+Caching (Sec. III-B2) on a circuit with mid-circuit resets: a
    22-qubit brickwork with three layers of two resets each (every kept
    instance has 2^6 Kraus-branch leaves).  For cache capacities K = 0..4 the
    uncompute traversal without drift checks (the cache is its only saved
    state) is timed on the device, with the paper's recovery metric
    alpha(K) = (N1 - N_K) / (N1 - N2): N1 = gate applications with every
    leaf from |0..0>, N2 = those of a DFTT that could uncompute the resets,
    N_K = those executed with capacity K.  The snapshot traversal and the
    from-scratch form are timed beside them."""
    circ = W.mcm_brickwork(args.mcm_qubits, 12, 3, 2, 0, 1e-3, 1e-2)
    pl = T.plan(circ, 1_000_000, 0)
    st = pl.stats()
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    probs = torch.empty(1 << circ.n_qubits, dtype=torch.float64, device="cuda")

    def timed(**kw):
        ex = T.Exec(pl, T.run_opts(precision=T.C64, **kw), sp)
        ex.launch(probs.data_ptr(), sp)
        info = ex.finish()
        ms = []
        for _ in range(2):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            ex.launch(probs.data_ptr(), sp)
            b.record(stream)
            ex.finish()
            ms.append(a.elapsed_time(b))
        del ex
        return min(ms), info, probs.sum().item()

    n1_ms, n1_info, _ = timed(traversal=T.FROM_SCRATCH)
    N1 = n1_info["gate_apps"]
    N2 = st["dftt_gate_apps"]
    rows = []
    for K in range(0, 5):
        ms, info, total = timed(traversal=T.DFTT, drift_tol=-1.0, cache_states=K)
        rows.append({"K": K, "ms": ms, "gate_apps": info["gate_apps"], "passes": info["passes"],
                     "alpha": (N1 - info["gate_apps"]) / (N1 - N2), "cache_restores": info["cache_restores"],
                     "rederives": info["rederives"], "sum_probs": total})
    snap_ms, snap_info, _ = timed(traversal=T.DFTT_SNAPSHOT)
    return {"metric": "DFTT+Caching recovery alpha(K) and time, mid-circuit resets", "unit": "fraction",
            "value": rows[-1]["alpha"], "dtype": "c64", "data": "synthetic",
            "workload": {"circuit": circ.name, "qubits": circ.n_qubits, "gates": circ.n_gates,
                         "resets": st["n_noninvertible"], "layers": st["n_noninv_layers"],
                         "ecm_instances": st["n_ecm_instances"], "leaves": st["n_instances"], "shots": 1_000_000},
            "N1_scratch_gate_apps": N1, "N2_dftt_gate_apps": N2, "scratch_ms": n1_ms,
            "snapshot_ms": snap_ms, "snapshot_gate_apps": snap_info["gate_apps"], "uncompute": rows}


def served_measure(T, torch, plans, n_inst, qubits, rates, slots, budget, seed=1):
    """Serve `plans` through the serving loop: first all at once (capacity),
    then with Poisson arrivals at each fraction of that capacity.  Returns
    (capacity in jobs/s, per-rate latency and throughput rows)."""
    outs = [torch.empty(1 << n, dtype=torch.float64, device="cuda") for n in qubits]
    opts = T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT)
    srv = T.Server(budget, n_streams=slots)
    t0 = time.perf_counter()
    for p, o in zip(plans, outs):
        srv.submit(p, o.data_ptr(), opts)
    srv.drain()
    capacity = len(plans) / (time.perf_counter() - t0)
    del srv
    rng = np.random.default_rng(seed)
    results = []
    for frac in rates:
        lam = frac * capacity
        gaps = rng.exponential(1.0 / lam, len(plans))
        srv = T.Server(budget, n_streams=slots)
        t0 = time.perf_counter()
        ids = []
        for p, o in zip(plans, outs):
            target = t0 + (gaps[:len(ids) + 1].sum())
            while time.perf_counter() < target:
                time.sleep(0.0002)
            ids.append(srv.submit(p, o.data_ptr(), opts))
        srv.drain()
        wall = time.perf_counter() - t0
        lat = np.array([srv.poll(i)[1] for i in ids])
        results.append({"rate_frac_of_capacity": frac, "rate_jobs_per_s": lam,
                        "p50_latency_s": float(np.percentile(lat, 50)),
                        "p99_latency_s": float(np.percentile(lat, 99)),
                        "instances_per_s": sum(n_inst) / wall, "jobs_per_s": len(plans) / wall})
        del srv
    del outs
    torch.cuda.empty_cache()
    return capacity, results


def run_served(args, T, torch):
    """Config 5: Poisson arrivals of jobs (10-30 qubits, depth 20-100, p in
    [1e-4, 1e-2], 1e5-1e6 shots) into the serving loop (admission by HBM
    footprint, concurrent streams, state resident until done).  Reports
    latency (submit to completion) percentiles and throughput per rate."""
    all_jobs = W.served_stream(args.jobs, seed=0)
    kept, all_plans, rejected, plan_s = plan_admitted(T, [c for c, _ in all_jobs], lambda j: all_jobs[j][1],
                                                      args.max_job_work, args.max_job_instances)
    stream_jobs = [all_jobs[j] for j in kept]
    plans = [all_plans[j] for j in kept]
    del all_plans
    n_inst = [p.stats()["n_instances"] for p in plans]
    budget = int(args.hbm_budget_gb * (1 << 30))
    capacity, results = served_measure(T, torch, plans, n_inst, [c.n_qubits for c, _ in stream_jobs],
                                       args.rates, args.slots, budget)
    return {"metric": "served noisy jobs: p50/p99 latency and instances/s", "unit": "s / instances/s",
            "capacity_jobs_per_s": capacity, "jobs": len(plans), "hbm_budget_gb": args.hbm_budget_gb,
            "jobs_offered": args.jobs, "rejected_over_work_budget": rejected, "max_job_work": args.max_job_work,
            "max_job_instances": args.max_job_instances,
            "plan_seconds": plan_s,
            "qubits": [c.n_qubits for c, _ in stream_jobs], "rates": results, "dtype": "c64",
            "data": "synthetic"}


def served_subrun(args, T, torch):
    """A short served run for the headline line: args.served_jobs jobs of the
    served stream (10-args.served_max_qubits qubits), Poisson arrivals at
    args.served_rate x the measured capacity; p50/p99 job latency."""
    all_jobs = W.served_stream(args.served_jobs, seed=0, n_hi=args.served_max_qubits)
    kept, all_plans, rejected, plan_s = plan_admitted(T, [c for c, _ in all_jobs], lambda j: all_jobs[j][1],
                                                      args.max_job_work, args.max_job_instances)
    plans = [all_plans[j] for j in kept]
    qubits = [all_jobs[j][0].n_qubits for j in kept]
    del all_plans
    n_inst = [p.stats()["n_instances"] for p in plans]
    capacity, results = served_measure(T, torch, plans, n_inst, qubits, [args.served_rate], args.slots,
                                       int(args.hbm_budget_gb * (1 << 30)))
    r = results[0]
    return {"jobs": len(plans), "jobs_offered": args.served_jobs, "qubits": f"10-{args.served_max_qubits}",
            "rejected_over_work_budget": len(rejected), "capacity_jobs_per_s": capacity,
            "rate_frac_of_capacity": args.served_rate, "p50_latency_s": r["p50_latency_s"],
            "p99_latency_s": r["p99_latency_s"], "instances_per_s": r["instances_per_s"],
            "plan_seconds": plan_s}


def run_streamed_mode(args, T, torch):
    """Config 2 without pruning: the 20-qubit depth-40 brickwork, every one of
    the distinct instances of args.stream_shots shots kept (about 1e5 leaves),
    traversed by tusq_run_streamed -- DFS chunks of args.chunk_leaves leaves
    whose programs compile on host threads while the GPU runs the previous
    chunks.  One step = one whole streamed traversal, compile included (the
    program is never materialised whole).  Checked by the output's sum (the
    tally weights sum to 1)."""
    circ = W.WORKLOADS["brickwork_20q"]()
    t0 = time.perf_counter()
    pl = T.plan(circ, args.stream_shots, 0, prune=False)
    plan_s = time.perf_counter() - t0
    st = pl.stats()
    probs = torch.empty(1 << circ.n_qubits, dtype=torch.float64, device="cuda")
    sp = torch.cuda.current_stream().cuda_stream
    opts = T.run_opts(precision=T.C64, traversal=T.DFTT_SNAPSHOT, tc_mode=args.tc_mode)
    times, info = [], None
    with ClockSampler(torch.cuda.current_device()) as clk:
        for _ in range(max(1, args.steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            info = T.tusq_run_streamed(pl, probs.data_ptr(), args.chunk_leaves, opts, 0, sp)
            times.append(time.perf_counter() - t0)
    secs = min(times)
    n_inst = st["n_instances"]
    return {"metric": "noisy instances/s (streamed, unpruned)", "value": n_inst / secs, "unit": "instances/s",
            "seconds_per_traversal": secs, "steps": len(times), "warmup": 0, "dtype": "c64", "data": "synthetic",
            "config": {"workload": "20-qubit brickwork depth 40, Haar SU(2) + CZ, depolarizing 1e-3/1e-2, "
                                   f"{args.stream_shots} shots, no pruning",
                       "instances": n_inst, "chunk_leaves": args.chunk_leaves,
                       "chunks": (n_inst + args.chunk_leaves - 1) // args.chunk_leaves,
                       "compile_threads": "half the host cores", "tc_mode": args.tc_mode},
            "plan_seconds": plan_s, "sum_probs": float(probs.sum()),
            "run_info": {k: info[k] for k in ("passes", "gate_apps", "leaf_passes", "restores", "unrecovered",
                                              "program_bytes", "algorithmic_bytes")},
            "clocks": clk.summary()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qaoa_28q", choices=sorted(WORKLOAD_DESC))
    ap.add_argument("--traversal", default="snapshot", choices=["dftt", "scratch", "snapshot"])
    ap.add_argument("--precision", default="c64", choices=["c64", "c128"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--ref-gates", type=int, default=12)
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the other traversals (from scratch, uncompute DFTT) beside the headline")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the error against the oracle on an instance subset of the workload")
    ap.add_argument("--no-served", action="store_true", help="skip the short served sub-run")
    ap.add_argument("--served-jobs", type=int, default=16)
    ap.add_argument("--served-max-qubits", type=int, default=26)
    ap.add_argument("--served-rate", type=float, default=0.75)
    ap.add_argument("--stream-shots", type=int, default=100_000)
    ap.add_argument("--chunk-leaves", type=int, default=4096)
    ap.add_argument("--mode", default="main", choices=["main", "batch", "served", "fidelity", "caching", "streamed"],
                    help="main: the 28-qubit headline; batch: config 4; served: config 5; "
                         "fidelity: pruning delta and per-stage ablation")
    ap.add_argument("--fidelity-shots", type=int, default=20_000)
    ap.add_argument("--mcm-qubits", type=int, default=22, help="qubits of the --mode caching circuit")
    ap.add_argument("--streams", type=int, default=32,
                    help="batch: streams the jobs too large for one CTA are spread over")
    ap.add_argument("--slots", type=int, default=8,
                    help="served: stream slots of the serving loop (32 measured no higher capacity and a "
                         "higher p99 under load than 8)")
    ap.add_argument("--tc-mode", type=int, default=0, choices=[0, 1, 2, 3],
                    help="tensor-core dense stages: 0 none, 1 TF32x3, 2 BF16x3, 3 TF32 (main: the timed "
                         "traversal; batch: the jobs run per launch)")
    ap.add_argument("--subtrees", type=int, default=1,
                    help="main: traverse the DFS order as this many concurrent chunks (parallel subtrees)")
    ap.add_argument("--graph", type=int, default=1,
                    help="batch: replay each per-stream job's traversal from a captured CUDA graph; "
                         "main: time the traversal on a side stream with graph replay")
    ap.add_argument("--jobs", type=int, default=2048)
    ap.add_argument("--batch-shots", type=int, default=100_000)
    ap.add_argument("--hbm-budget-gb", type=float, default=200.0)
    ap.add_argument("--rates", type=float, nargs="+", default=[0.25, 0.5, 1.0, 2.0])
    ap.add_argument("--max-job-work", type=float, default=3e13,
                    help="batch/served: jobs whose pruned tree exceeds this many gate-amplitude updates "
                         "(tree edges x 2^n) are rejected at admission and reported")
    ap.add_argument("--max-job-instances", type=int, default=5000,
                    help="batch/served: jobs whose pruned tree keeps more leaves are rejected likewise")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2508_04880_b300 as T
    torch.cuda.set_device(local)
    if args.mode != "main":
        line = {"batch": run_batch, "served": run_served, "fidelity": run_fidelity,
                 "caching": run_caching, "streamed": run_streamed_mode}[args.mode](args, T, torch)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    trav = {"dftt": T.DFTT, "scratch": T.FROM_SCRATCH, "snapshot": T.DFTT_SNAPSHOT}[args.traversal]
    prec = T.C64 if args.precision == "c64" else T.C128
    circ = W.WORKLOADS[args.workload]()
    shots = SHOTS[args.workload]
    seed = rank     # weak scaling: every rank simulates its own noisy job
    t0 = time.perf_counter()
    plan = T.plan(circ, shots, seed)
    plan_s = time.perf_counter() - t0
    pst = plan.stats()
    n = circ.n_qubits
    # a side stream, so that the traversal can be captured into a CUDA graph
    # and replayed (one host call per traversal instead of one per pass)
    stream = torch.cuda.Stream() if args.graph else torch.cuda.current_stream()
    torch.cuda.set_stream(stream)
    sp = stream.cuda_stream
    opts = T.run_opts(precision=prec, traversal=trav, use_graph=int(args.graph), subtrees=args.subtrees,
                      tc_mode=args.tc_mode)
    ex = T.Exec(plan, opts, sp)
    probs = torch.empty(1 << n, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup):
        ex.launch(probs.data_ptr(), sp)
    info = ex.finish()

    # timed region: K traversals back to back on the stream; the state and
    # output (2 GiB each at 28 qubits) exceed the 126 MB L2
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            ex.launch(probs.data_ptr(), sp)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    info = ex.finish()
    ms = ev0.elapsed_time(ev1) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    n_inst = pst["n_instances"]
    secs = ms / 1e3
    value = n_inst * world / secs
    amps = float(1 << n)
    peaks, peak_kind = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))

    # live roofline of the pass kernel: events around every pass launch
    ex.set_profiling(True)
    ex.launch(probs.data_ptr(), sp)
    ex.finish()
    pms, pbytes = ex.pass_profile()
    ex.set_profiling(False)
    achieved = float(pbytes.sum() / (pms.sum() / 1e3) / 1e9) if len(pms) else 0.0
    ratio = traffic_from_profile(os.path.join(ROOT, "paper_2508_04880_b300", "csrc", "kernels.cu"))
    per_launch_bytes = float(pbytes.mean()) if len(pbytes) else 0.0
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "peak_kind": peak_kind,
                "traffic": (ratio * per_launch_bytes) if ratio else None,
                "kernel": "pass_kernel<float,5>", "launches_per_step": int(len(pms)),
                "mean_launch_ms": float(pms.mean()) if len(pms) else 0.0,
                "algorithmic_bytes_per_launch": per_launch_bytes}

    # measured FP32 / FP64 FMA peaks of this device (own kernels), with the
    # SM clock sampled meanwhile: the denominators of the SIMT rooflines
    with ClockSampler(local) as clk_alu:
        fp32_tf, fp64_tf = T.tusq_measure_alu_peaks(sp)
    alu_peaks = {"fp32_tflops": fp32_tf, "fp64_tflops": fp64_tf, "clocks": clk_alu.summary(),
                 "how": "FMA chains, 8 CTAs x 256 threads per SM, best of 3 timed launches (CUDA events)"}

    # shot sampling of the output (1e6 shots): integer prefix sum over the
    # 2^n outcomes, then one Philox draw and binary search per shot
    counts = torch.empty(1 << n, dtype=torch.uint64, device="cuda")
    T.tusq_sample(probs.data_ptr(), n, shots, 1, counts.data_ptr(), sp)
    sa, sb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sa.record(stream)
    T.tusq_sample(probs.data_ptr(), n, shots, 2, counts.data_ptr(), sp)
    sb.record(stream)
    torch.cuda.synchronize()
    sample_info = {"shots": shots, "ms": sa.elapsed_time(sb), "counted": int(counts.sum().item())}
    del counts

    # end to end through the C ABI from host buffers, over --e2e-steps jobs
    # (the same circuit with seeds seed, seed+1, ...): plan (ER draws on the
    # device on a private stream, tally, commutation and pruning on the host),
    # compile + upload of the device program, traversal, copy of the
    # distribution to pinned host memory.  Job k+1 is planned and compiled on
    # a host thread while job k traverses; its program upload is queued on
    # the traversal stream, behind job k's work.
    host_out = torch.empty(1 << n, dtype=torch.float64, pin_memory=True)
    dev = torch.cuda.current_device()

    def plan_job(sd):
        torch.cuda.set_device(dev)
        pl = T.plan(circ, shots, sd, device_sampling=True)
        return pl, T.Exec(pl, opts, sp)

    # one untimed warm-up job fills the pipeline; the clock runs over the
    # next jobs_e2e, each planned and compiled during its predecessor
    jobs_e2e = max(1, args.e2e_steps)
    h2d = 0
    e2e_inst = 0
    torch.cuda.synchronize()
    t0 = None
    with ThreadPoolExecutor(max_workers=1) as pool:
        fut = pool.submit(plan_job, seed)
        for k in range(jobs_e2e + 1):
            pl2, ex2 = fut.result()
            if k < jobs_e2e:
                fut = pool.submit(plan_job, seed + k + 1)
            ex2.launch(probs.data_ptr(), sp)
            host_out.copy_(probs, non_blocking=True)
            info2 = ex2.finish()
            torch.cuda.synchronize()
            if k > 0:
                e2e_inst += pl2.stats()["n_instances"]
                h2d = int(info2["program_bytes"])
            del ex2
            if k == 0:
                t0 = time.perf_counter()
    e2e_s = (time.perf_counter() - t0) / jobs_e2e
    total = float(host_out.sum())      # the last job's distribution, checked outside the timed region

    line = {
        "metric": "noisy instances/s", "value": value, "unit": "instances/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": WORKLOAD_DESC[args.workload], "qubits": n, "gates": circ.n_gates,
                   "shots": shots, "instances": n_inst, "traversal": args.traversal, "subtrees": args.subtrees,
                   "tc_mode": ["none", "tf32x3", "bf16x3", "tf32"][args.tc_mode],
                   "l2": "inputs larger than L2 (state and output 2^n x 8 B each)",
                   "parallelism": f"replica x{world}"},
        "gate_amp_updates_per_s": (info["gate_apps"] + info["pauli_apps"]) * amps * world / secs,
        "scratch_equiv_gate_amp_updates_per_s": pst["scratch_gate_apps"] * amps * world / secs,
        "hbm_fraction_whole_step": info["algorithmic_bytes"] / secs / 1e9 / hbm_peak,
        "roofline": roofline,
        "e2e": {"value": e2e_inst / jobs_e2e * world / e2e_s, "unit": "instances/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": int(8 * (1 << n)), "seconds": e2e_s, "plan_seconds": plan_s,
                "jobs": jobs_e2e, "pipelined": "job k+1 planned and compiled on a host thread during job k's traversal; "
                             "one untimed warm-up job before the timed ones",
                "sum_probs": total},
        "gpu_launches": int(info["kernel_launches"]) * args.steps,
        "sample": sample_info,
        "alu_peaks": alu_peaks,
        "run_info": {k: info[k] for k in ("passes", "gate_apps", "pauli_apps", "leaf_passes", "checks",
                                          "restores", "unrecovered", "resets", "max_drift")},
        "plan": {k: pst[k] for k in ("n_raw_unique", "n_commuted_unique", "n_instances",
                                     "dftt_gate_apps", "scratch_gate_apps")},
        "clocks": clk.summary(),
    }
    # the paper's uncompute DFTT (drift check after every uncompute) and the
    # plain GPU form (every instance from |0..0>) beside the headline
    # traversal, each timed over two traversals after one warm-up, with the
    # same kernels
    arms = [("snapshot", T.run_opts(precision=prec, traversal=T.DFTT_SNAPSHOT, tc_mode=args.tc_mode)),
            ("dftt_uncompute", T.run_opts(precision=prec, traversal=T.DFTT, drift_tol=1e-6, tc_mode=args.tc_mode)),
            ("from_scratch", T.run_opts(precision=prec, traversal=T.FROM_SCRATCH, tc_mode=args.tc_mode))]
    if not args.no_compare and rank == 0:
        other = {}
        for name, o in arms:
            e3 = T.Exec(plan, o, sp)
            e3.launch(probs.data_ptr(), sp)
            e3.finish()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(2):
                e3.launch(probs.data_ptr(), sp)
            b.record(stream)
            inf3 = e3.finish()
            t3 = a.elapsed_time(b) / 2
            other[name] = {"ms": t3, "passes": inf3["passes"], "gate_apps": inf3["gate_apps"],
                           "checks": inf3["checks"], "instances_per_s": n_inst / (t3 / 1e3)}
            del e3
        line["traversals"] = other
    if not args.no_error and rank == 0:
        line["error_vs_oracle"] = error_vs_oracle(T, torch, circ, shots, seed, arms, sp)
    if not args.no_served and rank == 0:
        line["served"] = served_subrun(args, T, torch)
    if rank == 0 and not args.no_cpu_baseline:
        inst = plan.instances()[0]
        line["cpu_baseline"] = cpu_baseline(circ, inst)
        line["cpu_baseline_1core"] = cpu_baseline(circ, inst, budget_s=8.0, threads=1)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
