#!/usr/bin/env python
"""Benchmark of the batched arithmetic-circuit hot path on one or more GB300s.

Default workload (32-qubit noise-free QAOA p=1 on a seeded random 3-regular graph,
compiled to a density AC of about 142K nodes, FP32 complex node values): one
step, per GPU, is a variational iteration over 64 parameter vectors --
  bind the angles (upward-pass leaves),
  <C> and its angle gradient for the Max-Cut cost C = sum_edges (1 - Z_i Z_j)/2
    (48 Z-string evidence columns per vector: upward + downward pass),
  10000 chain-rule samples per vector (qubit-by-qubit conditional sampling),
  drawn from the light-cone step AC (step j's density AC holds only the operations
  that can affect qubits <= j; --sampler memo uses the whole density AC).
`value` is samples/s over all GPUs (weak scaling: every GPU runs its own 64
vectors; there is no collective on the data path).

--workload hea16: 16-qubit noisy hardware-efficient ansatz (the largest AC,
about 2.35M nodes): 256 vectors x 16 Z-string terms, <H> + gradient over 192
angles; value = gradient columns/s.

--workload vqe25 / vqe9: the paper's 2D-Ising VQE (5x5 noise-free, one layer; 3x3 with
depolarising noise after every gate, two layers): 256 vectors x 1000 samples + <H> and
its gradient per step; value = samples/s.

--workload qaoa10: the paper's noisy QAOA at 10 qubits, p=2 (random 3-regular graph, 1q depolarising
0.001, 2q depolarising 0.01): 1024 vectors x 1000 samples per step by trajectory sampling on the
TRAJECTORY AC (each sample's noise branches drawn from their probabilities, then its outcome by the
chain rule on |A(x, r)|^2); value = samples/s.

--impl reference times the oracle (plain FP64 C evaluator, or for qaoa10 the state-vector trajectory
sampler) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["qaoa32", "hea16", "vqe25", "vqe9", "qaoa10", "serve", "gibbs_kl"],
                    default="qaoa32")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve: Poisson arrivals per second")
    ap.add_argument("--duration", type=float, default=10.0, help="serve: seconds of arrivals")
    ap.add_argument("--shots", type=int, default=None, help="samples per vector (qaoa32: 10000, vqe: 1000)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", choices=["step", "uppass", "gradpass", "samplepass", "reeval", "serveacs"], default="step",
                    help="uppass: only the upward pass over --columns sampling-prefix columns; gradpass: "
                         "upward + downward pass (gradient) over --columns Z-string columns; samplepass: one "
                         "sampling call over --vectors vectors x --shots shots; serveacs: each AC of the serving "
                         "mix alone (profiling cases)")
    ap.add_argument("--vectors", type=int, default=16, help="samplepass: parameter vectors")
    ap.add_argument("--columns", type=int, default=2048)
    ap.add_argument("--tile", type=int, default=0, help="cap the column tile (0: library default)")
    ap.add_argument("--memo-budget-gb", type=float, default=0.0, help="memoised-slot budget (0: library default)")
    ap.add_argument("--sampler", choices=["memo", "plain", "lightcone"], default="lightcone",
                    help="memo: memoised chain-rule passes (automatic fallback); plain: every node per group; "
                         "lightcone: memoised passes on the light-cone step AC (one AC per sampling step)")
    return ap.parse_args()


# ---------------------------------------------------------------- workloads
def make_workload(name, shots):
    from paper_2103_17226_gb300 import inputs as I
    if name == "qaoa32":
        c = I.workload("qaoa32_3reg_p1_ideal")
        edges = I.random_regular_graph(32, 3, seed=5)
        V = 64
        angles = I.uniform_angles(V, c.n_angles, seed=5)
        # Max-Cut cost C = sum_e (1 - Z_i Z_j) / 2: <C> = |E|/2 - 1/2 sum_e <Z_i Z_j>
        sup = np.zeros((len(edges), 32), dtype=bool)
        for k, (i, j) in enumerate(edges):
            sup[k, i] = sup[k, j] = True
        coef = np.full(len(edges), -0.5)
        return dict(name="qaoa32_3reg_p1_ideal", circuit=c, V=V, angles=angles, sup=sup, coef=coef,
                    shots=10000 if shots is None else shots,
                    seeds=I.vector_seeds(V, 5), unit="samples/s", metric="samples/s (chain-rule sampling, "
                    "with <C> + gradient, of a 32-qubit QAOA density AC)")
    if name in ("vqe25", "vqe9"):
        # the paper's second workload: VQE for the 2D Ising model (Sec. 4.1; Table 7 sizes): 5x5 grid
        # noise-free with one ansatz layer, or 3x3 grid with depolarising noise after every gate and
        # two layers; <H> + gradient of H = sum_<ij> Z_i Z_j + 0.5 sum_i Z_i, and 1000 samples per vector
        wl, (r, cl) = ("vqe_ising_5x5_ideal", (5, 5)) if name == "vqe25" else ("vqe_ising_3x3_noisy", (3, 3))
        c = I.workload(wl)
        V = 256
        sup, coef = I.ising_hamiltonian(r, cl)
        return dict(name=wl, circuit=c, V=V, angles=I.uniform_angles(V, c.n_angles, seed=7), sup=sup, coef=coef,
                    shots=1000 if shots is None else shots, seeds=I.vector_seeds(V, 7), unit="samples/s",
                    metric=f"samples/s (chain-rule sampling, with <H> + gradient, of a {c.n_qubits}-qubit "
                           f"2D-Ising VQE density AC)")
    if name == "qaoa10":
        c = I.workload("qaoa10_3reg_p2")
        V = 1024
        return dict(name="qaoa10_3reg_p2", circuit=c, V=V, angles=I.uniform_angles(V, c.n_angles, seed=2),
                    sup=None, coef=None, shots=1000 if shots is None else shots, seeds=I.vector_seeds(V, 2),
                    unit="samples/s", metric="samples/s (exact trajectory sampling of a 10-qubit noisy QAOA p=2 "
                    "on its TRAJECTORY AC)")
    c = I.workload("hea16_l6")
    V = 256
    sup, coef = I.z_string_hamiltonian(16, 16, seed=3)
    return dict(name="hea16_l6", circuit=c, V=V, angles=I.uniform_angles(V, c.n_angles, seed=3), sup=sup,
                coef=coef, shots=0, seeds=None, unit="gradient columns/s",
                metric="gradient columns/s (<H> + d<H>/dangles of a 16-qubit noisy HEA density AC)")


def hamiltonian_columns(W):
    V, T = W["V"], len(W["coef"])
    ev = np.array([[-2 if b else -1 for b in W["sup"][t]] for _ in range(V) for t in range(T)], dtype=np.int8)
    cv = np.repeat(np.arange(V, dtype=np.int32), T)
    w = np.tile(W["coef"], V).astype(np.float64)
    return ev, cv, w


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                pw.append(float(r[3]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        # samples under load: the upper half by power
        cut = statistics.median(pw)
        loaded = [s for s, p in zip(sm, pw) if p >= cut] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(pw)}


# ---------------------------------------------------------------- oracle timing (CPU baseline / reference arm)
def _oracle_sampler(job):
    """One host process of the all-cores baseline: the oracle's chain-rule samples (vector 0 of the
    workload) for `seconds`, from its own seed range; returns the number drawn."""
    ac_bytes, angles, seed, seconds = job
    from oracle import acref as R
    ref = R.ACRef(ac_bytes)
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        ref.sample(angles, seed + n, 4)
        n += 4
    return n, time.perf_counter() - t0


def host_cpu():
    """The host's CPU as far as the OS tells: architecture and a model string from /proc/cpuinfo."""
    import platform
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu part", "hardware") and not model:
                    model = line.split(":", 1)[1].strip()
    except OSError:
        pass
    return f"{platform.machine()} {model}".strip()


def oracle_all_cores(W, ac_bytes, seconds=6.0):
    """The oracle as it stands, one process per host core (a spawn-started pool: no process is
    forked from one that holds a CUDA context); aggregate chain-rule samples per second."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    a = W["angles"][0]
    jobs = [(ac_bytes, a, int(W["seeds"][0]) + (i << 32), seconds) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as pool:
        res = pool.map(_oracle_sampler, jobs)
    return sum(n for n, _ in res) / max(t for _, t in res), cores


def oracle_errors(W, ref, value, grad, first_samples, gpu):
    """The GPU's results for vector 0 against the oracle's (computed in the CPU-baseline leg from
    the same calls it times): |<H>| and gradient errors, p0/P on random prefixes, and sample indices
    (a mismatch is tolerated only where |u P - p0| <= 1e-5 P, the FP32 tie margin)."""
    from oracle import quantum as Q
    n = W["circuit"].n_qubits
    a = W["angles"][0]
    out = {"vs": "FP64 AC oracle (oracle/acref.c) on vector 0 of the workload",
           "value_abs_err": abs(gpu["value0"] - value), "grad_max_abs_err": float(np.abs(gpu["grad0"] - grad).max()),
           "value_scale": float(np.abs(W["coef"]).sum())}
    if gpu.get("prefix_ev") is not None:
        rel = []
        for ev, (gP, gp0) in zip(gpu["prefix_ev"], gpu["prefix_vals"]):
            P = ref.up(a, ev).real
            ev0 = list(ev)
            ev0[ev0.index(-1)] = 0
            p0 = ref.up(a, ev0).real
            rel.append(abs(gp0 / gP - p0 / P) / (p0 / P))
        out["p0_over_P_max_rel_err"] = max(rel)
        out["prefixes_checked"] = len(rel)
    if first_samples is not None:
        got = gpu["bits0"][:len(first_samples)].astype(np.uint64)
        seed = int(W["seeds"][0])
        mis, beyond = 0, 0
        for s in np.nonzero(got != first_samples)[0]:
            mis += 1
            g, r = int(got[s]), int(first_samples[s])
            j = next(k for k in range(n) if ((g ^ r) >> (n - 1 - k)) & 1)
            pre = [(r >> (n - 1 - k)) & 1 for k in range(j)]
            ev = pre + [-1] * (n - j)
            P = ref.up(a, ev).real
            ev[j] = 0
            p0 = ref.up(a, ev).real
            beyond += abs(Q.sample_uniform(seed, int(s), j, n) * P - p0) > 1e-5 * P
        out.update(samples_checked=len(first_samples), sample_mismatches=mis, mismatches_beyond_tie_margin=beyond)
    return out


def oracle_rate(W, ac_bytes, budget_s=12.0, all_cores=True, gpu=None):
    """Time the oracle as it stands (acref.c, FP64, one host core) on a bounded sample of
    the workload: the per-vector gradient columns, then samples until the budget.  With the
    GPU's results for vector 0 (`gpu`), the same oracle outputs also give the error report."""
    from oracle import acref as R
    ref = R.ACRef(ac_bytes)
    a = W["angles"][0]
    t0 = time.perf_counter()
    value, grad = 0.0, np.zeros(W["circuit"].n_angles)
    for t, (s, cf) in enumerate(zip(W["sup"], W["coef"])):
        v_, g_ = ref.gradient(a, [-2 if b else -1 for b in s], cf)
        value += v_
        grad += g_
    t_grad = time.perf_counter() - t0
    T = len(W["coef"])
    if W["shots"] == 0:
        res = dict(value=T / t_grad, unit=W["unit"], cores=1, kind="oracle",
                   sample=f"1 vector x {T} Z-string columns (up + down pass each) on acref.c, FP64, one core")
        if gpu is not None:
            res["errors"] = oracle_errors(W, ref, value, grad, None, gpu)
        return res
    t1 = time.perf_counter()
    first = ref.sample(a, int(W["seeds"][0]), 64)  # the GPU's first 64 samples of vector 0
    n_s = 64
    while time.perf_counter() - t1 < max(1.0, budget_s - t_grad):
        ref.sample(a, int(W["seeds"][0]) + n_s, 4)
        n_s += 4
    t_s = (time.perf_counter() - t1) / n_s
    errors = oracle_errors(W, ref, value, grad, first, gpu) if gpu is not None else None
    per_vec = t_grad + W["shots"] * t_s
    one_core = W["shots"] / per_vec
    if not all_cores:
        res = dict(value=one_core, unit=W["unit"], cores=1, kind="oracle",
                   sample=(f"1 vector: {T} gradient columns ({t_grad:.2f} s) + {n_s} chain-rule samples "
                           f"({t_s * 1e3:.1f} ms each) on acref.c, FP64, one core; rate = {W['shots']} samples / "
                           f"(gradient + {W['shots']} x per-sample time)"))
    else:
        agg, cores = oracle_all_cores(W, ac_bytes)
        # all cores: samples at the aggregate rate, the gradient columns split over the cores
        per_vec_all = t_grad / cores + W["shots"] / agg
        res = dict(value=W["shots"] / per_vec_all, unit=W["unit"], cores=cores, kind="oracle",
                   sample=(f"1 vector: {T} gradient columns ({t_grad:.2f} s on one core, counted / {cores}) + "
                           f"chain-rule samples on {cores} spawned processes ({agg:.1f} samples/s together) on "
                           f"acref.c, FP64; one core alone: {one_core:.2f} samples/s "
                           f"({t_s * 1e3:.1f} ms per sample); host CPU: {host_cpu()}"))
    if errors is not None:
        res["errors"] = errors
    return res


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native as N
    W = make_workload(args.workload, args.shots)
    b = N.compile(W["circuit"], N.QKC_AC_DENSITY)
    rates = []
    for i in range(args.warmup + args.steps):
        r = oracle_rate(W, b, budget_s=8.0)
        if i >= args.warmup:
            rates.append(r)
    val = statistics.median([r["value"] for r in rates])
    line = {"impl": "reference", "metric": W["metric"], "value": val, "unit": W["unit"], "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": W["name"]},
            "cpu_baseline": {"value": val, "unit": W["unit"], "cores": rates[-1]["cores"], "kind": "oracle",
                             "sample": rates[-1]["sample"]},
            "e2e": {"value": val, "unit": W["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def gpu_results(W, ac, step, dev):
    """Vector 0's GPU results at the workload's base angles, for the error report: one more step
    (outside the timed regions), and p0 and P of 16 random prefixes by the FP32 upward pass."""
    import torch
    from paper_2103_17226_gb300 import inputs as I, native as N
    val, grad, bits = step(0)
    out = {"value0": float(val[0]), "grad0": grad[0].cpu().numpy(),
           "bits0": bits[0, :64].cpu().numpy() if bits is not None else None}
    if W["shots"]:
        n = W["circuit"].n_qubits
        rng = I.SplitMix(99)
        evs = []
        for _ in range(16):
            L = 1 + rng.randint(n - 1)
            pre = [rng.randint(2) for _ in range(L)]
            evs.append(pre + [-1] * (n - L))
        cols = [e for ev in evs for e in (ev, [x if i != ev.index(-1) else 0 for i, x in enumerate(ev)])]
        r = N.evaluate(ac, torch.zeros(len(cols), dtype=torch.int32, device=dev),
                       torch.tensor(np.array(cols, dtype=np.int8), device=dev)).cpu().numpy()
        out["prefix_ev"] = evs
        out["prefix_vals"] = [(r[2 * k, 0], r[2 * k + 1, 0]) for k in range(len(evs))]
    return out


# ---------------------------------------------------------------- trajectory sampling (qaoa10)
def _traj_oracle_job(job):
    circuit, angles, seed, seconds = job
    from oracle import trajectory as T
    n, t0 = 0, time.perf_counter()
    while time.perf_counter() - t0 < seconds or n == 0:
        T.trajectory_samples(circuit, angles, seed + n, 8)
        n += 8
    return n, time.perf_counter() - t0


def oracle_trajectory_rate(W, seconds=6.0, gpu=None):
    """The trajectory oracle as it stands (oracle/trajectory.py: a state-vector run per distinct
    trajectory, chain rule on |A(x, r)|^2), one spawn-started process per host core, vectors of the
    workload in turn; with the GPU's first samples of vector 0, also the error report."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    from oracle import quantum as Q, trajectory as T
    cores = os.cpu_count() or 1
    c = W["circuit"]
    jobs = [(c, W["angles"][i % W["V"]], int(W["seeds"][i % W["V"]]) + (i << 32), seconds) for i in range(cores)]
    with ProcessPoolExecutor(cores, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_traj_oracle_job, jobs))
    rate = sum(n for n, _ in res) / max(t_ for _, t_ in res)
    out = dict(value=rate, unit=W["unit"], cores=cores, kind="oracle",
               sample=(f"state-vector trajectory sampler (oracle/trajectory.py, FP64) on {cores} spawned processes, "
                       f"{seconds:.0f} s each, batches of 8 samples of vectors 0..{cores - 1}; host CPU: {host_cpu()}"))
    if gpu is not None:
        n, seed, a = c.n_qubits, int(W["seeds"][0]), W["angles"][0]
        want = T.trajectory_samples(c, a, seed, len(gpu["bits0"]))
        got = gpu["bits0"].astype(np.uint64)
        mis, beyond = 0, 0
        for s_ in np.nonzero(got != want)[0]:
            mis += 1
            r = T.draw_trajectory(c, seed, int(s_))
            prob = (np.abs(Q.statevector(c, a, r)) ** 2).reshape((2,) * n)
            g, w = int(got[s_]), int(want[s_])
            j = next(k for k in range(n) if ((g ^ w) >> (n - 1 - k)) & 1)
            pre = tuple((w >> (n - 1 - k)) & 1 for k in range(j))
            P, p0 = float(prob[pre].sum()), float(prob[pre + (0,)].sum())
            beyond += abs(Q.sample_uniform(seed, int(s_), j, n) * P - p0) > 1e-5 * P
        out["errors"] = {"vs": "FP64 trajectory oracle (oracle/trajectory.py) on vector 0 of the workload",
                         "samples_checked": len(want), "sample_mismatches": mis, "mismatches_beyond_tie_margin": beyond}
    return out


def run_trajectory(args):
    """Config 2: exact batched sampling of the 10-qubit noisy QAOA p=2 through noise trajectories."""
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native as N
    W = make_workload("qaoa10", args.shots)
    V, S = W["V"], W["shots"]
    ac = N.load_ac(N.Context(local), N.compile(W["circuit"], N.QKC_AC_TRAJECTORY), precision=32)
    if args.tile:
        N.set_tile_limit(ac, args.tile)
    info = ac.info()
    angle_sets = [W["angles"] + 0.01 * k for k in range(4)]
    d_angles = [torch.tensor(a, device=dev) for a in angle_sets]
    d_seeds = torch.tensor(W["seeds"].astype(np.int64), device=dev)
    d_shots = torch.full((V,), S, dtype=torch.int32, device=dev)
    d_bits = torch.empty((V, S), dtype=torch.int64, device=dev)

    def step(k, angles=None, seeds=None, shots=None):
        N.set_params(ac, angles if angles is not None else d_angles[k % 4])
        return N.sample(ac, seeds if seeds is not None else d_seeds, shots if shots is not None else d_shots, S,
                        out=d_bits, total_shots=V * S)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for k in range(args.warmup):
        step(k)
    barrier()
    N.stats_enable(ac, True, 1 << 20)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(k)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    stats = N.get_stats(ac)
    N.stats_enable(ac, False, 0)
    N.check_status(ac)
    ms_max = max_over_ranks(ms, world, dev)
    value = whole_job_rate(V * S, world, args.steps, ms_max / 1e3)
    h_angles = [torch.tensor(a).pin_memory() for a in angle_sets]
    h_seeds = torch.tensor(W["seeds"].astype(np.int64)).pin_memory()
    h_shots = torch.full((V,), S, dtype=torch.int32).pin_memory()
    h_bits = torch.empty((V, S), dtype=torch.int64).pin_memory()

    def e2e_step(k):
        bits = step(k, h_angles[k % 4].to(dev, non_blocking=True), h_seeds.to(dev, non_blocking=True),
                    h_shots.to(dev, non_blocking=True))
        h_bits.copy_(bits, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_step(0)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    barrier()
    e2e_value = whole_job_rate(V * S, world, args.steps, max_over_ranks(time.perf_counter() - t0, world, dev))
    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except OSError:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        ach = stats["up_bytes"] / (stats["up_ms"] * 1e6) if stats["up_ms"] > 0 else None
        line = {
            "metric": W["metric"], "value": value, "unit": W["unit"], "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": W["name"], "qubits": W["circuit"].n_qubits, "vectors_per_gpu": V, "shots": S,
                       "ac_kind": "TRAJECTORY", "ac_nodes": info["n_nodes"], "ac_edges": info["n_edges"],
                       "ac_levels": info["n_levels"], "noise_variables": info["n_vars"] - W["circuit"].n_qubits,
                       "precision": "complex FP32 nodes, power-of-two scale per (level, column); FP64 decisions",
                       "l2": "inputs larger than L2: each column tile of the AC's values is tens of GB"},
            "roofline": {"bound": "hbm", "kernel": "up_level_f32 (upward pass per group column)", "achieved": ach,
                         "peak": hbm, "unit": "GB/s", "frac": (ach / hbm) if ach else None,
                         "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                         "bytes_per_launch": stats["up_bytes"] / max(1, stats["up_passes"]),
                         "launch": "one event-timed upward pass over one column tile", "traffic": None},
            "gpu_launches": stats["launches"],
            "edge_evals_per_s": (stats["up_edges"]) * world / (ms_max / 1e3),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": W["unit"], "h2d_bytes_per_step": h_angles[0].numel() * 8 + V * 12,
                    "d2h_bytes_per_step": V * S * 8},
        }
        if not args.no_cpu_baseline:
            step(0)
            torch.cuda.synchronize()
            cb = oracle_trajectory_rate(W, gpu={"bits0": d_bits[0, :64].cpu().numpy()})
            line["errors"] = cb.pop("errors", None)
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------- multi-rank aggregation
def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's figure (timing is the max over ranks; no data-path collective)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_step: int, world: int, steps: int, seconds: float) -> float:
    """Weak scaling: every rank processes its own units; the job rate is all units over the max time."""
    return units_per_step * world * steps / seconds


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native as N

    W = make_workload(args.workload, args.shots)
    ac_bytes = N.compile(W["circuit"], N.QKC_AC_DENSITY)
    ctx = N.Context(local)
    ac = N.load_ac(ctx, ac_bytes, precision=32)
    N.set_sampler(ac, 0 if args.sampler == "plain" else 1, int(args.memo_budget_gb * 2 ** 30))
    V, S = W["V"], W["shots"]
    ev, cv, w = hamiltonian_columns(W)
    n_cols = len(cv)
    # the AC that samples: the density AC itself, or the light-cone step AC beside it
    sac = ac
    if args.sampler == "lightcone" and S:
        sac = N.load_ac(ctx, N.compile(W["circuit"], N.QKC_AC_DENSITY_STEPS), precision=32)
        N.set_sampler(sac, 1, int(args.memo_budget_gb * 2 ** 30))
    if args.tile:
        N.set_tile_limit(ac, args.tile)
        N.set_tile_limit(sac, args.tile)
    N.reserve(ac, V, n_cols if sac is not ac else max(n_cols, V * max(S, 1)))
    info = ac.info()

    # device inputs (kernel-only timing) -- a few angle sets, rotated per step
    angle_sets = [W["angles"] + 0.01 * k for k in range(4)]
    d_angles = [torch.tensor(a, device=dev) for a in angle_sets]
    d_ev, d_cv, d_w = torch.tensor(ev, device=dev), torch.tensor(cv, device=dev), torch.tensor(w, device=dev)
    d_seeds = torch.tensor(W["seeds"].astype(np.int64), device=dev) if S else None
    d_shots = torch.full((V,), S, dtype=torch.int32, device=dev) if S else None
    d_bits = torch.empty((V, S), dtype=torch.int64, device=dev) if S else None
    d_val = torch.empty(V, dtype=torch.float64, device=dev)
    d_grad = torch.empty((V, W["circuit"].n_angles), dtype=torch.float64, device=dev)

    def step(k, angles=None, ev_t=None, cv_t=None, w_t=None, seeds=None, shots=None):
        a_k = angles if angles is not None else d_angles[k % 4]
        N.set_params(ac, a_k)
        if sac is not ac:
            N.set_params(sac, a_k)
        val, grad = N.gradient(ac, cv_t if cv_t is not None else d_cv, ev_t if ev_t is not None else d_ev,
                               w_t if w_t is not None else d_w, V)
        bits = None
        if S:
            bits = N.sample(sac, seeds if seeds is not None else d_seeds, shots if shots is not None else d_shots,
                            S, out=d_bits)
        return val, grad, bits

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    for k in range(args.warmup):
        step(k)
    barrier()
    acs = [ac] if sac is ac else [ac, sac]
    for x in acs:
        N.stats_enable(x, True, 1 << 20)
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(args.steps):
        step(k)
    e1.record()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    stats = N.get_stats(ac)
    if sac is not ac:  # both ACs' launches and passes
        st2 = N.get_stats(sac)
        stats = {k: stats[k] + st2[k] for k in stats}
    for x in acs:
        N.stats_enable(x, False, 0)
    ms_max = max_over_ranks(ms, world, dev)
    units_per_step = V * S if S else n_cols
    value = whole_job_rate(units_per_step, world, args.steps, ms_max / 1e3)

    # ---- end to end through the public API: pinned host inputs in, results out, every step
    h_angles = [torch.tensor(a).pin_memory() for a in angle_sets]
    h_ev, h_cv, h_w = torch.tensor(ev).pin_memory(), torch.tensor(cv).pin_memory(), torch.tensor(w).pin_memory()
    h_seeds = torch.tensor(W["seeds"].astype(np.int64)).pin_memory() if S else None
    h_shots = torch.full((V,), S, dtype=torch.int32).pin_memory() if S else None
    h_bits = torch.empty((V, S), dtype=torch.int64).pin_memory() if S else None
    h_val = torch.empty(V, dtype=torch.float64).pin_memory()
    h_grad = torch.empty((V, W["circuit"].n_angles), dtype=torch.float64).pin_memory()
    h2d = (h_angles[0].numel() * 8 + h_ev.numel() + h_cv.numel() * 4 + h_w.numel() * 8 +
           (h_seeds.numel() * 8 + h_shots.numel() * 4 if S else 0))
    d2h = h_val.numel() * 8 + h_grad.numel() * 8 + (h_bits.numel() * 8 if S else 0)

    def e2e_step(k):
        a = h_angles[k % 4].to(dev, non_blocking=True)
        e_ = h_ev.to(dev, non_blocking=True)
        c_ = h_cv.to(dev, non_blocking=True)
        w_ = h_w.to(dev, non_blocking=True)
        sd = h_seeds.to(dev, non_blocking=True) if S else None
        sh = h_shots.to(dev, non_blocking=True) if S else None
        val, grad, bits = step(k, a, e_, c_, w_, sd, sh)
        h_val.copy_(val, non_blocking=True)
        h_grad.copy_(grad, non_blocking=True)
        if S:
            h_bits.copy_(bits, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    for k in range(min(args.warmup, 2)):
        e2e_step(k)
    barrier()
    t0 = time.perf_counter()
    for k in range(args.steps):
        e2e_step(k)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_value = whole_job_rate(units_per_step, world, args.steps, max_over_ranks(e2e_s, world, dev))

    if rank == 0:
        peaks = {}
        try:
            with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
                peaks = json.load(f)
        except OSError:
            pass
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
        def gbs(kind):
            return stats[kind + "_bytes"] / (stats[kind + "_ms"] * 1e6) if stats[kind + "_ms"] > 0 else None

        # per-kind (algorithmic bytes, event ms, timed chains): the memoised pass splits into its tiers
        kinds = {"up": (stats["up_bytes"], stats["up_ms"], stats["up_passes"]),
                 "down": (stats["down_bytes"], stats["down_ms"], stats["down_passes"]),
                 "memo_b": (stats["memo_bytes"] - stats["memo_a_bytes"], stats["memo_ms"] - stats["memo_a_ms"],
                            stats["memo_passes"]),
                 "memo_a": (stats["memo_a_bytes"], stats["memo_a_ms"], stats["memo_passes"])}
        names = {"up": "up_level_f32 (upward pass)", "down": "down_light_f32/down_heavy_f32 (downward pass)",
                 "memo_b": "memoB_level_f32 (tier B of the memoised sampling pass: per group column; with its "
                           "scale and group-key kernels)",
                 "memo_a": "memoA_level<float2> (tier A of the memoised sampling pass: per (vector, key) slot)"}
        dom = max(kinds, key=lambda k: kinds[k][1])
        ach = kinds[dom][0] / (kinds[dom][1] * 1e6) if kinds[dom][1] > 0 else None
        per_launch_bytes = kinds[dom][0] / max(1, kinds[dom][2])
        up_gbs, dn_gbs, memo_gbs = gbs("up"), gbs("down"), gbs("memo")
        # child references the level kernels actually evaluated (tier-A slots, tier-B group columns,
        # upward and downward passes of the gradient columns)
        edge_evals = stats["up_edges"] + stats["down_edges"] + stats["memo_edges"]
        line = {
            "metric": W["metric"], "value": value, "unit": W["unit"], "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": W["name"], "qubits": W["circuit"].n_qubits, "vectors_per_gpu": V, "shots": S,
                       "hamiltonian_terms": len(W["coef"]), "ac_nodes": info["n_nodes"],
                       "ac_edges": info["n_edges"], "ac_levels": info["n_levels"],
                       "precision": "complex FP32 nodes, power-of-two scale per (level, column); FP64 decisions",
                       "sampler": args.sampler,
                       "l2": "inputs larger than L2: the sampling AC's value tile holds "
                             f"{sac.info()['reserved_columns']} group columns of its tier-B nodes (GBs) and "
                             "the tier-A slots of 64 vectors up to key width 12 are tens of GB"},
            "roofline": {"bound": "hbm", "kernel": names[dom], "achieved": ach, "peak": hbm, "unit": "GB/s",
                         "frac": (ach / hbm) if ach else None, "peak_source": peak_src,
                         "bytes_per_launch": per_launch_bytes, "launch": "one event-timed chain (all tiles of "
                         "one sampling step for the memoised tiers, one column tile for up/down)",
                         "traffic": None,
                         "up_pass_gbs": up_gbs, "down_pass_gbs": dn_gbs, "memo_pass_gbs": memo_gbs,
                         "memo_tier_a_gbs": (stats["memo_a_bytes"] / (stats["memo_a_ms"] * 1e6)
                                             if stats["memo_a_ms"] > 0 else None),
                         "memo_tier_b_gbs": ((stats["memo_bytes"] - stats["memo_a_bytes"])
                                             / ((stats["memo_ms"] - stats["memo_a_ms"]) * 1e6)
                                             if stats["memo_ms"] > stats["memo_a_ms"] else None),
                         "time_ms": {k: stats[k + "_ms"] for k in ("up", "down", "memo", "memo_a")}},
            "gpu_launches": stats["launches"],
            "edge_evals_per_s": edge_evals * world / (ms_max / 1e3),
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": W["unit"], "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        }
        if not args.no_cpu_baseline:
            cb = oracle_rate(W, ac_bytes, gpu=gpu_results(W, ac, step, dev))
            line["errors"] = cb.pop("errors", None)
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_gradpass(args):
    """Small profiling case: qkc_gradient (upward + downward pass) over `--columns`
    Z-string columns of the workload's Hamiltonian."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native as N
    W = make_workload(args.workload, args.shots)
    ac = N.load_ac(N.Context(0), N.compile(W["circuit"], N.QKC_AC_DENSITY), precision=32)
    ev, cv, w = hamiltonian_columns(W)
    reps = (args.columns + len(cv) - 1) // len(cv)
    ev, cv, w = np.tile(ev, (reps, 1))[:args.columns], np.tile(cv, reps)[:args.columns], np.tile(w, reps)[:args.columns]
    d_ev, d_cv, d_w = (torch.tensor(x, device="cuda") for x in (ev, cv, w))
    N.set_params(ac, torch.tensor(W["angles"], device="cuda"))
    N.reserve(ac, W["V"], args.columns)
    for _ in range(args.warmup + 1):
        N.gradient(ac, d_cv, d_ev, d_w, W["V"])
    torch.cuda.synchronize()
    N.stats_enable(ac, True, 1 << 12)
    for _ in range(args.steps):
        N.gradient(ac, d_cv, d_ev, d_w, W["V"])
    st = N.get_stats(ac)
    print(json.dumps({"mode": "gradpass", "workload": W["name"], "columns": args.columns,
                      "up_gbs": st["up_bytes"] / (st["up_ms"] * 1e6), "down_gbs": st["down_bytes"] / (st["down_ms"] * 1e6),
                      "down_ms_per_pass": st["down_ms"] / max(1, st["down_passes"]), "launches": st["launches"]}),
          flush=True)


def run_samplepass(args):
    """Small profiling case: one qkc_sample call (the --sampler's AC and passes) over --vectors
    vectors x --shots shots of the workload, with the tier-A / tier-B rates of its memoised passes."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import inputs as I, native as N
    W = make_workload(args.workload, args.shots)
    c, V, S = W["circuit"], args.vectors, W["shots"]
    kind = N.QKC_AC_DENSITY_STEPS if args.sampler == "lightcone" else N.QKC_AC_DENSITY
    ac = N.load_ac(N.Context(0), N.compile(c, kind), precision=32)
    if args.tile:
        N.set_tile_limit(ac, args.tile)
    N.set_sampler(ac, 0 if args.sampler == "plain" else 2, int(args.memo_budget_gb * 2 ** 30))
    N.set_params(ac, torch.tensor(I.uniform_angles(V, c.n_angles, seed=5), device="cuda"))
    seeds = torch.tensor(I.vector_seeds(V, 11).astype(np.int64), device="cuda")
    shots = torch.full((V,), S, dtype=torch.int32, device="cuda")
    N.stats_enable(ac, True, 1 << 16)
    N.sample(ac, seeds, shots, S, total_shots=V * S)
    torch.cuda.synchronize()
    st = N.get_stats(ac)
    b_ms = st["memo_ms"] - st["memo_a_ms"]
    print(json.dumps({"mode": "samplepass", "workload": W["name"], "sampler": args.sampler, "vectors": V, "shots": S,
                      "launches": st["launches"], "memo_ms": st["memo_ms"], "memo_a_ms": st["memo_a_ms"],
                      "tier_a_gbs": st["memo_a_bytes"] / (st["memo_a_ms"] * 1e6) if st["memo_a_ms"] > 0 else None,
                      "tier_b_gbs": (st["memo_bytes"] - st["memo_a_bytes"]) / (b_ms * 1e6) if b_ms > 0 else None,
                      "up_ms": st["up_ms"]}), flush=True)


def run_reeval(args):
    """Incremental re-evaluation (qkc_reevaluate) against a full upward pass: the workload's
    Z-string columns for 64 vectors are evaluated once; then every angle slot in turn is moved
    (all vectors) and re-evaluated incrementally. Reports the time per slot update against a
    full qkc_evaluate of the same columns, and checks the values against a full evaluation."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import native as N
    W = make_workload(args.workload, args.shots)
    c = W["circuit"]
    V = min(64, W["V"])
    ev, cv, w = hamiltonian_columns(dict(W, V=V))
    ctx = N.Context(0)
    ac = N.load_ac(ctx, N.compile(c, N.QKC_AC_DENSITY), precision=32)
    N.reserve(ac, V, len(cv))
    angles = W["angles"][:V].copy()
    d_ev, d_cv = torch.tensor(ev, device="cuda"), torch.tensor(cv, device="cuda")
    N.set_params(ac, torch.tensor(angles, device="cuda"))
    for _ in range(3):
        N.evaluate(ac, d_cv, d_ev)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(5):
        full = N.evaluate(ac, d_cv, d_ev)
    e1.record()
    torch.cuda.synchronize()
    t_full = e0.elapsed_time(e1) / 5
    slots = list(range(c.n_angles))
    d_angles = []
    for k in slots:  # angles after moving slots 0..k in turn
        angles[:, k] += 0.25
        d_angles.append(torch.tensor(angles, device="cuda"))
    N.reevaluate(ac, 0, d_cv, len(cv))  # same angles as evaluated: builds slot 0's cone outside the timing
    for k in slots[1:]:
        N.reevaluate(ac, k, d_cv, len(cv))  # every slot's dirty cone, built once
    torch.cuda.synchronize()
    N.set_params(ac, torch.tensor(W["angles"][:V], device="cuda"))
    N.evaluate(ac, d_cv, d_ev)
    torch.cuda.synchronize()
    e0.record()
    for k in slots:
        N.set_params(ac, d_angles[k])
        out = N.reevaluate(ac, k, d_cv, len(cv))
    e1.record()
    torch.cuda.synchronize()
    t_inc = e0.elapsed_time(e1) / len(slots)
    ref = N.evaluate(ac, d_cv, d_ev)
    err = float((out - ref).abs().max())
    print(json.dumps({"mode": "reeval", "workload": W["name"], "columns": len(cv), "angle_slots": len(slots),
                      "full_evaluate_ms": t_full, "reevaluate_ms_per_slot": t_inc, "speedup": t_full / t_inc,
                      "max_abs_diff_vs_full": err}), flush=True)


def run_uppass(args):
    """Small profiling case: the upward pass alone over `--columns` columns whose
    evidence fixes a random prefix of the qubits (the sampler's column shape)."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import inputs as I, native as N
    W = make_workload(args.workload, args.shots)
    c = W["circuit"]
    n = c.n_qubits
    ac = N.load_ac(N.Context(0), N.compile(c, N.QKC_AC_DENSITY), precision=32)
    rng = I.SplitMix(17)
    ev = np.full((args.columns, n), -1, dtype=np.int8)
    for k in range(args.columns):
        L = rng.randint(n)
        ev[k, :L] = [rng.randint(2) for _ in range(L)]
    cv = np.array([k % W["V"] for k in range(args.columns)], dtype=np.int32)
    d_ev, d_cv = torch.tensor(ev, device="cuda"), torch.tensor(cv, device="cuda")
    N.set_params(ac, torch.tensor(W["angles"], device="cuda"))
    N.reserve(ac, W["V"], args.columns)
    out = N.evaluate(ac, d_cv, d_ev)
    for _ in range(args.warmup):
        N.evaluate(ac, d_cv, d_ev, out=out)
    torch.cuda.synchronize()
    N.stats_enable(ac, True, 1 << 12)
    for _ in range(args.steps):
        N.evaluate(ac, d_cv, d_ev, out=out)
    st = N.get_stats(ac)
    print(json.dumps({"mode": "uppass", "workload": W["name"], "columns": args.columns,
                      "up_ms_per_pass": st["up_ms"] / max(1, st["up_passes"]),
                      "up_gbs": st["up_bytes"] / (st["up_ms"] * 1e6), "launches": st["launches"]}), flush=True)


def serve_circuits():
    """The serving mix: noisy QAOA p=1 on 8, 12, 16 and 20 qubits (two random 3-regular graphs at 12, 16 and
    20; density ACs) and p=2 on 8 qubits (TRAJECTORY AC), noise as config 2."""
    from paper_2103_17226_gb300 import inputs as I, native as N
    circs, kinds = {}, {}
    for n in (8, 12, 16, 20):
        for g in ((0,) if n == 8 else (0, 1)):
            k = f"qaoa{n}_p1_g{g}"
            circs[k] = I.qaoa_maxcut(n, I.random_regular_graph(n, 3, seed=40 + n + 100 * g), 1, I.NOISE_CFG2, name=k)
            kinds[k] = N.QKC_AC_DENSITY
    circs["qaoa8_p2"] = I.qaoa_maxcut(8, I.random_regular_graph(8, 3, seed=48), 2, I.NOISE_CFG2, name="qaoa8_p2")
    kinds["qaoa8_p2"] = N.QKC_AC_TRAJECTORY
    return circs, kinds


def run_serveacs(args):
    """Profiling case for the serving mix: each AC alone, one sampling call of 32 requests x 2150 shots (the
    mix's mean) as the serving bench makes them (FP32, 8192-column tiles; light-cone step ACs for p=1) but with a
    2 GB memo budget, timed with CUDA events over three calls; one JSON line per AC with its samples/s and its
    memoised tiers' (or per-group passes') algorithmic GB/s."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import inputs as I, native as N
    circs, kinds = serve_circuits()
    ctx = N.Context(0)
    dev = torch.device("cuda", 0)
    V, S = 32, 2150
    for k, c in circs.items():
        kind = N.QKC_AC_DENSITY_STEPS if kinds[k] == N.QKC_AC_DENSITY else kinds[k]
        b = N.compile(c, kind)
        ac = N.load_ac(ctx, b, precision=32)
        N.set_tile_limit(ac, 8192)
        N.set_sampler(ac, 1, 2 << 30)
        N.set_params(ac, torch.tensor(I.uniform_angles(V, c.n_angles, seed=1), device=dev))
        seeds = torch.tensor(I.vector_seeds(V, 3).astype(np.int64), device=dev)
        shots = torch.full((V,), S, dtype=torch.int32, device=dev)
        N.sample(ac, seeds, shots, S)  # warm-up: scratch, memoised metadata, graphs
        torch.cuda.synchronize()
        N.stats_enable(ac, True, 1 << 16)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            N.sample(ac, seeds, shots, S)
        e1.record()
        torch.cuda.synchronize()
        st = N.get_stats(ac)
        ms = e0.elapsed_time(e1) / 3
        b_ms = st["memo_ms"] - st["memo_a_ms"]
        print(json.dumps({"mode": "serveacs", "ac": k, "kind": "steps" if kind == N.QKC_AC_DENSITY_STEPS else "trajectory",
                          "nodes": N.header(b)["n_nodes"], "vectors": V, "shots": S, "ms_per_call": ms,
                          "samples_per_s": V * S / ms * 1e3,
                          "tier_a_gbs": st["memo_a_bytes"] / (st["memo_a_ms"] * 1e6) if st["memo_a_ms"] > 0 else None,
                          "tier_b_gbs": (st["memo_bytes"] - st["memo_a_bytes"]) / (b_ms * 1e6) if b_ms > 0 else None,
                          "up_gbs": st["up_bytes"] / (st["up_ms"] * 1e6) if st["up_ms"] > 0 else None}), flush=True)
        del ac
        torch.cuda.empty_cache()


def run_serve(args):
    """Serving: Poisson arrivals over 8 resident noisy-QAOA ACs (1q depolarising 0.001, 2q depolarising 0.01 after
    every gate): p=1 on 8, 12, 16 and 20 qubits (two random 3-regular graphs at 12, 16 and 20) as density ACs, and
    p=2 on 8 qubits as a TRAJECTORY AC (p=2 at 12 qubits compiles to a 5.4M-node TRAJECTORY AC, about 0.3 s of GPU
    per 2000-shot request, and at 16 and 20 qubits to elimination widths 24 and 32: out of a serving budget); one
    parameter vector and log-uniform shots in [100, 10000] per request.  Continuous batching (FP32, 2 lanes per
    AC, light-cone step ACs for p=1 with --sampler lightcone, an 8 GB memo budget per lane unless --memo-budget-gb
    says otherwise) against the FP64 one-request-at-a-time path on the
    same stream.  Both serve every admitted request to completion (arrivals for --duration seconds, at most six
    times that in all); p50/p99 are over every admitted request."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import inputs as I, native as N
    from paper_2103_17226_gb300.serve import Server, poisson_requests
    circs, kinds = serve_circuits()
    acs = {k: N.compile(c, kinds[k]) for k, c in circs.items()}
    # ours samples p=1 from the light-cone step ACs (--sampler lightcone, the default) or the density ACs
    ours = {k: (N.compile(c, N.QKC_AC_DENSITY_STEPS) if args.sampler == "lightcone" and kinds[k] == N.QKC_AC_DENSITY
                else acs[k]) for k, c in circs.items()}
    reqs = poisson_requests(list(acs), {k: c.n_angles for k, c in circs.items()}, args.rate, args.duration, seed=4)
    ctx = N.Context(0)
    cap = args.duration * 6
    srv = Server(ctx, ours, precision=32, lanes=2, max_batch=32, max_shots=10000, tile_columns=8192,
                 memoised=args.sampler != "plain",
                 memo_budget_bytes=int(args.memo_budget_gb * 2 ** 30) if args.memo_budget_gb > 0 else 8 << 30)
    res, st = srv.run(reqs, time_limit=cap)
    del srv
    torch.cuda.empty_cache()
    base = Server(ctx, acs, precision=64, lanes=1, max_batch=1, max_shots=10000, tile_columns=4096, serial=True,
                  memoised=False)
    res_b, st_b = base.run(reqs, time_limit=cap)
    same = sum(1 for rid, r in res.items() if rid in res_b and np.array_equal(r.bits, res_b[rid].bits))
    both = sum(1 for rid in res if rid in res_b)
    print(json.dumps({"metric": "serving samples/s and p50/p99 latency", "workload": "serve_qaoa_8acs",
                      "rate_per_s": args.rate, "duration_s": args.duration, "time_cap_s": cap, "requests": len(reqs),
                      "sampler": args.sampler, "ours_fp32_continuous": st, "baseline_fp64_one_at_a_time": st_b,
                      "identical_samples_ours_vs_fp64": f"{same} of {both} requests served by both",
                      "ac_nodes": {k: N.header(b)["n_nodes"] for k, b in acs.items()},
                      "ac_kind": {k: ("TRAJECTORY" if kinds[k] == N.QKC_AC_TRAJECTORY else "DENSITY") for k in acs}}),
          flush=True)


def run_gibbs_kl(args):
    """Sampling error vs number of samples (the paper's Sec. 3.3.3 evaluation): KL divergence
    of the empirical distribution from the exact one, for the exact chain-rule sampler on the
    density AC and for the Gibbs chain on the amplitude AC; an 8-qubit noisy QAOA (symmetric
    depolarising 0.5% after every gate) and a 16-qubit noise-free QAOA."""
    import torch
    from paper_2103_17226_gb300.build import build_library
    build_library()
    from paper_2103_17226_gb300 import inputs as I, native as N
    ctx = N.Context(0)
    out = {}
    cases = {"qaoa8_noisy": I.qaoa_maxcut(8, I.random_regular_graph(8, 3, seed=8), 1, [("DEP1", 0.005, "all")]),
             "qaoa16_ideal": I.qaoa_maxcut(16, I.random_regular_graph(16, 3, seed=16), 1, None)}
    for name, c in cases.items():
        n = c.n_qubits
        ang = I.uniform_angles(1, c.n_angles, seed=31)
        den = N.load_ac(ctx, N.compile(c, N.QKC_AC_DENSITY), precision=64)
        N.set_params(den, torch.tensor(ang, device="cuda"))
        ev = torch.tensor([[(x >> (n - 1 - q)) & 1 for q in range(n)] for x in range(2 ** n)], dtype=torch.int8,
                          device="cuda")
        P = N.evaluate(den, torch.zeros(2 ** n, dtype=torch.int32, device="cuda"), ev)[:, 0].cpu().numpy()
        P = np.clip(P, 0, None)
        P /= P.sum()

        def kl(samples):
            cnt = np.bincount(samples.astype(np.int64), minlength=2 ** n).astype(float)
            q = cnt / cnt.sum()
            m = q > 0
            return float(np.sum(q[m] * np.log(q[m] / P[m])))

        Ns = [100, 1000, 10000, 100000]
        exact = N.sample(den, torch.tensor([12345], dtype=torch.int64, device="cuda"),
                         torch.tensor([Ns[-1]], dtype=torch.int32, device="cuda"), Ns[-1])[0].cpu().numpy()
        amp = N.load_ac(ctx, N.compile(c, N.QKC_AC_AMPLITUDE), precision=32)
        N.set_params(amp, torch.tensor(ang, device="cuda"))
        chains, burn = 1000, 20
        n_rv = amp.n_vars - n
        # start: every noise variable at its first (no-error) value, outputs at the most likely noise-free one
        x0 = int(np.argmax(P))
        st = np.zeros((chains, amp.n_vars), dtype=np.int8)
        st[:, :n] = [(x0 >> (n - 1 - q)) & 1 for q in range(n)]
        state = torch.tensor(st, device="cuda")
        cv = torch.zeros(chains, dtype=torch.int32, device="cuda")
        seeds = torch.tensor(I.vector_seeds(chains, 77).astype(np.int64), device="cuda")
        t0 = time.perf_counter()
        N.gibbs(amp, cv, seeds, state, burn)
        sweeps = Ns[-1] // chains
        g = N.gibbs(amp, cv, seeds, state, sweeps, sweep_offset=burn).cpu().numpy()
        t_gibbs = time.perf_counter() - t0
        gs = g.T.reshape(-1)  # sweep-major: the first N samples use every chain
        out[name] = {"qubits": n, "noise_variables": n_rv,
                     "kl_exact": {str(k): kl(exact[:k]) for k in Ns},
                     "kl_gibbs": {str(k): kl(gs[:k]) for k in Ns},
                     "gibbs": {"chains": chains, "burn_in_sweeps": burn, "seconds": t_gibbs}}
    print(json.dumps({"metric": "KL(empirical || exact) vs samples", **out}), flush=True)


def main():
    args = parse()
    if args.workload == "gibbs_kl":
        run_gibbs_kl(args)
        return
    if args.mode == "serveacs":
        run_serveacs(args)
        return
    if args.workload == "serve":
        run_serve(args)
        return
    if args.mode == "uppass":
        run_uppass(args)
        return
    if args.mode == "gradpass":
        run_gradpass(args)
        return
    if args.mode == "samplepass":
        run_samplepass(args)
        return
    if args.mode == "reeval":
        run_reeval(args)
        return
    if args.workload == "qaoa10":
        if args.impl == "reference":
            if int(os.environ.get("RANK", "0")) == 0:
                W = make_workload("qaoa10", args.shots)
                rates = [oracle_trajectory_rate(W) for _ in range(args.warmup + args.steps)][args.warmup:]
                val = statistics.median([r["value"] for r in rates])
                print(json.dumps({"impl": "reference", "metric": W["metric"], "value": val, "unit": W["unit"],
                                  "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                                  "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
                                  "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                                  "config": {"workload": W["name"]},
                                  "cpu_baseline": dict(rates[-1], value=val),
                                  "e2e": {"value": val, "unit": W["unit"], "h2d_bytes_per_step": 0,
                                          "d2h_bytes_per_step": 0}}), flush=True)
        else:
            run_trajectory(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
