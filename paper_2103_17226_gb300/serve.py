"""Continuous-batching request loop over resident ACs.

Each request asks for `shots` chain-rule samples of one compiled AC at one
parameter vector (a variational circuit evaluation, Sec. 3.3.2's sampling task).
The server keeps every AC resident on the device with `lanes` handles per AC,
each handle with its own CUDA stream and pre-sized scratch, and runs this loop
on the host:

  * arrivals are moved into a FIFO queue per AC;
  * every free lane takes the oldest requests of its AC, up to `max_batch`
    requests, as long as the samples in flight stay within the sample budget,
    and launches one batched sampling call on its stream
    (host->device copy of angles/seeds/shots, parameter binding, sampling,
    device->host copy of the outcome indices, completion event);
  * lanes of different ACs, and the lanes of one AC, run concurrently on the
    device, so requests that arrive while others are on the GPU are admitted as
    soon as a lane and memory free up;
  * a batch is complete when its event has fired; every request in it records
    its latency from arrival to completion.

The one-request-at-a-time FP64 baseline is the same loop with precision 64,
one lane, batches of one request, at most one batch in flight and the plain
sampler (every node evaluated once per prefix group).

A request's samples depend only on its AC, angles, seed and shot count: every
column of a batch is computed on its own (per-column scale words included), so
a request gives the same outcome indices alone and in any mix.

Admission by memory: all device memory a lane uses (the AC's value tile, the
sampler's group and sample arrays, the memoised slots) is reserved when the
server starts, by a warm-up call sized for `max_batch` requests of `max_shots`
shots, so no call in the loop allocates; a request is admitted when a lane of
its AC is free and holds it (its shots at most `max_shots`; larger requests are
refused when they arrive and counted), and `budget_samples` bounds the samples
in flight over all lanes.  Statistics: `run` serves until every admitted request
has completed (a run that hits `time_limit` counts each unfinished request at
its elapsed time, a lower bound of its latency, and reports how many there
were), so p50/p99 are taken over every admitted request.
"""
from __future__ import annotations

import heapq
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import native as N


@dataclass
class Request:
    rid: int
    ac: str
    angles: np.ndarray
    shots: int
    seed: int
    arrival: float  # seconds from the start of the run


@dataclass
class Result:
    rid: int
    bits: np.ndarray
    arrival: float
    done: float

    @property
    def latency(self):
        return self.done - self.arrival


@dataclass
class _Lane:
    name: str
    ac: N.AC
    stream: torch.cuda.Stream
    d_angles: torch.Tensor
    d_seeds: torch.Tensor
    d_shots: torch.Tensor
    d_bits: torch.Tensor
    h_angles: torch.Tensor
    h_seeds: torch.Tensor
    h_shots: torch.Tensor
    h_bits: torch.Tensor
    batch: list = field(default_factory=list)
    max_shots_in_batch: int = 0
    event: torch.cuda.Event = None
    start: torch.cuda.Event = None  # recorded before the batch's first copy: GPU time per batch


class Server:
    def __init__(self, ctx: N.Context, ac_bytes: dict, precision: int = 32, lanes: int = 2, max_batch: int = 32,
                 max_shots: int = 10000, tile_columns: int = 16384, budget_samples: int = 4_000_000,
                 serial: bool = False, memoised: bool = True, memo_budget_bytes: int = 2 << 30):
        self.max_batch = max_batch
        self.max_shots = max_shots
        self.budget = budget_samples
        self.serial = serial
        self.lanes = {}
        self.n_angles = {}
        dev = torch.device("cuda", ctx.device)
        for name, b in ac_bytes.items():
            self.lanes[name] = []
            for _ in range(lanes):
                ac = N.load_ac(ctx, b, precision=precision)
                N.set_tile_limit(ac, tile_columns)
                N.set_sampler(ac, 1 if memoised else 0, memo_budget_bytes)
                na = max(1, ac.n_angles)
                self.n_angles[name] = ac.n_angles
                ln = _Lane(
                    name=name, ac=ac, stream=torch.cuda.Stream(device=dev),
                    d_angles=torch.zeros((max_batch, na), dtype=torch.float64, device=dev),
                    d_seeds=torch.zeros(max_batch, dtype=torch.int64, device=dev),
                    d_shots=torch.zeros(max_batch, dtype=torch.int32, device=dev),
                    d_bits=torch.zeros((max_batch, max_shots), dtype=torch.int64, device=dev),
                    h_angles=torch.zeros((max_batch, na), dtype=torch.float64).pin_memory(),
                    h_seeds=torch.zeros(max_batch, dtype=torch.int64).pin_memory(),
                    h_shots=torch.zeros(max_batch, dtype=torch.int32).pin_memory(),
                    h_bits=torch.zeros((max_batch, max_shots), dtype=torch.int64).pin_memory(),
                )
                self.lanes[name].append(ln)
        self._warm()

    def _warm(self):
        """Size every lane's scratch for its largest batch now, so no call in the loop allocates."""
        for lanes in self.lanes.values():
            for ln in lanes:
                with torch.cuda.stream(ln.stream):
                    ln.h_shots.fill_(0)  # sizes the scratch for max_batch x max_shots without sampling
                    ln.d_shots.copy_(ln.h_shots)
                    N.set_params(ln.ac, ln.d_angles, stream=ln.stream)
                    N.sample(ln.ac, ln.d_seeds, ln.d_shots, self.max_shots, out=ln.d_bits, stream=ln.stream)
        torch.cuda.synchronize()

    def _launch(self, ln: _Lane, reqs):
        B = len(reqs)
        S = max(r.shots for r in reqs)
        na = self.n_angles[ln.name]
        for i, r in enumerate(reqs):
            if na:
                ln.h_angles[i, :na] = torch.from_numpy(np.asarray(r.angles, dtype=np.float64))
            ln.h_seeds[i] = int(np.int64(np.uint64(r.seed)))
            ln.h_shots[i] = r.shots
        with torch.cuda.stream(ln.stream):
            ln.start = torch.cuda.Event(enable_timing=True)
            ln.start.record(ln.stream)
            ln.d_angles[:B].copy_(ln.h_angles[:B], non_blocking=True)
            ln.d_seeds[:B].copy_(ln.h_seeds[:B], non_blocking=True)
            ln.d_shots[:B].copy_(ln.h_shots[:B], non_blocking=True)
            N.set_params(ln.ac, ln.d_angles[:B], stream=ln.stream)
            N.sample(ln.ac, ln.d_seeds[:B], ln.d_shots[:B], S, out=ln.d_bits[:B].view(-1)[:B * S].view(B, S),
                     stream=ln.stream, total_shots=sum(r.shots for r in reqs))
            ln.h_bits[:B].view(-1)[:B * S].copy_(ln.d_bits[:B].view(-1)[:B * S], non_blocking=True)
            ln.event = torch.cuda.Event(enable_timing=True)
            ln.event.record(ln.stream)
        ln.batch = list(reqs)
        ln.max_shots_in_batch = S

    def run(self, requests, time_limit: float = None):
        """Serve `requests` (arrival times in seconds from now) until every admitted one has completed, or
        until `time_limit` seconds. Returns (results, stats)."""
        refused = [r for r in requests if not 0 < r.shots <= self.max_shots]
        order = sorted((r for r in requests if 0 < r.shots <= self.max_shots), key=lambda r: r.arrival)
        queues = {name: [] for name in self.lanes}
        results = {}
        in_flight = 0
        nxt = 0
        t0 = time.perf_counter()
        busy = []
        gpu_ms = {name: 0.0 for name in self.lanes}  # event time of the batches of each AC
        batches = {name: 0 for name in self.lanes}
        while len(results) < len(order):
            now = time.perf_counter() - t0
            if time_limit is not None and now > time_limit:
                break
            while nxt < len(order) and order[nxt].arrival <= now:
                r = order[nxt]
                queues[r.ac].append(r)
                nxt += 1
            # completions
            still = []
            for ln in busy:
                if ln.event.query():
                    done = time.perf_counter() - t0
                    gpu_ms[ln.name] += ln.start.elapsed_time(ln.event)
                    batches[ln.name] += 1
                    S = ln.max_shots_in_batch
                    B = len(ln.batch)
                    bits = ln.h_bits[:B].view(-1)[:B * S].view(B, S).numpy()
                    for i, r in enumerate(ln.batch):
                        results[r.rid] = Result(r.rid, bits[i, :r.shots].copy(), r.arrival, done)
                        in_flight -= r.shots
                    ln.batch = []
                else:
                    still.append(ln)
            busy = still
            # admissions
            launched = False
            for name, lanes in self.lanes.items():
                q = queues[name]
                for ln in lanes:
                    if not q:
                        break
                    if ln.batch or (self.serial and busy):
                        continue
                    take = []
                    budget = self.budget - in_flight
                    while q and len(take) < self.max_batch and q[0].shots <= budget:
                        r = q.pop(0)
                        take.append(r)
                        budget -= r.shots
                    if not take:
                        continue
                    in_flight += sum(r.shots for r in take)
                    self._launch(ln, take)
                    busy.append(ln)
                    launched = True
            if not launched and not busy and nxt < len(order):
                wait = order[nxt].arrival - (time.perf_counter() - t0)
                if wait > 0:
                    time.sleep(min(wait, 0.001))
            elif not launched:
                time.sleep(20e-6)
        elapsed = time.perf_counter() - t0
        torch.cuda.synchronize()
        # every admitted request enters the percentiles: unfinished ones at their elapsed time (a lower bound)
        unfinished = [elapsed - r.arrival for r in order if r.rid not in results and r.arrival <= elapsed]
        lat = np.array([r.latency for r in results.values()] + unfinished) if (results or unfinished) else np.zeros(1)
        samples = sum(len(r.bits) for r in results.values())
        stats = dict(completed=len(results), submitted=len(order), refused=len(refused), unfinished=len(unfinished),
                     elapsed_s=elapsed, samples=samples, samples_per_s=samples / elapsed if elapsed > 0 else 0.0,
                     p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                     latency_over="every admitted request (unfinished ones at their elapsed time)",
                     # where the time goes: each batch's event time from its first copy to its last (lanes of
                     # different ACs overlap, so the sum can exceed the elapsed time)
                     batch_gpu_s={k: round(v / 1e3, 3) for k, v in gpu_ms.items()}, batches=batches,
                     batch_gpu_s_total=round(sum(gpu_ms.values()) / 1e3, 3))
        return results, stats


def poisson_requests(ac_names, n_angles, rate_per_s: float, duration_s: float, seed: int, shots_lo=100,
                     shots_hi=10000):
    """Open-loop Poisson arrivals over the ACs (uniform choice), one parameter vector and a
    log-uniform shot count per request."""
    from .inputs import SplitMix
    import math
    rng = SplitMix(seed)
    t = 0.0
    out = []
    rid = 0
    while True:
        t += -math.log(max(1e-300, 1.0 - rng.uniform())) / rate_per_s
        if t > duration_s:
            break
        name = ac_names[rng.randint(len(ac_names))]
        na = n_angles[name]
        ang = np.array([2 * math.pi * rng.uniform() for _ in range(na)])
        shots = int(round(math.exp(math.log(shots_lo) + (math.log(shots_hi) - math.log(shots_lo)) * rng.uniform())))
        out.append(Request(rid, name, ang, shots, rng.next_u64(), t))
        rid += 1
    return out
