"""Exact sampling of noisy circuits through noise trajectories (oracle; test infrastructure only).

Sec. 3.1 gives every noise channel a random variable whose value picks one of its Kraus
operators; the amplitude of an outcome x under a trajectory r (one value per channel) is the
pure-state amplitude A(x, r) with those operators applied, and P(x) = sum_r |A(x, r)|^2
(Sec. 3.3.1 sums the trajectories to the density matrix).  For a mixed-unitary channel every
Kraus operator is sqrt(p_k) times a unitary (depolarising: Paulis; phase and bit flip), so
sum_x |A(x, r)|^2 = prod_i p_{r_i} whatever the state: the trajectory can be drawn from these
branch probabilities first, and the outcome then from |A(x, r)|^2.  That samples P(x) exactly.

Here, plainly: for sample s of a parameter vector with seed `seed`
  * branch of channel i (circuit order): u = (SplitMix64_k(~seed) >> 11) 2^-53 with
    k = s * n_channels + i + 1; r_i = the smallest k with u < p_0 + ... + p_k (sums taken in
    value order), else the last value;
  * the state vector psi_r = (the circuit with E_{r_i} applied at each channel) |0...0>, by
    quantum.statevector (unnormalised: it carries the sqrt(p) factors);
  * qubit by qubit, x_j = 1 iff u * P(x_<j) >= P(x_<j, X_j = 0) with P the sums of |psi_r|^2
    over the outcomes with that prefix, u = quantum.sample_uniform(seed, s, j, n) -- the chain
    rule of quantum.chain_rule_samples on the trajectory's (unnormalised) distribution.
Parity unpinned: none -- pinned in tests/test_trajectory_oracle.py (every trajectory's norm is
the product of its branch probabilities; trajectory samples follow the density matrix's
distribution; branch frequencies follow the branch probabilities).
"""
from __future__ import annotations

import math

import numpy as np

from . import quantum as Q

U64 = (1 << 64) - 1


def branch_probabilities(kind: str, p: float) -> list:
    """p_k of the mixed-unitary channels: E_k = sqrt(p_k) U_k (quantum.kraus order)."""
    if kind == "DEP1":
        return [1 - p, p / 3, p / 3, p / 3]
    if kind == "DEP2":
        return [1 - p] + [p / 15] * 15
    if kind in ("PF", "BF"):
        return [1 - p, p]
    raise ValueError(f"{kind} is not a mixed-unitary channel")


def channels(circuit):
    return [op for op in circuit.ops if Q.is_channel(op.kind)]


def draw_trajectory(circuit, seed: int, s: int) -> list:
    chs = channels(circuit)
    r = []
    for i, op in enumerate(chs):
        z = Q.splitmix64((~int(seed)) & U64, s * len(chs) + i + 1)
        u = (z >> 11) * (1.0 / 9007199254740992.0)
        probs = branch_probabilities(op.kind, op.p)
        acc, pick = 0.0, len(probs) - 1
        for k in range(len(probs) - 1):
            acc += probs[k]
            if u < acc:
                pick = k
                break
        r.append(pick)
    return r


def trajectory_samples(circuit, angles, seed: int, shots: int, with_trajectories: bool = False):
    """Outcome indices (qubit 0 most significant) of `shots` samples; optionally their trajectories."""
    n = circuit.n_qubits
    out = np.zeros(shots, dtype=np.uint64)
    trajs = []
    cache = {}
    for s in range(shots):
        r = draw_trajectory(circuit, seed, s)
        key = tuple(r)
        if key not in cache:
            psi = Q.statevector(circuit, angles, r) if r else Q.statevector(circuit, angles)
            prob = (np.abs(psi) ** 2).reshape((2,) * n)
            pref = [None] * (n + 1)
            pref[n] = prob
            for j in range(n - 1, -1, -1):
                pref[j] = pref[j + 1].sum(axis=-1)
            cache[key] = pref
        pref = cache[key]
        bits = []
        for j in range(n):
            P = float(pref[j][tuple(bits)])
            p0 = float(pref[j + 1][tuple(bits) + (0,)])
            u = Q.sample_uniform(seed, s, j, n)
            bits.append(1 if u * P >= p0 else 0)
        idx = 0
        for b in bits:
            idx = (idx << 1) | b
        out[s] = idx
        trajs.append(r)
    return (out, trajs) if with_trajectories else out
