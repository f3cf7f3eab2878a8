"""The paper's Gibbs sampler written plainly (oracle; test infrastructure only).

Sec. 3.3.2: the chain moves over full assignments of the output qubits and the noise
random variables; the next state differs from the current one in one variable, drawn
with probability proportional to |A|^2 of each candidate assignment.  Here the chain
updates the variables in index order (outputs first, then the noise variables in
circuit order), and every candidate amplitude A(x, r) is recomputed from scratch by a
pure-state run that applies the chosen Kraus operator at each channel.

Decision rule (the same uniforms as the GPU sampler): for the update of variable V in
sweep t, u = (SplitMix64_k(seed) >> 11) 2^-53 with k = t * n_vars + V + 1, and the new
value is the smallest v with u * sum_w |A_w|^2 < sum_{w <= v} |A_w|^2.
"""
from __future__ import annotations

import numpy as np

from . import quantum as Q


def candidate_weights(circuit, angles, state, var):
    n = circuit.n_qubits
    cards = [2] * n + Q.channel_cards(circuit)
    w = []
    for v in range(cards[var]):
        st = list(state)
        st[var] = v
        psi = Q.statevector(circuit, angles, st[n:]) if len(cards) > n else Q.statevector(circuit, angles)
        w.append(abs(psi[tuple(st[:n])]) ** 2)
    return np.array(w)


def gibbs_chain(circuit, angles, state0, seed: int, n_sweeps: int, sweep_offset: int = 0):
    """Returns (final state, outcome index after every sweep)."""
    n = circuit.n_qubits
    state = list(int(x) for x in state0)
    nv = len(state)
    outs = []
    for t in range(sweep_offset, sweep_offset + n_sweeps):
        for var in range(nv):
            w = candidate_weights(circuit, angles, state, var)
            tot = w.sum()
            if not tot > 0:
                continue
            u = (Q.splitmix64(seed, t * nv + var + 1) >> 11) * (1.0 / 9007199254740992.0)
            acc = 0.0
            pick = len(w) - 1
            for v, wv in enumerate(w):
                acc += wv
                if u * tot < acc:
                    pick = v
                    break
            state[var] = pick
        idx = 0
        for q in range(n):
            idx = (idx << 1) | state[q]
        outs.append(idx)
    return state, outs
