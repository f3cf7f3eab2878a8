"""The paper's Bayesian-network semantics evaluated by brute force (oracle; test
infrastructure only).

Sec. 3.1: each gate contributes a conditional amplitude table (CAT) with
A(out = j | in = i) = U[j][i] -- rows are input basis states, columns output
states, so the table reads as the transpose of the unitary (Table 3a); a
monomial multi-qubit gate's table is a permutation of its unitary (Table 3c);
a noise channel contributes a random-variable node whose table holds its Kraus
operators (Table 3b).  The amplitude of an assignment of the output and noise
variables is the sum, over every assignment of the intermediate qubit
variables, of the product of all table entries (Sec. 3.2.1: each satisfying
assignment is a Feynman path; its weight is the product of its entries).

Here every operation, diagonal or not, gets fresh output variables for the
qubits it acts on, and the sum runs over all of them explicitly: nothing is
eliminated, factored or cached.  Exponential; tiny circuits only.
"""
from __future__ import annotations

import numpy as np

from . import quantum as Q


def cat(kind: str, theta=None) -> np.ndarray:
    """Conditional amplitude table of a one- or two-qubit gate: rows = input basis
    state, columns = output basis state (the paper's Table 3 layout)."""
    return Q.gate_matrix(kind, theta).T.copy()


def noise_cat(kind: str, p: float) -> np.ndarray:
    """CAT of a noise channel, indexed [k][in][out] = (E_k)[out][in]."""
    return np.array([E.T for E in Q.kraus(kind, p)])


def _paths(circuit, angles):
    """Enumerate (weight, output bits, trajectory) of every path with nonzero weight.

    Depth-first over the operations in circuit order: at each operation every
    value of its fresh output variables (and of its noise variable) is tried,
    the path weight is multiplied by the table entry, and zero-weight branches
    stop there.  Nothing is summed early or cached: each complete path is
    yielded on its own."""
    n = circuit.n_qubits
    ops = circuit.ops
    tables = []
    for op in ops:
        if Q.is_channel(op.kind):
            tables.append(("ch", noise_cat(op.kind, op.p)))          # [k][in][out]
        else:
            th = angles[op.angle] if op.angle >= 0 else None
            tables.append(("gate", cat(op.kind, th)))                # [in][out]

    def rec(i, cur, w, r):
        if i == len(ops):
            yield w, tuple(cur), tuple(r)
            return
        op = ops[i]
        qs = list(op.qubits)
        i_idx = 0
        for q in qs:
            i_idx = (i_idx << 1) | cur[q]
        kind, T = tables[i]
        ks = range(T.shape[0]) if kind == "ch" else [None]
        for k in ks:
            row = T[k][i_idx] if kind == "ch" else T[i_idx]
            for o_idx in range(1 << len(qs)):
                e = row[o_idx]
                if e == 0:
                    continue
                nxt = list(cur)
                for b, q in enumerate(qs):
                    nxt[q] = (o_idx >> (len(qs) - 1 - b)) & 1
                yield from rec(i + 1, nxt, w * e, r + ([k] if kind == "ch" else []))

    yield from rec(0, [0] * n, 1.0 + 0j, [])


def amplitude_table(circuit, angles) -> dict:
    """A(x, r) for every output assignment x and trajectory r with a nonzero path sum."""
    acc = {}
    for w, x, r in _paths(circuit, angles):
        acc[(x, r)] = acc.get((x, r), 0j) + w
    return acc


def amplitude_evidence(circuit, angles, ev_x, ev_r) -> complex:
    """sum_{x, r} prod lam(x) prod lam(r) A(x, r) by brute force."""
    lam_x = Q.indicator_vectors(ev_x)
    lam_r = Q.indicator_vectors(ev_r, Q.channel_cards(circuit))
    tot = 0j
    for (x, r), a in amplitude_table(circuit, angles).items():
        w = 1.0
        for j, xj in enumerate(x):
            w *= lam_x[j][xj]
        for i, ri in enumerate(r):
            w *= lam_r[i][ri]
        tot += w * a
    return tot


def density_evidence(circuit, angles, ev_x) -> complex:
    """sum_x prod lam(x) sum_r |A(x, r)|^2: the noisy outcome distribution through the
    paper's noise-as-random-variable encoding (each Kraus branch a spurious measurement)."""
    lam_x = Q.indicator_vectors(ev_x)
    tot = 0j
    for (x, r), a in amplitude_table(circuit, angles).items():
        w = 1.0
        for j, xj in enumerate(x):
            w *= lam_x[j][xj]
        tot += w * abs(a) ** 2
    return tot
