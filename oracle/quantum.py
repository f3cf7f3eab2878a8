"""Ground-truth quantum simulation in FP64 (oracle; test infrastructure only).

Every function here is the textbook definition written out with numpy:
  * pure states evolve as psi -> U psi (Sec. 2.1, Eq. 1);
  * mixed states as rho -> U rho U^dagger, and a noise channel with Kraus
    operators E_k as rho -> sum_k E_k rho E_k^dagger (Sec. 2.2; the paper prints
    E_k^T, which equals E_k^dagger for its real phase-damping example -- the
    conjugate transpose is the definition used here);
  * outcome probabilities are the diagonal of rho, P(x) = <x|rho|x>;
  * qubit 0 is the most significant bit of an outcome index (axis 0 of the
    state tensor).
Parity unpinned: none -- every function is pinned in tests/test_oracle_pins.py
(the chain-rule sampler also by planted mistakes in tests/test_oracle_sampler_pins.py).
"""
from __future__ import annotations

import itertools
import math

import numpy as np

U64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15  # SplitMix64 state increment
SQ2 = 1.0 / math.sqrt(2.0)
I2 = np.eye(2, dtype=complex)
PX = np.array([[0, 1], [1, 0]], dtype=complex)
PY = np.array([[0, -1j], [1j, 0]], dtype=complex)
PZ = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = [I2, PX, PY, PZ]


# --------------------------------------------------------------------------- gates
def gate_matrix(kind: str, theta: float | None = None) -> np.ndarray:
    """Unitary of a gate; RX/RY/RZ(t) = exp(-i t P / 2); CNOT with the first qubit as control."""
    if kind == "H":
        return np.array([[SQ2, SQ2], [SQ2, -SQ2]], dtype=complex)
    if kind == "X":
        return PX.copy()
    if kind == "Y":
        return PY.copy()
    if kind == "Z":
        return PZ.copy()
    if kind in ("RX", "RY", "RZ"):
        P = {"RX": PX, "RY": PY, "RZ": PZ}[kind]
        return math.cos(theta / 2) * I2 - 1j * math.sin(theta / 2) * P
    if kind == "CNOT":
        return np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]], dtype=complex)
    if kind == "CZ":
        return np.diag([1, 1, 1, -1]).astype(complex)
    raise KeyError(kind)


def gate_derivative(kind: str, theta: float) -> np.ndarray:
    """d/dtheta exp(-i theta P/2) = -(i/2) P exp(-i theta P/2)."""
    P = {"RX": PX, "RY": PY, "RZ": PZ}[kind]
    return -0.5j * P @ gate_matrix(kind, theta)


def kraus(kind: str, p: float) -> list:
    """Kraus operators of the noise channels (Nielsen & Chuang Ch. 8.3; phase damping
    as in the paper's Sec. 2.2, with the sign of its Table 3b on the damping operator)."""
    if kind == "DEP1":
        return [math.sqrt(1 - p) * I2] + [math.sqrt(p / 3) * P for P in (PX, PY, PZ)]
    if kind == "DEP2":
        ops = []
        for a in range(4):
            for b in range(4):
                w = math.sqrt(1 - p) if (a == 0 and b == 0) else math.sqrt(p / 15)
                ops.append(w * np.kron(PAULI[a], PAULI[b]))
        return ops
    if kind == "AD":
        return [np.array([[1, 0], [0, math.sqrt(1 - p)]], dtype=complex),
                np.array([[0, math.sqrt(p)], [0, 0]], dtype=complex)]
    if kind == "PD":
        return [np.array([[1, 0], [0, math.sqrt(1 - p)]], dtype=complex),
                np.array([[0, 0], [0, -math.sqrt(p)]], dtype=complex)]
    if kind == "PF":
        return [math.sqrt(1 - p) * I2, math.sqrt(p) * PZ]
    if kind == "BF":
        return [math.sqrt(1 - p) * I2, math.sqrt(p) * PX]
    raise KeyError(kind)


def is_channel(kind: str) -> bool:
    return kind in ("DEP1", "DEP2", "AD", "PD", "PF", "BF")


# --------------------------------------------------------------------------- tensor helpers
def _apply_ket(t: np.ndarray, mat: np.ndarray, axes) -> np.ndarray:
    """Apply a (2^k x 2^k) matrix to tensor axes `axes` (k of them): t' = M t."""
    k = len(axes)
    m = mat.reshape((2,) * (2 * k))
    out = np.tensordot(m, t, axes=(list(range(k, 2 * k)), list(axes)))
    # tensordot puts the new axes first; move them back into place
    return np.moveaxis(out, list(range(k)), list(axes))


def _apply_rho(rho: np.ndarray, n: int, mat: np.ndarray, qubits) -> np.ndarray:
    """rho -> M rho M^dagger on the given qubits (rho has n ket axes then n bra axes)."""
    r = _apply_ket(rho, mat, list(qubits))
    return _apply_ket(r, mat.conj(), [n + q for q in qubits])


# --------------------------------------------------------------------------- simulators
def statevector(circuit, angles, kraus_choice=None) -> np.ndarray:
    """Pure-state simulation.  With `kraus_choice` (one Kraus index per channel, in
    circuit order) the chosen, unnormalised Kraus operator is applied at each
    channel, giving the amplitude of a noise trajectory A(x, r); without it every
    channel is an error (use it for noise-free circuits only)."""
    n = circuit.n_qubits
    psi = np.zeros((2,) * n, dtype=complex)
    psi[(0,) * n] = 1.0
    ch = 0
    for op in circuit.ops:
        if is_channel(op.kind):
            if kraus_choice is None:
                raise ValueError("noisy circuit needs a Kraus choice for a pure-state run")
            E = kraus(op.kind, op.p)[kraus_choice[ch]]
            ch += 1
            psi = _apply_ket(psi, E, list(op.qubits))
        else:
            th = angles[op.angle] if op.angle >= 0 else None
            psi = _apply_ket(psi, gate_matrix(op.kind, th), list(op.qubits))
    return psi


def density_matrix(circuit, angles) -> np.ndarray:
    """Mixed-state simulation from |0...0><0...0|; returns rho as a (2^n x 2^n) matrix."""
    n = circuit.n_qubits
    rho = np.zeros((2,) * (2 * n), dtype=complex)
    rho[(0,) * (2 * n)] = 1.0
    for op in circuit.ops:
        if is_channel(op.kind):
            acc = np.zeros_like(rho)
            for E in kraus(op.kind, op.p):
                acc += _apply_rho(rho, n, E, op.qubits)
            rho = acc
        else:
            th = angles[op.angle] if op.angle >= 0 else None
            rho = _apply_rho(rho, n, gate_matrix(op.kind, th), op.qubits)
    return rho.reshape(2 ** n, 2 ** n)


def density_matrix_and_derivative(circuit, angles, k: int):
    """rho and d rho / d angle_k by forward-mode differentiation of the evolution:
    for a gate using angle k, d(M rho M^+) = dM rho M^+ + M rho dM^+ + M drho M^+."""
    n = circuit.n_qubits
    rho = np.zeros((2,) * (2 * n), dtype=complex)
    rho[(0,) * (2 * n)] = 1.0
    drho = np.zeros_like(rho)
    for op in circuit.ops:
        if is_channel(op.kind):
            acc = np.zeros_like(rho)
            dacc = np.zeros_like(rho)
            for E in kraus(op.kind, op.p):
                acc += _apply_rho(rho, n, E, op.qubits)
                dacc += _apply_rho(drho, n, E, op.qubits)
            rho, drho = acc, dacc
            continue
        th = angles[op.angle] if op.angle >= 0 else None
        M = gate_matrix(op.kind, th)
        new_d = _apply_rho(drho, n, M, op.qubits)
        if op.angle == k:
            dM = gate_derivative(op.kind, th)
            qs = list(op.qubits)
            t1 = _apply_ket(_apply_ket(rho, dM, qs), M.conj(), [n + q for q in qs])
            t2 = _apply_ket(_apply_ket(rho, M, qs), dM.conj(), [n + q for q in qs])
            new_d = new_d + t1 + t2
        rho = _apply_rho(rho, n, M, op.qubits)
        drho = new_d
    return rho.reshape(2 ** n, 2 ** n), drho.reshape(2 ** n, 2 ** n)


def probabilities(circuit, angles) -> np.ndarray:
    """P(x) = <x|rho|x> for every outcome index x (qubit 0 most significant)."""
    return np.real(np.diag(density_matrix(circuit, angles))).copy()


# --------------------------------------------------------------------------- evidence
def indicator_vectors(evidence, cards=None):
    """Indicator values per variable from evidence codes: -1 free (all 1), k observed
    (1 at k, 0 elsewhere), -2 Pauli-Z sign (1, -1).  Returns a list of vectors."""
    out = []
    for i, e in enumerate(evidence):
        c = 2 if cards is None else int(cards[i])
        if e == -1:
            out.append(np.ones(c))
        elif e == -2:
            if c != 2:
                raise ValueError("Z sign needs a binary variable")
            out.append(np.array([1.0, -1.0]))
        else:
            v = np.zeros(c)
            v[int(e)] = 1.0
            out.append(v)
    return out


def weighted_sum(probs: np.ndarray, lam) -> complex:
    """sum_x prod_j lam_j(x_j) P(x): the density polynomial at indicator values lam."""
    n = len(lam)
    t = probs.reshape((2,) * n).astype(complex)
    for j in range(n):
        t = np.tensordot(lam[j].astype(complex), t, axes=([0], [0]))
    return complex(t)


def density_evidence(probs: np.ndarray, evidence) -> complex:
    """Marginal probability of the evidence (or a Z-string expectation with code -2)."""
    return weighted_sum(probs, indicator_vectors(evidence))


def density_marginals(probs: np.ndarray, evidence) -> np.ndarray:
    """For every qubit j and value v: sum over x with x_j = v of prod_{i != j} lam_i(x_i) P(x),
    i.e. P(e without X_j, X_j = v).  Returns [n][2]."""
    n = int(round(math.log2(probs.size)))
    lam = indicator_vectors(evidence)
    out = np.zeros((n, 2), dtype=complex)
    for j in range(n):
        for v in range(2):
            l2 = list(lam)
            e = np.zeros(2)
            e[v] = 1.0
            l2[j] = e
            out[j, v] = weighted_sum(probs, l2)
    return out


def z_expectation(probs: np.ndarray, support) -> float:
    """<Z_S> = sum_x (-1)^{sum_{j in S} x_j} P(x)."""
    n = int(round(math.log2(probs.size)))
    ev = [-2 if support[j] else -1 for j in range(n)]
    return density_evidence(probs, ev).real


def hamiltonian_value_and_gradient(circuit, angles, supports, coefs, angle_slots=None):
    """<H> = sum_t c_t <Z_{S_t}> and its exact gradient (forward mode) in every angle, or in
    the listed angle slots only (the other entries stay 0)."""
    n = circuit.n_qubits
    probs = probabilities(circuit, angles)
    val = sum(c * z_expectation(probs, s) for s, c in zip(supports, coefs))
    grad = np.zeros(circuit.n_angles)
    for k in (range(circuit.n_angles) if angle_slots is None else angle_slots):
        _, drho = density_matrix_and_derivative(circuit, angles, k)
        dprobs = np.real(np.diag(drho))
        grad[k] = sum(c * z_expectation(dprobs, s) for s, c in zip(supports, coefs))
    return val, grad


# --------------------------------------------------------------------------- amplitude polynomial
def channel_cards(circuit):
    return [len(kraus(op.kind, op.p)) for op in circuit.ops if is_channel(op.kind)]


def amplitude_evidence(circuit, angles, ev_x, ev_r) -> complex:
    """The paper's amplitude polynomial (Table 5) at evidence:
    sum over outcomes x and trajectories r of prod lam(x) prod lam(r) A(x, r),
    with A(x, r) from a pure-state run applying the chosen Kraus operators."""
    n = circuit.n_qubits
    cards = channel_cards(circuit)
    lam_x = indicator_vectors(ev_x)
    lam_r = indicator_vectors(ev_r, cards)
    total = 0j
    choices = [range(c) if ev_r[i] == -1 else [int(ev_r[i])] for i, c in enumerate(cards)]
    for r in itertools.product(*choices):
        w = 1.0
        for i, ri in enumerate(r):
            w *= lam_r[i][ri]
        if w == 0:
            continue
        amp = statevector(circuit, angles, r) if cards else statevector(circuit, angles)
        t = amp
        for j in range(n):
            t = np.tensordot(lam_x[j].astype(complex), t, axes=([0], [0]))
        total += w * complex(t)
    return total


# --------------------------------------------------------------------------- sampling
def splitmix64(seed: int, k: int) -> int:
    """k-th output of a SplitMix64 stream (Steele, Lea, Flood 2014)."""
    z = (int(seed) + k * GOLDEN_GAMMA) & U64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & U64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & U64
    return z ^ (z >> 31)


def sample_uniform(seed: int, s: int, j: int, n: int) -> float:
    """Uniform in [0, 1) for sample s, qubit j: top 53 bits of output k = s*n + j + 1."""
    return (splitmix64(seed, s * n + j + 1) >> 11) * (1.0 / 9007199254740992.0)


def chain_rule_samples(probs: np.ndarray, seed: int, shots: int) -> np.ndarray:
    """Exact sampling by the chain rule P(x) = prod_j P(x_j | x_<j): x_j = 1 iff
    u * P(x_<j) >= P(x_<j, X_j = 0).  Returns outcome indices (qubit 0 MSB)."""
    n = int(round(math.log2(probs.size)))
    t = probs.reshape((2,) * n)
    # prefix marginals: pref[j] has shape (2,)*j, P(x_<j)
    pref = [None] * (n + 1)
    pref[n] = t
    for j in range(n - 1, -1, -1):
        pref[j] = pref[j + 1].sum(axis=-1)
    out = np.zeros(shots, dtype=np.uint64)
    for s in range(shots):
        bits = []
        for j in range(n):
            P = float(pref[j][tuple(bits)])
            p0 = float(pref[j + 1][tuple(bits) + (0,)])
            u = sample_uniform(seed, s, j, n)
            bits.append(1 if u * P >= p0 else 0)
        idx = 0
        for b in bits:
            idx = (idx << 1) | b
        out[s] = idx
    return out


def _probabilities_job(job):
    circuit, angles = job
    return probabilities(circuit, angles)


def probabilities_many(circuit, angle_list, processes: int = 0):
    """probabilities() for several parameter vectors, one spawn-started process per vector (up to
    the host's cores); an executor raises if a worker dies rather than waiting for it."""
    import multiprocessing as mp
    import os
    from concurrent.futures import ProcessPoolExecutor
    jobs = [(circuit, np.asarray(a, dtype=float)) for a in angle_list]
    procs = processes or min(len(jobs), os.cpu_count() or 1)
    if procs <= 1:
        return [_probabilities_job(j) for j in jobs]
    # one thread per worker process: the workers already use the cores
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with ProcessPoolExecutor(procs, mp_context=mp.get_context("spawn")) as ex:
            return list(ex.map(_probabilities_job, jobs))
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
