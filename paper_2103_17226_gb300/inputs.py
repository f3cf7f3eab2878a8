"""Seeded synthetic inputs shared by the library, the oracle, the tests and the bench.

This module holds no arithmetic of the simulation method: it only builds gate
lists (names, qubits, angle slots, noise strengths), graphs, parameter vectors,
Hamiltonian terms and seeds.  Gate matrices, Kraus operators, conditional
amplitude tables and everything computed from them live on each side separately
(the oracle and the CUDA library never share them).

Workload shapes follow the paper's evaluation (Sec. 4): QAOA for Max-Cut on
random graphs whose vertices have three edges, and noisy variants with a
depolarising channel after each gate (Sec. 4.2); a hardware-efficient ansatz with
amplitude damping and phase flip noise stands in for the VQE family.

Conventions (readings of the paper, which leaves them unstated):
  * RX/RY/RZ(theta) = exp(-i theta P / 2); ZZ(gamma) is CNOT(i,j) RZ_j(gamma) CNOT(i,j).
  * QAOA opens with H on every qubit; each of its p layers is ZZ(gamma_l) per edge in
    sorted order, then RX(beta_l) on every qubit; angle slots are
    (gamma_1, beta_1, ..., gamma_p, beta_p).
  * Qubit 0 is the most significant bit of an outcome index.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

# Gate and channel names understood by both sides.  Integer codes are the ones the
# C-ABI uses for its circuit description (include/qkc.h, qkc_op.kind).
GATE_CODES = {
    "H": 0, "X": 1, "Y": 2, "Z": 3, "RX": 4, "RY": 5, "RZ": 6, "CNOT": 7, "CZ": 8,
}
CHANNEL_CODES = {
    "DEP1": 16, "DEP2": 17, "AD": 18, "PD": 19, "PF": 20, "BF": 21,
}
OP_CODES = {**GATE_CODES, **CHANNEL_CODES}
PARAMETRISED = {"RX", "RY", "RZ"}
TWO_QUBIT = {"CNOT", "CZ", "DEP2"}

U64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15


@dataclass(frozen=True)
class Op:
    """One circuit operation: a gate (angle slot >= 0 when parametrised) or a noise channel (p)."""
    kind: str
    qubits: tuple
    angle: int = -1
    p: float = 0.0


@dataclass
class Circuit:
    n_qubits: int
    n_angles: int
    ops: list = field(default_factory=list)
    name: str = ""

    def add(self, kind, qubits, angle=-1, p=0.0):
        if isinstance(qubits, int):
            qubits = (qubits,)
        self.ops.append(Op(kind, tuple(int(q) for q in qubits), int(angle), float(p)))
        return self

    def n_gates(self):
        return sum(1 for o in self.ops if o.kind in GATE_CODES)

    def n_channels(self):
        return sum(1 for o in self.ops if o.kind in CHANNEL_CODES)

    def as_records(self):
        """The circuit as a numpy structured array laid out like the C struct qkc_op."""
        rec = np.zeros(len(self.ops), dtype=OP_DTYPE)
        for i, o in enumerate(self.ops):
            rec[i]["kind"] = OP_CODES[o.kind]
            rec[i]["q0"] = o.qubits[0]
            rec[i]["q1"] = o.qubits[1] if len(o.qubits) > 1 else -1
            rec[i]["angle"] = o.angle
            rec[i]["p"] = o.p
        return rec


OP_DTYPE = np.dtype([("kind", "<i4"), ("q0", "<i4"), ("q1", "<i4"), ("angle", "<i4"), ("p", "<f8")],
                    align=True)


# --------------------------------------------------------------------------- random numbers
def splitmix64(seed: int, k: int) -> int:
    """k-th output (k >= 1) of a SplitMix64 stream seeded with `seed`.

    SplitMix64 (Steele, Lea, Flood, OOPSLA 2014): the state advances by the golden
    gamma and each output is the state passed through the variant-13 mixer.  Used
    here only to draw seeded synthetic inputs."""
    z = (seed + k * GOLDEN_GAMMA) & U64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & U64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & U64
    return z ^ (z >> 31)


class SplitMix:
    """Sequential SplitMix64 stream for input generation."""

    def __init__(self, seed: int):
        self.seed = seed & U64
        self.k = 0

    def next_u64(self) -> int:
        self.k += 1
        return splitmix64(self.seed, self.k)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, n: int) -> int:
        return int(self.uniform() * n)

    def normal(self) -> float:
        # Box-Muller transform.
        u1 = self.uniform()
        u2 = self.uniform()
        u1 = max(u1, 1e-300)
        return math.sqrt(-2.0 * math.log(u1)) * math.cos(2.0 * math.pi * u2)


# --------------------------------------------------------------------------- graphs
def random_regular_graph(n: int, degree: int, seed: int, max_tries: int = 10000):
    """Random `degree`-regular simple graph by the pairing (configuration) model with
    rejection of self-loops and repeated edges.  Returns sorted edges (i < j)."""
    if (n * degree) % 2 or degree >= n:
        raise ValueError("no simple regular graph with these sizes")
    rng = SplitMix(seed)
    for _ in range(max_tries):
        stubs = [v for v in range(n) for _ in range(degree)]
        # Fisher-Yates shuffle driven by the seeded stream.
        for i in range(len(stubs) - 1, 0, -1):
            j = rng.randint(i + 1)
            stubs[i], stubs[j] = stubs[j], stubs[i]
        edges = set()
        ok = True
        for a, b in zip(stubs[0::2], stubs[1::2]):
            e = (min(a, b), max(a, b))
            if a == b or e in edges:
                ok = False
                break
            edges.add(e)
        if ok:
            return sorted(edges)
    raise RuntimeError("pairing model did not produce a simple graph")


def ring_graph(n: int):
    return sorted((min(i, (i + 1) % n), max(i, (i + 1) % n)) for i in range(n))


# --------------------------------------------------------------------------- circuits
def _noise_after(c: Circuit, gate: str, qubits, noise):
    """Append the noise channels that follow one gate.

    `noise` maps to a list of (channel, p, arity) entries:
      * ("DEP1", p, "1q")  -> after single-qubit gates only, on that qubit
      * ("DEP1", p, "all") -> after every gate, on each qubit it touches
      * ("DEP2", p, "2q")  -> after two-qubit gates, on the pair
      * ("AD"/"PF"/..., p, "all") -> after every gate, on each touched qubit
    """
    if not noise:
        return
    two = len(qubits) == 2
    for ch, p, scope in noise:
        if scope == "2q":
            if two:
                c.add(ch, qubits, p=p)
        elif scope == "1q":
            if not two:
                c.add(ch, qubits[0], p=p)
        else:
            for q in qubits:
                c.add(ch, q, p=p)


def qaoa_maxcut(n: int, edges, p: int, noise=None, name="") -> Circuit:
    """QAOA for Max-Cut: H on all qubits, then p layers of (ZZ(gamma_l) per edge, RX(beta_l) all)."""
    c = Circuit(n, 2 * p, name=name or f"qaoa_n{n}_p{p}")
    for q in range(n):
        c.add("H", q)
        _noise_after(c, "H", (q,), noise)
    for layer in range(p):
        g, b = 2 * layer, 2 * layer + 1
        for (i, j) in edges:
            c.add("CNOT", (i, j))
            _noise_after(c, "CNOT", (i, j), noise)
            c.add("RZ", j, angle=g)
            _noise_after(c, "RZ", (j,), noise)
            c.add("CNOT", (i, j))
            _noise_after(c, "CNOT", (i, j), noise)
        for q in range(n):
            c.add("RX", q, angle=b)
            _noise_after(c, "RX", (q,), noise)
    return c


def hardware_efficient_ansatz(n: int, layers: int, noise=None, name="") -> Circuit:
    """Hardware-efficient ansatz: per layer RY then RZ on every qubit, then CZ(i, i+1)."""
    c = Circuit(n, 2 * n * layers, name=name or f"hea_n{n}_l{layers}")
    a = 0
    for _ in range(layers):
        for q in range(n):
            c.add("RY", q, angle=a)
            a += 1
            _noise_after(c, "RY", (q,), noise)
        for q in range(n):
            c.add("RZ", q, angle=a)
            a += 1
            _noise_after(c, "RZ", (q,), noise)
        for q in range(n - 1):
            c.add("CZ", (q, q + 1))
            _noise_after(c, "CZ", (q, q + 1), noise)
    return c


def grid_edges(rows: int, cols: int):
    """Nearest-neighbour couplings of a rows x cols grid, qubit r * cols + c, sorted (i < j)."""
    e = []
    for r in range(rows):
        for c in range(cols):
            q = r * cols + c
            if c + 1 < cols:
                e.append((q, q + 1))
            if r + 1 < rows:
                e.append((q, q + cols))
    return sorted(e)


def vqe_ising_2d(rows: int, cols: int, layers: int, noise=None, name="") -> Circuit:
    """Variational ansatz for the 2D Ising model (the paper's VQE workload: a qubit per grid
    point, two-qubit gates along the couplings): H on every qubit, then per layer RY(theta_{l,q})
    on every qubit and ZZ(phi_l) = CNOT RZ(phi_l) CNOT on every grid coupling.  Angle slots:
    per layer n qubit angles then one coupling angle."""
    n = rows * cols
    edges = grid_edges(rows, cols)
    c = Circuit(n, layers * (n + 1), name=name or f"vqe_ising_{rows}x{cols}_l{layers}")
    for q in range(n):
        c.add("H", q)
        _noise_after(c, "H", (q,), noise)
    for layer in range(layers):
        base = layer * (n + 1)
        for q in range(n):
            c.add("RY", q, angle=base + q)
            _noise_after(c, "RY", (q,), noise)
        for (i, j) in edges:
            c.add("CNOT", (i, j))
            _noise_after(c, "CNOT", (i, j), noise)
            c.add("RZ", j, angle=base + n)
            _noise_after(c, "RZ", (j,), noise)
            c.add("CNOT", (i, j))
            _noise_after(c, "CNOT", (i, j), noise)
    return c


def ising_hamiltonian(rows: int, cols: int, J: float = 1.0, h: float = 0.5):
    """H = J sum_<ij> Z_i Z_j + h sum_i Z_i on the grid, as Z-string supports and coefficients."""
    n = rows * cols
    sup, coef = [], []
    for (i, j) in grid_edges(rows, cols):
        row = np.zeros(n, dtype=bool)
        row[i] = row[j] = True
        sup.append(row)
        coef.append(J)
    for q in range(n):
        row = np.zeros(n, dtype=bool)
        row[q] = True
        sup.append(row)
        coef.append(h)
    return np.array(sup), np.array(coef, dtype=np.float64)


def random_circuit(n: int, n_ops: int, seed: int, noise_prob: float = 0.3, n_angles: int = 3) -> Circuit:
    """Random small noisy circuit over every gate and channel kind (test input)."""
    rng = SplitMix(seed)
    gates = ["H", "X", "Y", "Z", "RX", "RY", "RZ", "CNOT", "CZ"]
    chans = ["DEP1", "DEP2", "AD", "PD", "PF", "BF"]
    c = Circuit(n, n_angles, name=f"random_n{n}_s{seed}")
    for _ in range(n_ops):
        g = gates[rng.randint(len(gates))]
        if g in TWO_QUBIT and n < 2:
            g = "H"
        if g in TWO_QUBIT:
            a = rng.randint(n)
            b = (a + 1 + rng.randint(n - 1)) % n
            c.add(g, (a, b))
        else:
            c.add(g, rng.randint(n), angle=rng.randint(n_angles) if g in PARAMETRISED else -1)
        if rng.uniform() < noise_prob:
            ch = chans[rng.randint(len(chans))]
            pr = 0.02 + 0.2 * rng.uniform()
            if ch == "DEP2":
                if n < 2:
                    continue
                a = rng.randint(n)
                b = (a + 1 + rng.randint(n - 1)) % n
                c.add(ch, (a, b), p=pr)
            else:
                c.add(ch, rng.randint(n), p=pr)
    return c


def noisy_bell(gamma: float = 0.36) -> Circuit:
    """The paper's worked example (Sec. 2.2, Fig. 2a): H on q0, phase damping on q0, CNOT(q0, q1)."""
    c = Circuit(2, 0, name="noisy_bell")
    c.add("H", 0)
    c.add("PD", 0, p=gamma)
    c.add("CNOT", (0, 1))
    return c


# --------------------------------------------------------------------------- parameters etc.
def uniform_angles(n_vectors: int, n_angles: int, seed: int) -> np.ndarray:
    """Parameter vectors with every angle uniform in [0, 2 pi), shape [V][n_angles] float64."""
    rng = SplitMix(seed)
    out = np.empty((n_vectors, n_angles), dtype=np.float64)
    for v in range(n_vectors):
        for a in range(n_angles):
            out[v, a] = 2.0 * math.pi * rng.uniform()
    return out


def vector_seeds(n_vectors: int, seed: int) -> np.ndarray:
    """One 64-bit sampling seed per parameter vector."""
    rng = SplitMix(seed ^ 0x5EED)
    return np.array([rng.next_u64() for _ in range(n_vectors)], dtype=np.uint64)


def z_string_hamiltonian(n: int, n_terms: int, seed: int):
    """Random Pauli-Z string Hamiltonian: each term's support takes every qubit with
    probability 1/2 (redrawn if empty); coefficients are standard normal.
    Returns (supports [n_terms][n] bool, coefficients [n_terms] float64)."""
    rng = SplitMix(seed ^ 0x4A11)
    sup = np.zeros((n_terms, n), dtype=bool)
    coef = np.empty(n_terms, dtype=np.float64)
    for t in range(n_terms):
        while True:
            row = [rng.uniform() < 0.5 for _ in range(n)]
            if any(row):
                break
        sup[t] = row
        coef[t] = rng.normal()
    return sup, coef


def log_uniform_shots(n: int, lo: int, hi: int, seed: int) -> np.ndarray:
    rng = SplitMix(seed ^ 0x5407)
    return np.array([int(round(math.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * rng.uniform())))
                     for _ in range(n)], dtype=np.int32)


# --------------------------------------------------------------------------- named workloads
NOISE_CFG1 = [("DEP1", 0.01, "all")]
NOISE_CFG2 = [("DEP1", 0.001, "1q"), ("DEP2", 0.01, "2q")]
NOISE_CFG3 = [("AD", 0.005, "all"), ("PF", 0.005, "all")]


def workload(name: str):
    """Circuit and batch shapes of the named synthetic workloads."""
    if name == "qaoa4_ring_p1":
        return qaoa_maxcut(4, ring_graph(4), 1, NOISE_CFG1, name=name)
    if name == "qaoa10_3reg_p2":
        return qaoa_maxcut(10, random_regular_graph(10, 3, seed=2), 2, NOISE_CFG2, name=name)
    if name == "hea16_l6":
        return hardware_efficient_ansatz(16, 6, NOISE_CFG3, name=name)
    if name == "qaoa32_3reg_p1_ideal":
        return qaoa_maxcut(32, random_regular_graph(32, 3, seed=5), 1, None, name=name)
    if name == "vqe_ising_3x3_noisy":
        return vqe_ising_2d(3, 3, 2, [("DEP1", 0.005, "all")], name=name)
    if name == "vqe_ising_5x5_ideal":
        return vqe_ising_2d(5, 5, 1, None, name=name)
    if name.startswith("serve_qaoa"):
        # serve_qaoa{n}_p{p}
        body = name[len("serve_qaoa"):]
        nq, pp = body.split("_p")
        nq, pp = int(nq), int(pp)
        return qaoa_maxcut(nq, random_regular_graph(nq, 3, seed=40 + nq), pp, NOISE_CFG2, name=name)
    raise KeyError(name)
