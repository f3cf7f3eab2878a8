"""CPU pins of the trajectory oracle (oracle/trajectory.py) and of the compiler's TRAJECTORY ACs.

* Every trajectory of a mixed-unitary noisy circuit has norm sum_x |A(x, r)|^2 equal to the product
  of its branch probabilities (the branch probabilities are checked against the Kraus operators of
  quantum.kraus, not against themselves).
* Summing |A(x, r)|^2 over all trajectories gives the density matrix's diagonal (Sec. 2.2, 3.3.1).
* Trajectory samples follow the density matrix's outcome distribution and the branch
  probabilities (chi-square, seeded).
* The compiled TRAJECTORY AC, evaluated by the oracle's AC evaluator, gives |A(x, r)|^2 of the
  state-vector run for every trajectory and outcome tried, and its marginals over the outputs.
"""
import itertools
import math

import numpy as np
import pytest

from oracle import acref as R
from oracle import quantum as Q
from oracle import trajectory as T
from paper_2103_17226_gb300 import inputs as I

MIXED = [("DEP1", 0.3), ("DEP2", 0.4), ("PF", 0.25), ("BF", 0.2)]


def _mixed_circuit(n, n_ops, seed):
    rng = I.SplitMix(seed)
    gates = ["H", "RX", "RY", "RZ", "CNOT", "CZ", "X", "Y"]
    c = I.Circuit(n, 3, name=f"mixed{seed}")
    for _ in range(n_ops):
        g = gates[rng.randint(len(gates))]
        if g in ("CNOT", "CZ"):
            a = rng.randint(n)
            b = (a + 1 + rng.randint(n - 1)) % n
            c.add(g, (a, b))
        else:
            c.add(g, rng.randint(n), angle=rng.randint(3) if g.startswith("R") else -1)
        if rng.uniform() < 0.5:
            ch, p = MIXED[rng.randint(len(MIXED))]
            if ch == "DEP2":
                a = rng.randint(n)
                c.add(ch, (a, (a + 1) % n), p=p)
            else:
                c.add(ch, rng.randint(n), p=p)
    return c


@pytest.mark.parametrize("kind,p", MIXED)
def test_branch_probabilities_are_the_kraus_weights(kind, p):
    """E_k^dagger E_k = p_k I for each Kraus operator of the channel."""
    ks = Q.kraus(kind, p)
    pr = T.branch_probabilities(kind, p)
    assert len(ks) == len(pr) and abs(sum(pr) - 1) < 1e-15
    for E, w in zip(ks, pr):
        assert np.allclose(E.conj().T @ E, w * np.eye(E.shape[0]), atol=1e-15)


@pytest.mark.parametrize("seed", range(3))
def test_trajectory_norms_and_sum_equal_density_matrix(seed):
    c = _mixed_circuit(3, 7, 300 + seed)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    chs = T.channels(c)
    cards = [len(T.branch_probabilities(o.kind, o.p)) for o in chs]
    total = np.zeros(2 ** c.n_qubits)
    for r in itertools.product(*[range(k) for k in cards]):
        prob = np.abs(Q.statevector(c, ang, list(r)).reshape(-1)) ** 2
        want = math.prod(T.branch_probabilities(o.kind, o.p)[k] for o, k in zip(chs, r))
        assert abs(prob.sum() - want) < 1e-13
        total += prob
    assert np.allclose(total, Q.probabilities(c, ang), atol=1e-13)


def test_trajectory_samples_follow_the_density_matrix():
    from scipy.stats import chisquare
    c = _mixed_circuit(3, 8, 311)
    ang = I.uniform_angles(1, c.n_angles, seed=3)[0]
    S = 6000
    bits, trajs = T.trajectory_samples(c, ang, seed=12345, shots=S, with_trajectories=True)
    P = Q.probabilities(c, ang)
    cnt = np.bincount(bits.astype(np.int64), minlength=P.size).astype(float)
    keep = P * S > 5
    e = P[keep] * S
    assert chisquare(cnt[keep] * e.sum() / cnt[keep].sum(), e).pvalue > 0.01
    # branch frequencies of every channel against its branch probabilities
    for i, op in enumerate(T.channels(c)):
        pr = np.array(T.branch_probabilities(op.kind, op.p))
        f = np.bincount([t[i] for t in trajs], minlength=len(pr)).astype(float)
        k2 = pr * S > 5
        assert chisquare(f[k2] * (pr[k2] * S).sum() / f[k2].sum(), pr[k2] * S).pvalue > 0.01


def test_trajectory_sampler_planted_mistake_is_caught():
    """Drawing the branches from the qubit stream (seed instead of ~seed) changes the samples."""
    c = _mixed_circuit(3, 8, 312)
    ang = I.uniform_angles(1, c.n_angles, seed=4)[0]
    good = [T.draw_trajectory(c, 99, s) for s in range(200)]
    chs = T.channels(c)
    bad = []
    for s in range(200):
        r = []
        for i, op in enumerate(chs):
            u = (Q.splitmix64(99, s * len(chs) + i + 1) >> 11) * (1.0 / 9007199254740992.0)
            acc, pick = 0.0, len(T.branch_probabilities(op.kind, op.p)) - 1
            for k, w in enumerate(T.branch_probabilities(op.kind, op.p)[:-1]):
                acc += w
                if u < acc:
                    pick = k
                    break
            r.append(pick)
        bad.append(r)
    assert good != bad


@pytest.fixture(scope="module")
def _lib(native_lib):
    return native_lib


@pytest.mark.parametrize("seed", range(4))
def test_trajectory_ac_equals_statevector_per_trajectory(_lib, seed):
    from paper_2103_17226_gb300 import native as N
    c = _mixed_circuit(3 + seed % 2, 8, 320 + seed)
    n = c.n_qubits
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    b = N.compile(c, N.QKC_AC_TRAJECTORY)
    ref = R.ACRef(b)
    chs = T.channels(c)
    cards = [len(T.branch_probabilities(o.kind, o.p)) for o in chs]
    assert ref.kind == 3 and ref.n_vars == n + len(chs)
    rng = I.SplitMix(77 + seed)
    for _ in range(6):
        r = [rng.randint(k) for k in cards]
        prob = np.abs(Q.statevector(c, ang, r).reshape(-1)) ** 2
        for x in range(2 ** n):
            ev = [(x >> (n - 1 - j)) & 1 for j in range(n)] + r
            assert abs(ref.up(ang, ev) - prob[x]) < 1e-13
        # outputs free: the trajectory's probability; a prefix: the prefix marginal
        assert abs(ref.up(ang, [-1] * n + r) - prob.sum()) < 1e-13
        pt = prob.reshape((2,) * n)
        assert abs(ref.up(ang, [1] + [-1] * (n - 1) + r) - pt[1].sum()) < 1e-13


def test_trajectory_kind_rejects_damping_channels(_lib):
    from paper_2103_17226_gb300 import native as N
    c = I.Circuit(2, 0).add("H", 0).add("AD", 0, p=0.1)
    with pytest.raises(N.QKCError) as e:
        N.compile(c, N.QKC_AC_TRAJECTORY)
    assert e.value.status == 1 and "mixed-unitary" in str(e.value)


def test_config2_trajectory_ac_fits():
    """The 10-qubit QAOA p=2 with config-2 noise: the shared-noise density AC's elimination width is
    28 bits; the TRAJECTORY AC's stays near the noise-free circuit's (width <= 16)."""
    from paper_2103_17226_gb300 import native as N
    c = I.workload("qaoa10_3reg_p2")
    e1, w1 = N.plan(c, N.QKC_AC_DENSITY)
    e3, w3 = N.plan(c, N.QKC_AC_TRAJECTORY)
    assert w1 >= 26 and w3 <= 16 and e3 < 1e-3 * e1
