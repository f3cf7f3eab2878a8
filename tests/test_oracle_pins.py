"""Pins of the oracle against what the paper and the mathematics fix (CPU only).

Each test checks an oracle function against something other than itself: the
numbers the paper prints for its worked example, closed forms, textbook
identities, an independent formulation (density matrix vs state vector vs the
Bayesian-network path sum), or finite differences.  A plausible slip in the
oracle (a transposed table, a dropped conjugate, a wrong sign or index) fails
at least one of them; the last tests plant such slips and check that they do.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

from oracle import bn as B
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

GOLD = json.loads((Path(__file__).parent / "golden" / "noisy_bell.json").read_text())
S2 = math.sqrt(2.0)


def num(x):
    if isinstance(x, (int, float)):
        return float(x)
    x = x.replace("sqrt2", str(S2))
    return float(eval(x, {"__builtins__": {}}))  # printed fractions such as "-0.6/sqrt2"


# ---------------------------------------------------------------- the paper's worked example
def test_cat_tables_match_paper():
    """Tables 3a-3c: CAT rows are inputs, columns outputs (the transpose of the unitary)."""
    h = np.array([[num(v) for v in row] for row in GOLD["cat_hadamard_rows_in_cols_out"]["value"]])
    assert np.allclose(B.cat("H"), h, atol=1e-15)
    pd = B.noise_cat("PD", GOLD["gamma"])  # [k][in][out]; diagonal channel -> A(rv=k | q=i) = E_k[i][i]
    table3b = np.array([[pd[k][i][i].real for k in range(2)] for i in range(2)])
    assert np.allclose(table3b, GOLD["cat_phase_damping_rows_q_cols_rv"]["value"], atol=1e-15)
    cn = B.cat("CNOT")  # rows (control, target) in, columns (control, target) out
    table3c = np.array([[cn[(c << 1) | t][(c << 1) | o].real for o in range(2)] for c in range(2) for t in range(2)])
    assert np.array_equal(table3c, np.array(GOLD["cat_cnot_rows_control_target_cols_out"]["value"], dtype=float))


def test_upward_pass_amplitudes_match_table5():
    c = I.noisy_bell(GOLD["gamma"])
    amps = B.amplitude_table(c, [])
    for rv, q0, q1, a in GOLD["upward_pass_amplitudes"]["value"]:
        got = amps.get(((q0, q1), (rv,)), 0j)
        assert abs(got - num(a)) < 1e-15, (rv, q0, q1, got)


def test_density_components_and_final_rho_match_paper():
    c = I.noisy_bell(GOLD["gamma"])
    amps = B.amplitude_table(c, [])
    for rv, key in ((0, "density_component_rv0"), (1, "density_component_rv1")):
        psi = np.zeros(4, dtype=complex)
        for (x, r), a in amps.items():
            if r == (rv,):
                psi[(x[0] << 1) | x[1]] = a
        assert np.allclose(np.outer(psi, psi.conj()), GOLD[key]["value"], atol=1e-15)
    rho = Q.density_matrix(c, [])
    assert np.allclose(rho, GOLD["final_rho"]["value"], atol=1e-15)
    # intermediate state after the phase damping channel on q0 alone
    c1 = I.Circuit(1, 0).add("H", 0).add("PD", 0, p=GOLD["gamma"])
    assert np.allclose(Q.density_matrix(c1, []), GOLD["rho_q0m2_after_pd"]["value"], atol=1e-15)


# ---------------------------------------------------------------- textbook identities
@pytest.mark.parametrize("kind,p", [("DEP1", 0.07), ("DEP2", 0.13), ("AD", 0.3), ("PD", 0.36), ("PF", 0.2),
                                    ("BF", 0.1)])
def test_kraus_completeness(kind, p):
    ks = Q.kraus(kind, p)
    d = ks[0].shape[0]
    assert np.allclose(sum(E.conj().T @ E for E in ks), np.eye(d), atol=1e-14)


def test_gates_unitary_and_closed_forms():
    for k in ("H", "X", "Y", "Z", "CNOT", "CZ"):
        U = Q.gate_matrix(k)
        assert np.allclose(U.conj().T @ U, np.eye(U.shape[0]))
    for k in ("RX", "RY", "RZ"):
        U = Q.gate_matrix(k, 0.7)
        assert np.allclose(U.conj().T @ U, np.eye(2))
    # RX(t)|0>: P(1) = sin^2(t/2); RY likewise; RZ leaves populations alone
    for t in (0.3, 1.9, 4.4):
        c = I.Circuit(1, 1).add("RX", 0, angle=0)
        assert abs(Q.probabilities(c, [t])[1] - math.sin(t / 2) ** 2) < 1e-15
        c = I.Circuit(1, 1).add("RY", 0, angle=0)
        assert abs(Q.probabilities(c, [t])[1] - math.sin(t / 2) ** 2) < 1e-15
    # RY(t)|0> = cos(t/2)|0> + sin(t/2)|1>  (a sign slip in RY flips the amplitude)
    c = I.Circuit(1, 1).add("RY", 0, angle=0)
    assert np.allclose(Q.statevector(c, [1.1]), [math.cos(0.55), math.sin(0.55)])
    # RZ phase: H RZ(t) H |0> gives P(1) = sin^2(t/2)
    c = I.Circuit(1, 1).add("H", 0).add("RZ", 0, angle=0).add("H", 0)
    assert abs(Q.probabilities(c, [1.3])[1] - math.sin(0.65) ** 2) < 1e-15
    # CNOT control is the first qubit: X on q0 then CNOT(0,1) -> |11>; X on q1 then CNOT(0,1) -> |01>
    assert Q.probabilities(I.Circuit(2, 0).add("X", 0).add("CNOT", (0, 1)), [])[3] == pytest.approx(1.0)
    assert Q.probabilities(I.Circuit(2, 0).add("X", 1).add("CNOT", (0, 1)), [])[1] == pytest.approx(1.0)
    # qubit 0 is the most significant bit
    assert Q.probabilities(I.Circuit(3, 0).add("X", 0), [])[4] == pytest.approx(1.0)


def test_channel_closed_forms():
    # amplitude damping of |1>: P(1) = 1 - gamma; depolarising of |0>: P(1) = 2p/3
    c = I.Circuit(1, 0).add("X", 0).add("AD", 0, p=0.3)
    assert abs(Q.probabilities(c, [])[1] - 0.7) < 1e-15
    c = I.Circuit(1, 0).add("DEP1", 0, p=0.09)
    assert abs(Q.probabilities(c, [])[1] - 0.06) < 1e-15
    # phase flip on |+>: off-diagonal 1/2 (1 - 2p); two-qubit depolarising of |00>: P(00) = 1 - 12p/15 ... =
    # 1 - p + p/15 * 3 (the Pauli products with only Z's leave |00> alone: IZ, ZI, ZZ)
    c = I.Circuit(1, 0).add("H", 0).add("PF", 0, p=0.2)
    assert abs(Q.density_matrix(c, [])[0, 1] - 0.5 * 0.6) < 1e-15
    c = I.Circuit(2, 0).add("DEP2", (0, 1), p=0.15)
    assert abs(Q.probabilities(c, [])[0] - (1 - 0.15 + 3 * 0.15 / 15)) < 1e-15
    # Y error carries an i: Y|0> = i|1>, and Y rho Y^dagger keeps rho Hermitian with trace 1
    c = I.Circuit(1, 0).add("H", 0).add("DEP1", 0, p=0.3).add("RX", 0, angle=-1)
    rho = Q.density_matrix(I.Circuit(1, 0).add("H", 0).add("DEP1", 0, p=0.3), [])
    assert np.allclose(rho, rho.conj().T) and abs(np.trace(rho) - 1) < 1e-15
    # depolarising shrinks the Bloch vector by (1 - 4p/3)
    assert abs(rho[0, 1] - 0.5 * (1 - 4 * 0.3 / 3)) < 1e-15


@pytest.mark.parametrize("seed", range(6))
def test_density_matrix_properties(seed):
    c = I.random_circuit(3, 10, seed=seed)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    rho = Q.density_matrix(c, ang)
    assert abs(np.trace(rho) - 1) < 1e-13
    assert np.allclose(rho, rho.conj().T, atol=1e-14)
    assert np.linalg.eigvalsh(rho).min() > -1e-13


@pytest.mark.parametrize("seed", range(4))
def test_noise_free_dm_equals_statevector(seed):
    c = I.random_circuit(4, 14, seed=100 + seed, noise_prob=0.0)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    psi = Q.statevector(c, ang).reshape(-1)
    rho = Q.density_matrix(c, ang)
    assert np.allclose(rho, np.outer(psi, psi.conj()), atol=1e-14)
    assert abs(np.trace(rho @ rho) - 1) < 1e-13  # purity


@pytest.mark.parametrize("seed", range(5))
def test_dm_equals_bn_path_sum(seed):
    """Noisy outcome distribution two ways: Kraus evolution of rho vs the paper's
    BN encoding with noise random variables, P(x) = sum_r |A(x, r)|^2."""
    c = I.random_circuit(3, 6, seed=200 + seed, noise_prob=0.5)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    P = Q.probabilities(c, ang)
    for x in range(8):
        ev = [(x >> 2) & 1, (x >> 1) & 1, x & 1]
        assert abs(B.density_evidence(c, ang, ev) - P[x]) < 1e-13


@pytest.mark.parametrize("seed", range(4))
def test_trajectory_amplitude_equals_bn_path_sum(seed):
    c = I.random_circuit(3, 6, seed=300 + seed, noise_prob=0.5)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    cards = Q.channel_cards(c)
    rng = I.SplitMix(seed)
    for _ in range(4):
        ev_x = [rng.randint(3) - 1 for _ in range(3)]
        ev_r = [rng.randint(k + 1) - 1 for k in cards]
        assert abs(Q.amplitude_evidence(c, ang, ev_x, ev_r) - B.amplitude_evidence(c, ang, ev_x, ev_r)) < 1e-13


def test_evidence_polynomial_definitions():
    c = I.random_circuit(3, 8, seed=7)
    ang = I.uniform_angles(1, c.n_angles, seed=7)[0]
    P = Q.probabilities(c, ang)
    assert abs(Q.density_evidence(P, [-1, -1, -1]) - 1) < 1e-13
    # a marginal is the brute-force sum over the free qubits
    assert abs(Q.density_evidence(P, [1, -1, 0]) - (P[0b100] + P[0b110])) < 1e-15
    # Z sign: <Z_0 Z_2> = sum_x (-1)^(x0 + x2) P(x)
    zz = sum(((-1) ** (((x >> 2) & 1) + (x & 1))) * P[x] for x in range(8))
    assert abs(Q.density_evidence(P, [-2, -1, -2]) - zz) < 1e-15
    # marginals: multilinearity, f(e) = sum_v d f / d lambda_{j,v} for a free X_j, and the observed case
    m = Q.density_marginals(P, [-1, 0, -1])
    for j in (0, 2):
        assert abs(m[j].sum() - Q.density_evidence(P, [-1, 0, -1])) < 1e-15
    assert abs(m[0, 1] - (P[0b100] + P[0b101])) < 1e-15
    assert abs(m[1, 1] - (P[0b010] + P[0b011] + P[0b110] + P[0b111])) < 1e-15


def test_gradient_forward_mode_vs_finite_differences_and_shift_rule():
    c = I.hardware_efficient_ansatz(3, 2, I.NOISE_CFG3)
    ang = I.uniform_angles(1, c.n_angles, seed=11)[0]
    sup, coef = I.z_string_hamiltonian(3, 4, seed=11)
    val, grad = Q.hamiltonian_value_and_gradient(c, ang, sup, coef)

    def H(a):
        P = Q.probabilities(c, a)
        return sum(cf * Q.z_expectation(P, s) for s, cf in zip(sup, coef))

    assert abs(val - H(ang)) < 1e-14
    h = 1e-5
    for k in range(c.n_angles):
        e = np.zeros_like(ang)
        e[k] = h
        fd = (H(ang + e) - H(ang - e)) / (2 * h)
        assert abs(fd - grad[k]) < 1e-8
        # parameter-shift rule, exact for a gate exp(-i t P / 2) whose angle appears once
        e[k] = math.pi / 2
        ps = (H(ang + e) - H(ang - e)) / 2
        assert abs(ps - grad[k]) < 1e-12


def test_chain_rule_sampler_distribution():
    c = I.workload("qaoa4_ring_p1")
    ang = I.uniform_angles(1, c.n_angles, seed=3)[0]
    P = Q.probabilities(c, ang)
    shots = 20000
    bits = Q.chain_rule_samples(P, seed=12345, shots=shots)
    counts = np.bincount(bits.astype(np.int64), minlength=16)
    from scipy.stats import chisquare
    keep = P * shots > 5
    exp = P[keep] * shots
    obs = counts[keep].astype(float)
    obs = obs * exp.sum() / obs.sum()
    assert chisquare(obs, exp).pvalue > 0.01
    # the decision rule itself: with a point mass every sample is that outcome
    Pm = np.zeros(16)
    Pm[0b1010] = 1.0
    assert set(Q.chain_rule_samples(Pm, 1, 50).tolist()) == {0b1010}


def test_splitmix64_published_value():
    # first output of SplitMix64 seeded with 0 (Steele, Lea, Flood 2014 reference stream)
    assert Q.splitmix64(0, 1) == 0xE220A8397B1DCDAF
    assert I.splitmix64(0, 1) == 0xE220A8397B1DCDAF


# ---------------------------------------------------------------- planted mistakes are caught
def test_planted_untransposed_cat_is_caught(monkeypatch):
    monkeypatch.setattr(B, "cat", lambda kind, theta=None: Q.gate_matrix(kind, theta).copy())
    c = I.Circuit(1, 1).add("RY", 0, angle=0)
    # RY is not symmetric, so using U instead of U^T in the table changes the amplitude
    amps = B.amplitude_table(c, [0.9])
    assert abs(amps[((1,), ())] - math.sin(0.45)) > 0.5


def test_planted_transpose_instead_of_dagger_is_caught(monkeypatch):
    c = I.Circuit(1, 0).add("H", 0).add("RX", 0, angle=-1)
    good = Q.density_matrix(I.Circuit(1, 0).add("H", 0).add("DEP1", 0, p=0.3), [])
    real_apply = Q._apply_rho

    def wrong(rho, n, mat, qubits):  # E rho E^T instead of E rho E^dagger
        r = Q._apply_ket(rho, mat, list(qubits))
        return Q._apply_ket(r, mat, [n + q for q in qubits])

    monkeypatch.setattr(Q, "_apply_rho", wrong)
    bad = Q.density_matrix(I.Circuit(1, 0).add("H", 0).add("DEP1", 0, p=0.3), [])
    monkeypatch.setattr(Q, "_apply_rho", real_apply)
    assert abs(bad[0, 1] - good[0, 1]) > 0.05  # the Y Kraus operator is complex: caught by the closed form


def test_gibbs_oracle_kernel_has_the_noisy_distribution_as_stationary_law():
    """The oracle's Gibbs update (Sec. 3.3.2): with a uniform u, variable V moves to v with
    probability |A(., V=v)|^2 / sum_w |A(., V=w)|^2.  The product of one update per variable
    (a sweep) must leave pi(x, r) = |A(x, r)|^2 / Z invariant, and the x-marginal of pi must be
    the density-matrix distribution."""
    import itertools
    from oracle import gibbs as G
    c = I.Circuit(2, 1).add("H", 0).add("DEP1", 0, p=0.2).add("CNOT", (0, 1)).add("RY", 1, angle=0)
    c.add("AD", 1, p=0.3)
    ang = [0.7]
    cards = [2, 2] + Q.channel_cards(c)
    states = list(itertools.product(*[range(k) for k in cards]))
    idx = {s: i for i, s in enumerate(states)}
    pi = np.zeros(len(states))
    for s in states:
        psi = Q.statevector(c, ang, list(s[2:]))
        pi[idx[s]] = abs(psi[s[0], s[1]]) ** 2
    pi /= pi.sum()
    T = np.eye(len(states))
    for var in range(len(cards)):
        Tv = np.zeros_like(T)
        for s in states:
            w = G.candidate_weights(c, ang, list(s), var)
            if w.sum() == 0:
                Tv[idx[s], idx[s]] = 1.0
                continue
            for v, wv in enumerate(w):
                s2 = list(s)
                s2[var] = v
                Tv[idx[s], idx[tuple(s2)]] += wv / w.sum()
        T = T @ Tv
    assert np.abs(pi @ T - pi).max() < 1e-14
    P = Q.probabilities(c, ang)
    marg = np.zeros(4)
    for s in states:
        marg[s[0] * 2 + s[1]] += pi[idx[s]]
    assert np.abs(marg - P).max() < 1e-14
