"""CPU tests: the oracle's AC evaluator against closed forms, then the compiler
(circuit -> BN -> AC) against the ground-truth simulators, through that evaluator."""
import itertools
import math

import numpy as np
import pytest

from oracle import acref as R
from oracle import bn as B
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I
from tests import acbytes

# ---------------------------------------------------------------- acref on a hand-built AC
EVS = [(-1, -1), (0, -1), (1, 0), (-1, 1), (-2, -1), (0, -2), (1, 1)]


def lam_of(ev):
    return [list(Q.indicator_vectors([e])[0]) for e in ev]


@pytest.mark.parametrize("ev", EVS)
def test_acref_closed_form(ev):
    r = R.ACRef(acbytes.toy_ac())
    ang = [0.8, 2.9]
    lam = lam_of(ev)
    assert abs(r.up(ang, ev) - acbytes.toy_value(ang, lam)) < 1e-15
    root, adj = r.marginals(ang, ev)
    dl, dt0, dt1 = acbytes.toy_derivatives(ang, lam)
    assert np.allclose(adj, dl, atol=1e-15)
    val, grad = r.gradient(ang, ev, weight=0.7)
    assert abs(val - 0.7 * acbytes.toy_value(ang, lam).real) < 1e-15
    assert abs(grad[0] - 0.7 * dt0.real) < 1e-15 and abs(grad[1] - 0.7 * dt1.real) < 1e-15


def test_acref_multilinearity():
    """Indicator adjoint = f(lambda = 1) - f(lambda = 0) for a polynomial linear in each indicator."""
    r = R.ACRef(acbytes.toy_ac())
    ang = [1.3, 0.4]
    _, adj = r.marginals(ang, [-1, -1])
    for i, (var, val) in enumerate([(0, 0), (0, 1), (1, 0), (1, 1)]):
        lam1 = [[1.0, 1.0], [1.0, 1.0]]
        lam0 = [[1.0, 1.0], [1.0, 1.0]]
        lam0[var][val] = 0.0
        assert abs(adj[i] - (acbytes.toy_value(ang, lam1) - acbytes.toy_value(ang, lam0))) < 1e-15


# ---------------------------------------------------------------- compiler
def compile_ac(c, kind=1, order=0, max_nodes=0):
    from paper_2103_17226_gb300 import native as N
    return N.compile(c, kind, order, max_nodes)


def outcome_ev(x, n):
    return [(x >> (n - 1 - j)) & 1 for j in range(n)]


@pytest.fixture(scope="module", autouse=True)
def _lib(native_lib):
    return native_lib


def test_compiled_noisy_bell_matches_paper():
    c = I.noisy_bell(0.36)
    amp = R.ACRef(compile_ac(c, kind=0))
    s2 = math.sqrt(2)
    table5 = {(0, 0, 0): 1 / s2, (0, 1, 1): 0.8 / s2, (1, 1, 1): -0.6 / s2}
    for rv, q0, q1 in itertools.product((0, 1), repeat=3):
        assert abs(amp.up([], [q0, q1, rv]) - table5.get((rv, q0, q1), 0.0)) < 1e-15
    den = R.ACRef(compile_ac(c, kind=1))
    for x, p in enumerate([0.5, 0, 0, 0.5]):
        assert abs(den.up([], outcome_ev(x, 2)) - p) < 1e-15


@pytest.mark.parametrize("seed", range(8))
def test_density_ac_equals_density_matrix(seed):
    n = 3 + seed % 2
    c = I.random_circuit(n, 9 + seed, seed=400 + seed, noise_prob=0.4)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    P = Q.probabilities(c, ang)
    r = R.ACRef(compile_ac(c, kind=1))
    for x in range(2 ** n):
        assert abs(r.up(ang, outcome_ev(x, n)) - P[x]) < 1e-13
    rng = I.SplitMix(seed)
    for _ in range(6):
        ev = [rng.randint(4) - 2 for _ in range(n)]  # -2 Z sign, -1 free, 0, 1
        assert abs(r.up(ang, ev) - Q.density_evidence(P, ev)) < 1e-13
        root, adj = r.marginals(ang, ev)
        m = Q.density_marginals(P, ev)
        assert np.allclose(adj.reshape(n, 2), m, atol=1e-13)
    assert abs(r.up(ang, [-1] * n) - 1.0) < 1e-13  # trace


@pytest.mark.parametrize("seed", range(5))
def test_amplitude_ac_equals_trajectory_amplitudes(seed):
    c = I.random_circuit(3, 7, seed=500 + seed, noise_prob=0.5)
    ang = I.uniform_angles(1, c.n_angles, seed=seed)[0]
    r = R.ACRef(compile_ac(c, kind=0))
    cards = Q.channel_cards(c)
    rng = I.SplitMix(77 + seed)
    for _ in range(8):
        ev_x = [rng.randint(3) - 1 for _ in range(3)]
        ev_r = [rng.randint(k + 1) - 1 if rng.uniform() < 0.4 else rng.randint(k) for k in cards]
        want = Q.amplitude_evidence(c, ang, ev_x, ev_r)
        assert abs(r.up(ang, ev_x + ev_r) - want) < 1e-13
        assert abs(B.amplitude_evidence(c, ang, ev_x, ev_r) - want) < 1e-13


def test_noise_free_acs_equal_statevector():
    c = I.qaoa_maxcut(5, [(0, 1), (1, 2), (2, 3), (3, 4), (0, 4)], 2)
    ang = I.uniform_angles(1, c.n_angles, seed=9)[0]
    psi = Q.statevector(c, ang).reshape(-1)
    amp = R.ACRef(compile_ac(c, kind=0))
    den = R.ACRef(compile_ac(c, kind=1))
    for x in range(32):
        ev = outcome_ev(x, 5)
        assert abs(amp.up(ang, ev) - psi[x]) < 1e-13
        assert abs(den.up(ang, ev) - abs(psi[x]) ** 2) < 1e-13


def test_qaoa4_workload_all_vectors():
    c = I.workload("qaoa4_ring_p1")
    r = R.ACRef(compile_ac(c, kind=1))
    for a in I.uniform_angles(4, c.n_angles, seed=1):
        P = Q.probabilities(c, a)
        for x in range(16):
            assert abs(r.up(a, outcome_ev(x, 4)) - P[x]) < 1e-13


def test_gradient_through_ac_equals_oracle_gradient():
    c = I.hardware_efficient_ansatz(3, 2, I.NOISE_CFG3)
    ang = I.uniform_angles(1, c.n_angles, seed=21)[0]
    sup, coef = I.z_string_hamiltonian(3, 3, seed=21)
    val, grad = Q.hamiltonian_value_and_gradient(c, ang, sup, coef)
    r = R.ACRef(compile_ac(c, kind=1))
    v_ac, g_ac = 0.0, np.zeros(c.n_angles)
    for s, w in zip(sup, coef):
        v, g = r.gradient(ang, [-2 if b else -1 for b in s], w)
        v_ac += v
        g_ac += g
    assert abs(v_ac - val) < 1e-13
    assert np.abs(g_ac - grad).max() < 1e-12


@pytest.mark.parametrize("order", [1, 2, 3])
def test_elimination_orders_agree(order):
    c = I.random_circuit(4, 12, seed=31, noise_prob=0.3)
    ang = I.uniform_angles(1, c.n_angles, seed=31)[0]
    P = Q.probabilities(c, ang)
    r = R.ACRef(compile_ac(c, kind=1, order=order))
    for x in range(16):
        assert abs(r.up(ang, outcome_ev(x, 4)) - P[x]) < 1e-13


def test_compile_is_deterministic_and_well_formed():
    from paper_2103_17226_gb300 import native as N
    c = I.workload("qaoa4_ring_p1")
    b1, b2 = compile_ac(c), compile_ac(c)
    assert b1 == b2
    h = N.header(b1)
    r = R.ACRef(b1)
    assert r.n_ind == 2 * 4 and h["n_vars"] == 4
    # structure: level-sorted, children on lower levels, MUL binary, root alone on the top level
    import struct
    off = 64
    def arr(dt, cnt):
        nonlocal off
        off = (off + 7) // 8 * 8
        a = np.frombuffer(b1, dtype=dt, count=cnt, offset=off)
        off += a.nbytes
        return a
    nv, N_, E, D = h["n_vars"], h["n_nodes"], h["n_edges"], h["n_levels"]
    arr("<u4", nv); arr("<i4", nv)
    lo = arr("<u4", D + 1); op = arr("u1", N_); co = arr("<u4", N_ + 1); ch = arr("<u4", E)
    lev = np.zeros(N_, dtype=int)
    for l in range(D):
        lev[lo[l]:lo[l + 1]] = l
    for i in range(h["n_leaves"], N_):
        kids = ch[co[i]:co[i + 1]]
        assert (lev[kids] < lev[i]).all()
        if op[i] == 4:
            assert len(kids) == 2
    assert lo[D - 1] + 1 == lo[D] == N_ and h["root"] == N_ - 1
    assert (op[:h["n_ind"]] == 0).all()


def test_compile_rejects_bad_circuits():
    from paper_2103_17226_gb300 import native as N
    bad = I.Circuit(2, 1).add("RX", 0, angle=3)  # angle slot out of range
    with pytest.raises(N.QKCError) as e:
        compile_ac(bad)
    assert e.value.status == 1 and "operation 0" in str(e.value)
    with pytest.raises(N.QKCError):
        compile_ac(I.Circuit(2, 0).add("CNOT", (1, 1)))
    with pytest.raises(N.QKCError) as e:
        compile_ac(I.workload("qaoa4_ring_p1"), max_nodes=50)
    assert e.value.status == 7


def test_plan_reports_sizes():
    from paper_2103_17226_gb300 import native as N
    entries, width = N.plan(I.workload("qaoa4_ring_p1"))
    assert entries > 100 and 2 <= width <= 12


def test_ctx_create_fails_cleanly_without_gpu():
    import torch
    from paper_2103_17226_gb300 import native as N
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(N.QKCError) as e:
        N.Context(0)
    assert e.value.status in (1, 4)


def test_vqe_ising_density_ac_equals_density_matrix():
    """The 2D-Ising VQE family (3x3 grid, 2 layers, depolarising 0.5% after every gate):
    outcome probabilities and <H> through the compiled density AC vs the density matrix."""
    c = I.workload("vqe_ising_3x3_noisy")
    sup, coef = I.ising_hamiltonian(3, 3)
    r = R.ACRef(compile_ac(c, kind=1))
    for a in I.uniform_angles(2, c.n_angles, seed=23):
        P = Q.probabilities(c, a)
        rng = I.SplitMix(23)
        for _ in range(12):
            x = rng.randint(2 ** 9)
            assert abs(r.up(a, outcome_ev(x, 9)) - P[x]) < 1e-13
        val = sum(w * Q.z_expectation(P, s) for s, w in zip(sup, coef))
        got = sum(r.gradient(a, [-2 if b else -1 for b in s], w)[0] for s, w in zip(sup, coef))
        assert abs(got - val) < 1e-12


def steps_roots(b: bytes):
    """The roots table of a light-cone-steps AC (its layout is documented in include/qkc.h)."""
    h = np.frombuffer(b[:64], dtype="<u4")
    nv, N, E, D, nl = int(h[5]), int(h[6]), int(h[7]), int(h[8]), int(h[9])
    off = 64
    for nbytes in (4 * nv, 4 * nv, 4 * (D + 1), N, 4 * (N + 1), 4 * E, 4 * nl, 4 * nl, 16 * nl):
        off = (off + nbytes + 7) & ~7
    return np.frombuffer(b, dtype="<u4", count=int(h[12]), offset=off), int(h[10])


@pytest.mark.parametrize("seed", range(4))
def test_light_cone_step_roots_are_marginals(seed):
    """Root j of a light-cone-steps AC, evaluated with qubits < j fixed, qubit j fixed and the rest
    free, equals the marginal of qubits <= j of the density matrix of the whole circuit."""
    n = 4 + seed % 3
    c = (I.workload("qaoa4_ring_p1") if seed == 0 else
         I.random_circuit(n, 14 + 3 * seed, seed=900 + seed, noise_prob=0.4))
    n = c.n_qubits
    ang = I.uniform_angles(1, c.n_angles, seed=seed + 3)[0]
    P = Q.probabilities(c, ang)
    b = compile_ac(c, kind=2)
    roots, root = steps_roots(b)
    assert len(roots) == n and roots[-1] == root
    r = R.ACRef(b)
    full = R.ACRef(compile_ac(c, kind=1))
    rng = I.SplitMix(seed + 11)
    for j in range(n):
        for _ in range(4):
            ev = [rng.randint(2) for _ in range(j + 1)] + [-1] * (n - j - 1)
            r.up(ang, ev)
            got = r.values()[roots[j]]
            assert abs(got - Q.density_evidence(P, ev)) < 1e-13
        # the last root is the whole circuit's AC value
        ev = [rng.randint(2) for _ in range(n)]
        assert abs(r.up(ang, ev) - full.up(ang, ev)) < 1e-13


def test_light_cone_steps_shrink_early_steps():
    """On the 32-qubit QAOA the early steps' light cones give much smaller ACs than the whole circuit."""
    b = compile_ac(I.workload("qaoa32_3reg_p1_ideal"), kind=2)
    roots, _ = steps_roots(b)
    h = np.frombuffer(b[:64], dtype="<u4")
    N, E, D, nv = int(h[6]), int(h[7]), int(h[8]), int(h[5])
    off = 64
    offs = []
    for nbytes in (4 * nv, 4 * nv, 4 * (D + 1), N, 4 * (N + 1), 4 * E):
        offs.append(off)
        off = (off + nbytes + 7) & ~7
    coff = np.frombuffer(b, dtype="<u4", count=N + 1, offset=offs[4])
    child = np.frombuffer(b, dtype="<u4", count=E, offset=offs[5])

    def reach(r0):
        seen = np.zeros(N, dtype=bool)
        st = [int(r0)]
        seen[r0] = True
        while st:
            v = st.pop()
            for e in range(coff[v], coff[v + 1]):
                cc = int(child[e])
                if not seen[cc]:
                    seen[cc] = True
                    st.append(cc)
        return int(seen.sum())

    sizes = [reach(roots[j]) for j in (0, 8, 14, 31)]
    assert sizes[0] < sizes[1] < sizes[2] < sizes[3]
    assert sizes[2] * 10 < sizes[3]


def test_auto_order_takes_the_order_with_fewer_nodes():
    """The automatic elimination order builds min-fill and min-weight and keeps the one that adds fewer
    nodes (the table-size estimates can be off severalfold): on a 12-qubit noisy QAOA of the serving mix
    it is never larger than either fixed order; a step AC may take either order throughout when that
    saves at least 10%.  The AUTO AC still gives the density matrix's probabilities."""
    from paper_2103_17226_gb300 import native as N
    c = I.qaoa_maxcut(12, I.random_regular_graph(12, 3, seed=52), 1, I.NOISE_CFG2, name="q12")
    size = {o: N.header(compile_ac(c, kind=1, order=o))["n_nodes"] for o in (0, 1, 2)}
    assert size[0] <= min(size[1], size[2]), size
    steps = {o: N.header(compile_ac(c, kind=2, order=o))["n_nodes"] for o in (0, 1, 2)}
    assert steps[0] <= min(steps[1], steps[2]) / 0.9, steps
    c6 = I.random_circuit(6, 24, seed=907, noise_prob=0.4)
    ang = I.uniform_angles(1, c6.n_angles, seed=7)[0]
    P = Q.probabilities(c6, ang)
    r = R.ACRef(compile_ac(c6, kind=1, order=0))
    for x in range(64):
        assert abs(r.up(ang, outcome_ev(x, 6)) - P[x]) < 1e-13
