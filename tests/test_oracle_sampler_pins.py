"""CPU pins of the AC oracle's sampler and of compiled ACs at the benchmarked circuit family.

* acref's chain-rule sampler (oac_sample: two upward passes per qubit, Sec. 3.3's exact
  sampling task) draws, index for index, the samples of the density-matrix oracle's chain
  rule on the same uniforms, on noisy circuits of up to 10 qubits.  A wrong uniform index,
  bit order or comparison direction in either fails here.
* The density AC and every root of the light-cone step AC of the noise-free QAOA p=1 on
  random 3-regular graphs (the generator of the 32-qubit workload) give, on random
  prefixes, the conditional marginals P(x_<j) and P(x_<j, X_j = 0) of the state vector
  (Sec. 2.1: P(x) = |<x|psi>|^2) at 16, 18 and 20 qubits.
"""
import numpy as np
import pytest

from oracle import acref as R
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I


@pytest.fixture(scope="module", autouse=True)
def _lib(native_lib):
    return native_lib


def _compile(c, kind):
    from paper_2103_17226_gb300 import native as N
    return N.compile(c, kind)


def _circuits():
    return [
        ("qaoa4_ring_p1", I.workload("qaoa4_ring_p1")),
        ("vqe_ising_3x3_noisy", I.workload("vqe_ising_3x3_noisy")),
        ("hea5_ad_pf", I.hardware_efficient_ansatz(5, 2, I.NOISE_CFG3)),
        ("qaoa8_dep", I.qaoa_maxcut(8, I.random_regular_graph(8, 3, seed=8), 1, [("DEP1", 0.02, "all")])),
        ("qaoa10_cfg2_p1", I.qaoa_maxcut(10, I.random_regular_graph(10, 3, seed=2), 1, I.NOISE_CFG2)),
        ("random6", I.random_circuit(6, 22, seed=950, noise_prob=0.4)),
        ("random7_bf_pd", I.random_circuit(7, 26, seed=951, noise_prob=0.5)),
    ]


def _margin(P_of, seed, n, s, g, r):
    """|u P - p0| / P at the first qubit where two sample indices differ (for a report)."""
    gb = [(int(g) >> (n - 1 - j)) & 1 for j in range(n)]
    rb = [(int(r) >> (n - 1 - j)) & 1 for j in range(n)]
    j = next(k for k in range(n) if gb[k] != rb[k])
    P, p0 = P_of(rb[:j])
    return abs(Q.sample_uniform(seed, s, j, n) * P - p0) / P


@pytest.mark.parametrize("name,c", _circuits(), ids=[n for n, _ in _circuits()])
def test_acref_sampler_equals_density_matrix_chain_rule(name, c):
    n = c.n_qubits
    shots = 1000
    ang = I.uniform_angles(1, c.n_angles, seed=len(name))[0]
    seed = int(I.vector_seeds(1, len(name) + 3)[0])
    ref = R.ACRef(_compile(c, 1))
    got = ref.sample(ang, seed, shots)
    P = Q.probabilities(c, ang)
    want = Q.chain_rule_samples(P, seed, shots)
    Pt = P.reshape((2,) * n)

    def P_of(prefix):
        a = Pt[tuple(prefix)] if prefix else Pt
        return float(a.sum()), float(a[0].sum())

    diff = [s for s in range(shots) if got[s] != want[s]]
    # FP64 on both sides: a difference may only come from a decision within rounding of a tie
    assert all(_margin(P_of, seed, n, s, got[s], want[s]) < 1e-12 for s in diff)
    assert len(diff) == 0, diff[:5]
    # and the draws are not degenerate: several distinct outcomes, none outside the support
    assert len(set(int(x) for x in got)) > 1
    assert all(P[int(x)] > 0 for x in got)


def test_acref_sampler_planted_mistakes_are_caught():
    """Two plausible slips (uniforms of sample s taken at k = s*n + j, i.e. one off; bits read in
    the reverse qubit order) change the samples of the density-matrix chain rule: the pin above
    would see either."""
    c = I.workload("qaoa4_ring_p1")
    n = c.n_qubits
    ang = I.uniform_angles(1, c.n_angles, seed=2)[0]
    seed = 1234567
    P = Q.probabilities(c, ang)
    want = Q.chain_rule_samples(P, seed, 400)
    Pt = P.reshape((2,) * n)

    def sample(off_by_one, reverse):
        out = []
        for s in range(400):
            bits = []
            for j in range(n):
                a = Pt[tuple(bits)] if bits else Pt
                Pp, p0 = float(a.sum()), float(a[0].sum())
                k = s * n + j + (0 if off_by_one else 1)
                u = (Q.splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0)
                bits.append(1 if u * Pp >= p0 else 0)
            if reverse:
                bits = bits[::-1]
            x = 0
            for b in bits:
                x = (x << 1) | b
            out.append(x)
        return np.array(out, dtype=np.uint64)

    assert np.array_equal(sample(False, False), want)
    assert not np.array_equal(sample(True, False), want)
    assert not np.array_equal(sample(False, True), want)


def _prefixes(n, count, seed):
    rng = I.SplitMix(seed)
    out = [[]]
    while len(out) < count:
        L = 1 + rng.randint(n - 1)
        out.append([rng.randint(2) for _ in range(L)])
    return out


def _steps_roots(b):
    h = np.frombuffer(b[:64], dtype="<u4")
    nv, N, E, D, nl = int(h[5]), int(h[6]), int(h[7]), int(h[8]), int(h[9])
    off = 64
    for nbytes in (4 * nv, 4 * nv, 4 * (D + 1), N, 4 * (N + 1), 4 * E, 4 * nl, 4 * nl, 16 * nl):
        off = (off + nbytes + 7) & ~7
    return np.frombuffer(b, dtype="<u4", count=int(h[12]), offset=off)


@pytest.mark.parametrize("n", [16, 18, 20])
def test_compiled_qaoa_acs_equal_statevector_conditionals(n):
    """Noise-free QAOA p=1 on a random 3-regular graph (the 32-qubit workload's generator and
    seed): on 60 random prefixes x_<j, the density AC gives P(x_<j) and P(x_<j, X_j = 0), and
    root j of the light-cone step AC (root j - 1 for P) gives the same, all equal to the sums of
    |psi(x)|^2 of the state vector (absolute 1e-12, relative 1e-10)."""
    c = I.qaoa_maxcut(n, I.random_regular_graph(n, 3, seed=5), 1, None)
    den = R.ACRef(_compile(c, 1))
    b2 = _compile(c, 2)
    steps = R.ACRef(b2)
    roots = _steps_roots(b2)
    for vec, ang in enumerate(I.uniform_angles(2, c.n_angles, seed=n)):
        prob = np.abs(Q.statevector(c, ang)) ** 2
        prob = prob.reshape((2,) * n)
        for pre in _prefixes(n, 30, seed=100 * n + vec):
            j = len(pre)
            a = prob[tuple(pre)] if pre else prob
            P, p0 = float(a.sum()), float(a[0].sum())
            ev = list(pre) + [-1] * (n - j)
            ev0 = list(pre) + [0] + [-1] * (n - j - 1)
            got_P = den.up(ang, ev)
            got_p0 = den.up(ang, ev0)
            for got, want in ((got_P, P), (got_p0, p0)):
                assert abs(got - want) < 1e-12 and abs(got - want) <= 1e-10 * want + 1e-300, (pre, got, want)
            steps.up(ang, ev0)
            got_s0 = steps.values()[roots[j]]
            assert abs(got_s0 - p0) < 1e-12 and abs(got_s0 - p0) <= 1e-10 * p0 + 1e-300
            if j:
                steps.up(ang, ev)
                got_sP = steps.values()[roots[j - 1]]
                assert abs(got_sP - P) < 1e-12 and abs(got_sP - P) <= 1e-10 * P + 1e-300
