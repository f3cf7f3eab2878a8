"""GPU parity: the CUDA path (through the C-ABI) against the oracle.

Tolerances: FP64 path 1e-12 absolute per probability / marginal, FP32 path
1e-5 absolute per probability (values of magnitude <= 1); gradients and
Hamiltonian values scale the same bounds by sum_t |c_t|.  Sample indices:
bit-exact, except where the oracle shows the decision u * P vs p0 sits within
the tie margin (1e-12 relative in FP64, 1e-5 relative in FP32).
"""
import math
import os

import numpy as np
import pytest

from oracle import acref as R
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda"
TOL = {64: 1e-12, 32: 1e-5}
TIE = {64: 1e-12, 32: 1e-5}


def N():
    from paper_2103_17226_gb300 import native
    return native


def t(x, dtype=None):
    return torch.tensor(np.asarray(x), device=DEV, dtype=dtype)


def outcome_evidence(n):
    return np.array([[(x >> (n - 1 - j)) & 1 for j in range(n)] for x in range(2 ** n)], dtype=np.int8)


def load(ctx, c, kind=1, prec=32):
    return N().load_ac(ctx, N().compile(c, kind), precision=prec)


_cache = {}


def compiled(name, kind=1):
    key = (name, kind)
    if key not in _cache:
        _cache[key] = N().compile(I.workload(name), kind)
    return _cache[key]


def mismatch_margins(prob_prefix, seed, gpu_bits, ref_bits, n):
    """For every sample whose index differs, |u P - p0| / P at the first differing qubit."""
    out = []
    for s, (g, r) in enumerate(zip(gpu_bits, ref_bits)):
        if int(g) == int(r):
            continue
        gb = [(int(g) >> (n - 1 - j)) & 1 for j in range(n)]
        rb = [(int(r) >> (n - 1 - j)) & 1 for j in range(n)]
        j = next(k for k in range(n) if gb[k] != rb[k])
        P, p0 = prob_prefix(rb[:j])
        u = Q.sample_uniform(seed, s, j, n)
        out.append(abs(u * P - p0) / max(P, 1e-300))
    return out


# ---------------------------------------------------------------- hand-built AC: closed form
@pytest.mark.parametrize("prec", [64, 32])
def test_toy_ac_closed_form(cuda_ctx, prec):
    from tests import acbytes
    ac = N().load_ac(cuda_ctx, acbytes.toy_ac(), precision=prec)
    angs = np.array([[0.8, 2.9], [4.1, 0.3], [2.2, 5.5]])
    N().set_params(ac, t(angs))
    evs = [(-1, -1), (0, -1), (1, 0), (-1, 1), (-2, -1), (0, -2), (1, 1)]
    ev = np.array([e for e in evs for _ in range(3)], dtype=np.int8)
    cv = np.array([v for _ in evs for v in range(3)], dtype=np.int32)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    root, marg = N().marginals(ac, t(cv), t(ev))
    w = np.linspace(0.3, 1.7, len(cv))
    val, grad = N().gradient(ac, t(cv), t(ev), t(w), 3)
    marg = marg.cpu().numpy()
    exp_val = np.zeros(3)
    exp_grad = np.zeros((3, 2))
    for c in range(len(cv)):
        lam = [list(Q.indicator_vectors([e])[0]) for e in ev[c]]
        f = acbytes.toy_value(angs[cv[c]], lam)
        assert abs(complex(*out[c]) - f) < TOL[prec] * 10
        dl, d0, d1 = acbytes.toy_derivatives(angs[cv[c]], lam)
        assert np.abs(marg[c, :, 0] + 1j * marg[c, :, 1] - np.array(dl)).max() < TOL[prec] * 10
        exp_val[cv[c]] += w[c] * f.real
        exp_grad[cv[c]] += w[c] * np.array([d0.real, d1.real])
    assert np.abs(val.cpu().numpy() - exp_val).max() < TOL[prec] * 50
    assert np.abs(grad.cpu().numpy() - exp_grad).max() < TOL[prec] * 50


# ---------------------------------------------------------------- upward pass: full distributions
@pytest.mark.parametrize("prec", [64, 32])
def test_qaoa4_full_distribution(cuda_ctx, prec):
    """4-qubit noisy QAOA ring, 16 parameter vectors x all 16 outcomes vs the density matrix."""
    c = I.workload("qaoa4_ring_p1")
    V = 16
    angs = I.uniform_angles(V, c.n_angles, seed=1)
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=prec)
    N().set_params(ac, t(angs))
    ev = np.tile(outcome_evidence(4), (V, 1))
    cv = np.repeat(np.arange(V, dtype=np.int32), 16)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    for v in range(V):
        P = Q.probabilities(c, angs[v])
        assert np.abs(out[v * 16:(v + 1) * 16, 0] - P).max() < TOL[prec]
        assert np.abs(out[v * 16:(v + 1) * 16, 1]).max() < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("seed", range(4))
def test_random_density_evidence_and_marginals(cuda_ctx, prec, seed):
    n = 3 + seed % 3
    c = I.random_circuit(n, 10 + 2 * seed, seed=600 + seed, noise_prob=0.4)
    V = 5
    angs = I.uniform_angles(V, c.n_angles, seed=seed)
    ac = load(cuda_ctx, c, 1, prec)
    N().set_params(ac, t(angs))
    rng = I.SplitMix(seed)
    cols = 70  # more than one 64-column chunk, ragged
    ev = np.array([[rng.randint(4) - 2 for _ in range(n)] for _ in range(cols)], dtype=np.int8)
    cv = np.array([rng.randint(V) for _ in range(cols)], dtype=np.int32)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    root, marg = N().marginals(ac, t(cv), t(ev))
    root, marg = root.cpu().numpy(), marg.cpu().numpy()
    probs = [Q.probabilities(c, a) for a in angs]
    for k in range(cols):
        want = Q.density_evidence(probs[cv[k]], ev[k])
        assert abs(complex(*out[k]) - want) < TOL[prec]
        assert abs(complex(*root[k]) - want) < TOL[prec]
        m = Q.density_marginals(probs[cv[k]], ev[k])
        got = (marg[k, :, 0] + 1j * marg[k, :, 1]).reshape(n, 2)
        assert np.abs(got - m).max() < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_random_amplitude_ac(cuda_ctx, prec):
    c = I.random_circuit(4, 10, seed=700, noise_prob=0.5)
    V = 3
    angs = I.uniform_angles(V, c.n_angles, seed=7)
    ac = load(cuda_ctx, c, 0, prec)
    N().set_params(ac, t(angs))
    cards = Q.channel_cards(c)
    rng = I.SplitMix(70)
    cols = 40
    evx = [[rng.randint(3) - 1 for _ in range(4)] for _ in range(cols)]
    evr = [[rng.randint(k) if rng.uniform() < 0.8 else -1 for k in cards] for _ in range(cols)]
    ev = np.array([a + b for a, b in zip(evx, evr)], dtype=np.int8)
    cv = np.array([k % V for k in range(cols)], dtype=np.int32)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    for k in range(cols):
        want = Q.amplitude_evidence(c, angs[cv[k]], evx[k], evr[k])
        assert abs(complex(*out[k]) - want) < TOL[prec]


# ---------------------------------------------------------------- gradient
@pytest.mark.parametrize("prec", [64, 32])
def test_hamiltonian_gradient_small_hea(cuda_ctx, prec):
    n, layers = 4, 2
    c = I.hardware_efficient_ansatz(n, layers, I.NOISE_CFG3)
    V, T = 6, 5
    angs = I.uniform_angles(V, c.n_angles, seed=13)
    sup, coef = I.z_string_hamiltonian(n, T, seed=13)
    ac = load(cuda_ctx, c, 1, prec)
    N().set_params(ac, t(angs))
    ev = np.array([[-2 if b else -1 for b in sup[tt]] for _ in range(V) for tt in range(T)], dtype=np.int8)
    cv = np.repeat(np.arange(V, dtype=np.int32), T)
    w = np.tile(coef, V)
    val, grad = N().gradient(ac, t(cv), t(ev), t(w), V)
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    scale = np.abs(coef).sum()
    for v in range(V):
        rv, rg = Q.hamiltonian_value_and_gradient(c, angs[v], sup, coef)
        assert abs(val[v] - rv) < TOL[prec] * scale
        assert np.abs(grad[v] - rg).max() < TOL[prec] * scale * 10


# ---------------------------------------------------------------- sampling
@pytest.mark.parametrize("prec", [64, 32])
def test_qaoa4_sampling_matches_oracle(cuda_ctx, prec):
    c = I.workload("qaoa4_ring_p1")
    V, S = 16, 1000
    angs = I.uniform_angles(V, c.n_angles, seed=1)
    seeds = I.vector_seeds(V, 1)
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=prec)
    N().set_params(ac, t(angs))
    bits = N().sample(ac, t(seeds.astype(np.int64)), t(np.full(V, S, dtype=np.int32)), S).cpu().numpy()
    total_mis = 0
    for v in range(V):
        P = Q.probabilities(c, angs[v])
        ref = Q.chain_rule_samples(P, int(seeds[v]), S)
        Pt = P.reshape((2,) * 4)

        def pref(prefix):
            a = Pt[tuple(prefix)] if prefix else Pt
            return float(np.sum(a)), float(np.sum(a[0]))

        margins = mismatch_margins(pref, int(seeds[v]), bits[v].astype(np.uint64), ref, 4)
        assert all(m <= TIE[prec] for m in margins), margins
        total_mis += len(margins)
    assert total_mis <= (0 if prec == 64 else 5)


def test_sampling_distribution_chi_square(cuda_ctx):
    from scipy.stats import chisquare
    c = I.workload("qaoa4_ring_p1")
    angs = I.uniform_angles(1, c.n_angles, seed=4)
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=32)
    N().set_params(ac, t(angs))
    S = 50000
    bits = N().sample(ac, t(np.array([99], dtype=np.int64)), t(np.array([S], dtype=np.int32)), S).cpu().numpy()[0]
    P = Q.probabilities(c, angs[0])
    counts = np.bincount(bits, minlength=16).astype(float)
    keep = P * S > 5
    exp = P[keep] * S
    obs = counts[keep] * exp.sum() / counts[keep].sum()
    assert chisquare(obs, exp).pvalue > 0.01


def test_sampling_ragged_shots_and_untouched_tail(cuda_ctx):
    c = I.workload("qaoa4_ring_p1")
    V = 5
    angs = I.uniform_angles(V, c.n_angles, seed=8)
    seeds = I.vector_seeds(V, 8)
    shots = np.array([0, 1, 17, 64, 3], dtype=np.int32)
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=64)
    N().set_params(ac, t(angs))
    out = torch.full((V, 64), -7, dtype=torch.int64, device=DEV)
    N().sample(ac, t(seeds.astype(np.int64)), t(shots), 64, out=out)
    out = out.cpu().numpy()
    for v in range(V):
        assert (out[v, shots[v]:] == -7).all()
        ref = Q.chain_rule_samples(Q.probabilities(c, angs[v]), int(seeds[v]), int(shots[v]))
        assert np.array_equal(out[v, :shots[v]].astype(np.uint64), ref)


# ---------------------------------------------------------------- tiling, batch invariance, edge cases
@pytest.mark.parametrize("prec", [64, 32])
def test_tiled_path_equals_untiled(cuda_ctx, prec, monkeypatch):
    c = I.random_circuit(5, 16, seed=800, noise_prob=0.3)
    V = 9
    angs = I.uniform_angles(V, c.n_angles, seed=80)
    b = N().compile(c, 1)
    rng = I.SplitMix(80)
    cols = 1000
    ev = t(np.array([[rng.randint(4) - 2 for _ in range(5)] for _ in range(cols)], dtype=np.int8))
    cv = t(np.array([rng.randint(V) for _ in range(cols)], dtype=np.int32))
    seeds = t(I.vector_seeds(V, 80).astype(np.int64))
    shots = t(np.full(V, 300, dtype=np.int32))
    res = []
    for cap in (None, "64"):
        if cap:
            monkeypatch.setenv("QKC_MAX_TILE_COLUMNS", cap)
        ac = N().load_ac(cuda_ctx, b, precision=prec)
        N().set_params(ac, t(angs))
        out = N().evaluate(ac, cv, ev)
        root, marg = N().marginals(ac, cv, ev)
        bits = N().sample(ac, seeds, shots, 300)
        if cap:
            assert ac.info()["reserved_columns"] == 64
        res.append((out.cpu().numpy(), marg.cpu().numpy(), bits.cpu().numpy()))
        monkeypatch.delenv("QKC_MAX_TILE_COLUMNS", raising=False)
    for a, b_ in zip(res[0], res[1]):
        assert np.array_equal(a, b_)


@pytest.mark.parametrize("prec", [64, 32])
def test_column_alone_equals_column_in_mix(cuda_ctx, prec):
    """Per-column arithmetic (including the FP32 per-(level, column) scale) makes every
    result independent of the other columns in the batch: bitwise equal alone and mixed."""
    c = I.workload("qaoa4_ring_p1")
    V = 8
    angs = I.uniform_angles(V, c.n_angles, seed=12)
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=prec)
    N().set_params(ac, t(angs))
    rng = I.SplitMix(12)
    cols = 300
    ev = np.array([[rng.randint(4) - 2 for _ in range(4)] for _ in range(cols)], dtype=np.int8)
    cv = np.array([rng.randint(V) for _ in range(cols)], dtype=np.int32)
    mixed = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    for k in (0, 77, 299):
        alone = N().evaluate(ac, t(cv[k:k + 1]), t(ev[k:k + 1])).cpu().numpy()
        assert np.array_equal(alone[0], mixed[k])
    perm = np.array([(k * 7919) % cols for k in range(cols)])
    shuffled = N().evaluate(ac, t(cv[perm]), t(ev[perm])).cpu().numpy()
    assert np.array_equal(shuffled, mixed[perm])


def test_edge_cases_and_errors(cuda_ctx):
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1"), precision=32)
    with pytest.raises(N().QKCError) as e:  # parameters not bound yet
        N().evaluate(ac, None, t(np.zeros((1, 4), dtype=np.int8)))
    assert e.value.status == 1
    N().set_params(ac, t(I.uniform_angles(2, 2, seed=3)))
    out = N().evaluate(ac, t(np.zeros(0, dtype=np.int32)), t(np.zeros((0, 4), dtype=np.int8)))
    assert out.shape == (0, 2)
    amp = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1", kind=0), precision=32)
    N().set_params(amp, t(I.uniform_angles(2, 2, seed=3)))
    with pytest.raises(N().QKCError) as e:
        N().sample(amp, t(np.array([1, 2], dtype=np.int64)), t(np.array([3, 3], dtype=np.int32)), 3)
    assert e.value.status == 6
    with pytest.raises(N().QKCError) as e:  # malformed bytes
        N().load_ac(cuda_ctx, b"QKAC" + bytes(60), precision=32)
    assert e.value.status == 2
    b = bytearray(compiled("qaoa4_ring_p1"))
    with pytest.raises(N().QKCError):
        N().load_ac(cuda_ctx, bytes(b[:len(b) // 2]), precision=32)
    with pytest.raises(N().QKCError):
        N().load_ac(cuda_ctx, bytes(b), precision=16)


# ---------------------------------------------------------------- full-size workloads (sampled checks)
def test_hea16_gradient_full_size_sampled(cuda_ctx):
    """16-qubit noisy HEA, 256 vectors x 16 Z-string terms (4096 columns), FP32: value and
    all 192 gradient entries of sampled vectors against the FP64 AC oracle."""
    c = I.workload("hea16_l6")
    b = compiled("hea16_l6")
    V, T = 256, 16
    angs = I.uniform_angles(V, c.n_angles, seed=3)
    sup, coef = I.z_string_hamiltonian(16, T, seed=3)
    ac = N().load_ac(cuda_ctx, b, precision=32)
    N().set_params(ac, t(angs))
    ev = np.array([[-2 if x else -1 for x in sup[tt]] for _ in range(V) for tt in range(T)], dtype=np.int8)
    cv = np.repeat(np.arange(V, dtype=np.int32), T)
    val, grad = N().gradient(ac, t(cv), t(ev), t(np.tile(coef, V)), V)
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    ref = R.ACRef(b)
    scale = np.abs(coef).sum()
    for v in (0, 131, 255):
        rv, rg = 0.0, np.zeros(c.n_angles)
        for tt in range(T):
            a, g = ref.gradient(angs[v], [-2 if x else -1 for x in sup[tt]], coef[tt])
            rv += a
            rg += g
        assert abs(val[v] - rv) < 1e-5 * scale
        assert np.abs(grad[v] - rg).max() < 1e-5 * scale * 10


def test_qaoa32_sampling_full_size_sampled(cuda_ctx):
    """32-qubit noise-free QAOA p=1, 64 vectors x 10000 samples, FP32 (the benchmarked
    launch): sampled indices against the FP64 AC oracle's chain rule, conditional
    marginals on random prefixes, and a chi-square test on two-qubit marginals."""
    from scipy.stats import chisquare
    c = I.workload("qaoa32_3reg_p1_ideal")
    b = compiled("qaoa32_3reg_p1_ideal")
    V, S, n = 64, 10000, 32
    angs = I.uniform_angles(V, c.n_angles, seed=5)
    seeds = I.vector_seeds(V, 5)
    ac = N().load_ac(cuda_ctx, b, precision=32)
    N().set_params(ac, t(angs))
    bits = N().sample(ac, t(seeds.astype(np.int64)), t(np.full(V, S, dtype=np.int32)), S).cpu().numpy()
    ref = R.ACRef(b)

    for v in (0, 37):
        k = 12
        want = ref.sample(angs[v], int(seeds[v]), k)

        def pref(prefix, v=v):
            ev = list(prefix) + [-1] * (n - len(prefix))
            P = ref.up(angs[v], ev).real
            ev[len(prefix)] = 0
            return P, ref.up(angs[v], ev).real

        margins = mismatch_margins(pref, int(seeds[v]), bits[v, :k].astype(np.uint64), want, n)
        assert all(m <= TIE[32] for m in margins), margins
    # conditional marginals on random prefixes
    rng = I.SplitMix(55)
    cols = 16
    ev = np.full((cols, n), -1, dtype=np.int8)
    cv = np.zeros(cols, dtype=np.int32)
    for k in range(cols):
        L = 1 + rng.randint(n - 1)
        ev[k, :L] = [rng.randint(2) for _ in range(L)]
        cv[k] = rng.randint(V)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    for k in range(cols):
        want = ref.up(angs[cv[k]], ev[k]).real  # ~2^-L: a relative bound (an absolute 1e-5 could not fail)
        assert abs(out[k, 0] - want) <= 1e-5 * want
    # two-qubit marginal histograms of one vector
    v = 3
    for (a, bq) in [(0, 1), (5, 17), (30, 31)]:
        exp = np.zeros(4)
        for x in range(4):
            e = [-1] * n
            e[a], e[bq] = x >> 1, x & 1
            exp[x] = ref.up(angs[v], e).real
        xa = (bits[v] >> (n - 1 - a)) & 1
        xb = (bits[v] >> (n - 1 - bq)) & 1
        counts = np.bincount(xa * 2 + xb, minlength=4).astype(float)
        keep = exp * S > 5
        e = exp[keep] * S
        o = counts[keep] * e.sum() / counts[keep].sum()
        assert chisquare(o, e).pvalue > 0.01


def test_qaoa10_p2_amplitude_ac_full_batch(cuda_ctx):
    """10-qubit noisy QAOA p=2 on a random 3-regular graph, the paper's amplitude AC over
    outputs and noise variables, batch of 1024 vectors in FP32: sampled trajectory
    amplitudes A(x, r) against the oracle's pure-state run with the chosen Kraus operators."""
    c = I.workload("qaoa10_3reg_p2")
    b = compiled("qaoa10_3reg_p2", kind=0)
    V = 1024
    angs = I.uniform_angles(V, c.n_angles, seed=2)
    ac = N().load_ac(cuda_ctx, b, precision=32)
    N().set_params(ac, t(angs))
    cards = Q.channel_cards(c)
    rng = I.SplitMix(22)
    cols = 24
    evx, evr = [], []
    for _ in range(cols):
        evx.append([rng.randint(2) for _ in range(10)])
        # mostly the no-error branch, a few errors, like a typical trajectory
        evr.append([0 if rng.uniform() < 0.97 else 1 + rng.randint(k - 1) for k in cards])
    ev = np.array([a + b_ for a, b_ in zip(evx, evr)], dtype=np.int8)
    cv = np.array([rng.randint(V) for _ in range(cols)], dtype=np.int32)
    out = N().evaluate(ac, t(cv), t(ev)).cpu().numpy()
    for k in range(cols):
        psi = Q.statevector(c, angs[cv[k]], evr[k])
        want = psi[tuple(evx[k])]
        assert abs(complex(*out[k]) - want) < 1e-5


def test_sample_total_shots_bound_exact_and_understated(cuda_ctx):
    """total_shots sizes the launches: the exact sum gives the same samples as no hint; an
    understated one drops samples without any out-of-range access and is reported."""
    c = I.random_circuit(7, 28, seed=905, noise_prob=0.4)  # up to 6 x 64 prefix groups: above the bound below
    V = 6
    angs = I.uniform_angles(V, c.n_angles, seed=9)
    seeds = t(I.vector_seeds(V, 9).astype(np.int64))
    shots = np.array([5, 300, 17, 0, 250, 64], dtype=np.int32)
    ac = N().load_ac(cuda_ctx, N().compile(c, 1), precision=32)
    N().set_params(ac, t(angs))
    a = N().sample(ac, seeds, t(shots), 300).cpu().numpy()
    b = N().sample(ac, seeds, t(shots), 300, total_shots=int(shots.sum())).cpu().numpy()
    for v in range(V):
        assert np.array_equal(a[v, :shots[v]], b[v, :shots[v]])
    N().check_status(ac)
    N().sample(ac, seeds, t(shots), 300, total_shots=40)
    with pytest.raises(N().QKCError) as e:
        N().check_status(ac)
    assert e.value.status == 1
    N().check_status(ac)  # cleared
    again = N().sample(ac, seeds, t(shots), 300, total_shots=int(shots.sum())).cpu().numpy()
    for v in range(V):
        assert np.array_equal(a[v, :shots[v]], again[v, :shots[v]])


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", ["qaoa4_ring_p1", "random6", "qaoa32_3reg_p1_ideal"])
def test_memoised_sampler_equals_per_group_sampler(cuda_ctx, prec, name):
    """The memoised sampler evaluates a node once per (vector, prefix bits on its support) and
    must give exactly the samples of the plain sampler (one column per prefix group)."""
    if name == "random6":
        c = I.random_circuit(6, 24, seed=901, noise_prob=0.4)
        b = N().compile(c, 1)
    else:
        c = I.workload(name)
        b = compiled(name)
    V, S = (5, 700) if c.n_qubits < 32 else (4, 400)
    angs = I.uniform_angles(V, c.n_angles, seed=17)
    seeds = t(I.vector_seeds(V, 17).astype(np.int64))
    shots = t(np.array([S, S // 3, 1, S - 7, 64][:V], dtype=np.int32))
    outs = []
    for mode in (0, 2):  # per group, memoised whenever it fits
        ac = N().load_ac(cuda_ctx, b, precision=prec)
        N().set_sampler(ac, mode)
        N().set_params(ac, t(angs))
        outs.append(N().sample(ac, seeds, shots, S).cpu().numpy())
        N().check_status(ac)
    sh = shots.cpu().numpy()
    for v in range(V):
        assert np.array_equal(outs[0][v, :sh[v]], outs[1][v, :sh[v]]), v
    if c.n_qubits <= 6:
        for v in range(V):
            ref = Q.chain_rule_samples(Q.probabilities(c, angs[v]), int(I.vector_seeds(V, 17)[v]), int(sh[v]))
            assert (outs[1][v, :sh[v]].astype(np.uint64) != ref).sum() <= (0 if prec == 64 else 2)


def test_vqe_ising_gradient(cuda_ctx):
    """2D-Ising VQE (3x3 grid, 2 layers, depolarising 0.5%): <H> of two vectors and the gradient in
    four of the 20 angles (a qubit angle and the coupling angle of each layer) in FP32 against the
    density-matrix oracle's forward-mode derivative."""
    c = I.workload("vqe_ising_3x3_noisy")
    sup, coef = I.ising_hamiltonian(3, 3)
    V, T = 2, len(coef)
    angs = I.uniform_angles(V, c.n_angles, seed=29)
    ac = N().load_ac(cuda_ctx, compiled("vqe_ising_3x3_noisy"), precision=32)
    N().set_params(ac, t(angs))
    ev = np.array([[-2 if b else -1 for b in sup[tt]] for _ in range(V) for tt in range(T)], dtype=np.int8)
    cv = np.repeat(np.arange(V, dtype=np.int32), T)
    val, grad = N().gradient(ac, t(cv), t(ev), t(np.tile(coef, V)), V)
    val, grad = val.cpu().numpy(), grad.cpu().numpy()
    scale = np.abs(coef).sum()
    slots = [4, 9, 13, 19]
    for v in range(V):
        rv, rg = Q.hamiltonian_value_and_gradient(c, angs[v], sup, coef, angle_slots=slots if v == 0 else [])
        assert abs(val[v] - rv) < 1e-5 * scale
        if v == 0:
            assert np.abs(grad[v][slots] - rg[slots]).max() < 1e-5 * scale * 10


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", ["vqe_ising_5x5_ideal", "vqe_ising_3x3_noisy"])
def test_memoised_step_sampler_equals_per_group_vqe(cuda_ctx, prec, name):
    """The 2D-Ising VQE step ACs put most of tier B in runs of small levels (chains of 15-20 levels of
    1-8 nodes per step, split into runs of at most 16 levels), with the group keys and root values
    formed inside the runs, and (25 qubits) every step's tier A in one launch: the memoised samples
    equal the per-group sampler's exactly, with ragged shot counts, and their probabilities agree to
    rounding (the two paths' kernels may round products and sums differently)."""
    c = I.workload(name)
    b = compiled(name, N().QKC_AC_DENSITY_STEPS)
    V, S = 6, 600
    angs = I.uniform_angles(V, c.n_angles, seed=23)
    seeds = t(I.vector_seeds(V, 23).astype(np.int64))
    shots = t(np.array([S, 1, S - 11, 97, S // 2, 2], dtype=np.int32))
    outs, probs = [], []
    for mode in (0, 2):  # per group, memoised whenever it fits
        ac = N().load_ac(cuda_ctx, b, precision=prec)
        N().set_sampler(ac, mode)
        N().set_params(ac, t(angs))
        o, pr = N().sample_probs(ac, seeds, shots, S)
        N().check_status(ac)
        outs.append(o.cpu().numpy())
        probs.append(pr.cpu().numpy())
    sh = shots.cpu().numpy()
    for v in range(V):
        assert np.array_equal(outs[0][v, :sh[v]], outs[1][v, :sh[v]]), v
        assert np.allclose(probs[1][v, :sh[v]], probs[0][v, :sh[v]], rtol=1e-12 if prec == 64 else 2e-6, atol=0), v


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("name", ["qaoa4_ring_p1", "random6", "qaoa32_3reg_p1_ideal"])
def test_light_cone_step_sampler(cuda_ctx, prec, name):
    """A light-cone step AC (root j: the density AC of the backward light cone of qubits <= j)
    gives the chain rule the same conditionals as the whole circuit's density AC: its samples,
    per group (mode 0) and memoised (mode 2), match the density AC's memoised samples and the
    oracle's, with differences only at decisions inside the tie margin."""
    if name == "random6":
        c = I.random_circuit(6, 24, seed=903, noise_prob=0.4)
        b1 = N().compile(c, 1)
    else:
        c = I.workload(name)
        b1 = compiled(name)
    b2 = N().compile(c, N().QKC_AC_DENSITY_STEPS)
    n = c.n_qubits
    V, S = (5, 700) if n < 32 else (4, 400)
    angs = I.uniform_angles(V, c.n_angles, seed=19)
    seeds_h = I.vector_seeds(V, 19)
    seeds = t(seeds_h.astype(np.int64))
    shots = t(np.array([S, S // 3, 1, S - 7, 64][:V], dtype=np.int32))
    outs = {}
    for key, b, mode in (("whole", b1, 2), ("steps_plain", b2, 0), ("steps_memo", b2, 2)):
        if n == 32 and key == "steps_plain" and prec == 32:
            continue  # every node of every step per group: covered in FP64
        ac = N().load_ac(cuda_ctx, b, precision=prec)
        N().set_sampler(ac, mode)
        N().set_params(ac, t(angs))
        outs[key] = N().sample(ac, seeds, shots, S).cpu().numpy()
        N().check_status(ac)
    sh = shots.cpu().numpy()
    allowed = 0 if prec == 64 else 3
    for key in outs:
        if key == "whole":
            continue
        diff = sum(int((outs[key][v, :sh[v]] != outs["whole"][v, :sh[v]]).sum()) for v in range(V))
        assert diff <= allowed, (key, diff)
        if n <= 6:
            for v in range(V):
                ref = Q.chain_rule_samples(Q.probabilities(c, angs[v]), int(seeds_h[v]), int(sh[v]))
                assert (outs[key][v, :sh[v]].astype(np.uint64) != ref).sum() <= (0 if prec == 64 else 2)


@pytest.mark.parametrize("prec", [64, 32])
def test_light_cone_step_ac_evaluate_and_unsupported_calls(cuda_ctx, prec):
    """qkc_evaluate on a step AC is the whole circuit's AC (its last root); the downward-pass
    calls are refused with an error status."""
    c = I.random_circuit(5, 20, seed=904, noise_prob=0.4)
    V = 3
    angs = I.uniform_angles(V, c.n_angles, seed=23)
    ev = np.array([[(x >> (4 - j)) & 1 if (x + j) % 3 else -1 for j in range(5)] for x in range(32)], dtype=np.int8)
    cv = np.arange(32, dtype=np.int32) % V
    vals = []
    for kind in (1, N().QKC_AC_DENSITY_STEPS):
        ac = N().load_ac(cuda_ctx, N().compile(c, kind), precision=prec)
        N().set_params(ac, t(angs))
        vals.append(N().evaluate(ac, t(cv), t(ev)).cpu().numpy())
        if kind == 2:
            with pytest.raises(Exception):
                N().marginals(ac, t(cv), t(ev))
            with pytest.raises(Exception):
                N().gradient(ac, t(cv), t(ev), t(np.ones(32)), V)
    assert np.abs(vals[0] - vals[1]).max() < TOL[prec]


@pytest.mark.parametrize("prec", [64, 32])
def test_reevaluate_after_one_angle_update(cuda_ctx, prec):
    """qkc_reevaluate recomputes only the dirty cone of the changed angle slot: after each of a chain
    of one-slot updates its values equal a fresh qkc_evaluate at the same angles (FP64 exactly,
    FP32 within the FP32 tolerance) and the density-matrix oracle's."""
    c = I.hardware_efficient_ansatz(4, 2, I.NOISE_CFG3)
    n, V = c.n_qubits, 3
    angs = I.uniform_angles(V, c.n_angles, seed=31).copy()
    ac = N().load_ac(cuda_ctx, N().compile(c, 1), precision=prec)
    fresh = N().load_ac(cuda_ctx, N().compile(c, 1), precision=prec)
    ev = np.array([[(x >> (n - 1 - j)) & 1 for j in range(n)] for x in range(2 ** n)] * V, dtype=np.int8)
    cv_h = np.repeat(np.arange(V, dtype=np.int32), 2 ** n)
    cv, ev_d = t(cv_h), t(ev)
    N().set_params(ac, t(angs))
    N().evaluate(ac, cv, ev_d)
    rng = I.SplitMix(77)
    for step in range(8):
        k = rng.randint(c.n_angles)
        angs[:, k] = angs[:, k] + 0.3 + 0.1 * step
        N().set_params(ac, t(angs))
        got = N().reevaluate(ac, k, cv, len(cv_h)).cpu().numpy()
        N().set_params(fresh, t(angs))
        ref = N().evaluate(fresh, cv, ev_d).cpu().numpy()
        if prec == 64:
            assert np.array_equal(got, ref), (step, k)
        else:
            assert np.abs(got - ref).max() < TOL[32]
        for v in range(V):
            P = Q.probabilities(c, angs[v])
            assert np.abs(got[v * 2 ** n:(v + 1) * 2 ** n, 0] - P).max() < TOL[prec]


def test_reevaluate_preconditions(cuda_ctx):
    """qkc_reevaluate refuses to run without a preceding evaluation of the same columns, after any
    other pass, and for an angle slot out of range."""
    c = I.hardware_efficient_ansatz(3, 1, None)
    ac = N().load_ac(cuda_ctx, N().compile(c, 1), precision=64)
    angs = I.uniform_angles(2, c.n_angles, seed=5)
    N().set_params(ac, t(angs))
    cv = t(np.array([0, 1, 1], dtype=np.int32))
    ev = t(np.full((3, 3), -1, dtype=np.int8))
    with pytest.raises(Exception):
        N().reevaluate(ac, 0, cv, 3)
    N().evaluate(ac, cv, ev)
    N().reevaluate(ac, 0, cv, 3)
    with pytest.raises(Exception):
        N().reevaluate(ac, c.n_angles, cv, 3)
    with pytest.raises(Exception):
        N().reevaluate(ac, 0, cv, 2)
    N().marginals(ac, cv, ev)
    with pytest.raises(Exception):
        N().reevaluate(ac, 0, cv, 3)


def test_light_cone_step_ac_malformed_bytes(cuda_ctx):
    """The loader checks a step AC's roots table: a root out of range, a last root that is not the
    header's root, or a root count that does not match the qubits are format errors."""
    c = I.workload("qaoa4_ring_p1")
    b = bytearray(N().compile(c, N().QKC_AC_DENSITY_STEPS))
    h = np.frombuffer(bytes(b[:64]), dtype="<u4")
    nv, Nn, E, D, nl, nq = int(h[5]), int(h[6]), int(h[7]), int(h[8]), int(h[9]), int(h[3])
    off = 64
    for nbytes in (4 * nv, 4 * nv, 4 * (D + 1), Nn, 4 * (Nn + 1), 4 * E, 4 * nl, 4 * nl, 16 * nl):
        off = (off + nbytes + 7) & ~7
    N().load_ac(cuda_ctx, bytes(b), precision=64).close()  # well formed
    bad = bytearray(b)
    bad[off:off + 4] = np.array([Nn + 5], dtype="<u4").tobytes()  # root of step 0 out of range
    with pytest.raises(Exception):
        N().load_ac(cuda_ctx, bytes(bad), precision=64)
    bad = bytearray(b)
    r0 = bytes(b[off:off + 4])
    bad[off + 4 * (nq - 1):off + 4 * nq] = r0 if r0 != bytes(b[40:44]) else np.array([0], dtype="<u4").tobytes()
    with pytest.raises(Exception):  # last step root is not the header's root
        N().load_ac(cuda_ctx, bytes(bad), precision=64)
    bad = bytearray(b)
    bad[48:52] = np.array([nq - 1], dtype="<u4").tobytes()  # root count
    with pytest.raises(Exception):
        N().load_ac(cuda_ctx, bytes(bad), precision=64)


@pytest.mark.parametrize("kind", [1, 2])
def test_sampling_after_scratch_reallocations_equals_fresh(cuda_ctx, kind):
    """One AC sampled again and again while its scratch is reallocated between calls (the memoised
    key cap, hence the tile rows, follows the shot count; the per-group sampler needs a row per node)
    gives, call by call, the samples of a fresh AC: captured launch sequences follow the buffers."""
    c = I.random_circuit(6, 24, seed=905, noise_prob=0.4)
    b = N().compile(c, kind)
    V = 3
    angs = t(I.uniform_angles(V, c.n_angles, seed=41))
    seeds = t(I.vector_seeds(V, 41).astype(np.int64))
    ac = N().load_ac(cuda_ctx, b, precision=32)
    N().set_tile_limit(ac, 256)
    for mode, S in ((2, 40), (2, 3000), (0, 500), (2, 40), (1, 1500), (0, 40), (2, 3000)):
        shots = t(np.full(V, S, dtype=np.int32))
        N().set_sampler(ac, mode)
        N().set_params(ac, angs)
        got = N().sample(ac, seeds, shots, S).cpu().numpy()
        fresh = N().load_ac(cuda_ctx, b, precision=32)
        N().set_tile_limit(fresh, 256)
        N().set_sampler(fresh, mode)
        N().set_params(fresh, angs)
        ref = N().sample(fresh, seeds, shots, S).cpu().numpy()
        fresh.close()
        assert np.array_equal(got, ref), (mode, S)


@pytest.mark.parametrize("prec", [64, 32])
def test_qaoa40_sampling_wide_prefixes(cuda_ctx, prec):
    """40 qubits: from step 33 on, group prefixes and key plans need 64-bit words (the 32-bit compress
    covers steps <= 32 only). Memoised and per-group samples agree bit for bit on the density AC, and
    the first samples of two vectors are the FP64 AC oracle's chain rule (the light-cone step AC runs
    the same memoised kernels; at 40 qubits its per-step metadata is several GB, so it is left out)."""
    n = 40
    c = I.qaoa_maxcut(n, I.random_regular_graph(n, 3, seed=7), 1, None)
    b = N().compile(c, 1)
    V, S = 2, 150
    angs = I.uniform_angles(V, c.n_angles, seed=43)
    seeds_h = I.vector_seeds(V, 43)
    seeds = t(seeds_h.astype(np.int64))
    shots = t(np.full(V, S, dtype=np.int32))
    outs = {}
    for key, bb, mode in (("plain", b, 0), ("memo", b, 2)):
        ac = N().load_ac(cuda_ctx, bb, precision=prec)
        N().set_sampler(ac, mode)
        N().set_params(ac, t(angs))
        outs[key] = N().sample(ac, seeds, shots, S).cpu().numpy()
        N().check_status(ac)
        ac.close()
    assert np.array_equal(outs["plain"], outs["memo"])
    ref = R.ACRef(b)
    for v in range(V):
        k = 2
        want = ref.sample(angs[v], int(seeds_h[v]), k)

        def pref(prefix, v=v):
            ev = list(prefix) + [-1] * (n - len(prefix))
            P = ref.up(angs[v], ev).real
            ev[len(prefix)] = 0
            return P, ref.up(angs[v], ev).real

        margins = mismatch_margins(pref, int(seeds_h[v]), outs["memo"][v, :k].astype(np.uint64), want, n)
        assert all(m <= TIE[prec] for m in margins), margins
        assert len(margins) <= (0 if prec == 64 else 1)


@pytest.mark.parametrize("prec", [64, 32])
@pytest.mark.parametrize("kind", [1, 2])
def test_sample_probs_are_outcome_probabilities(cuda_ctx, prec, kind):
    """qkc_sample_probs: each sample's probability as the sampler computed it is P(x) of its outcome
    (density AC and light-cone step AC), against the density matrix: FP64 within 1e-12, FP32 within
    1e-5 of the last step's prefix probability; the indices equal qkc_sample's."""
    c = I.workload("qaoa4_ring_p1")
    V, S = 6, 500
    angs = I.uniform_angles(V, c.n_angles, seed=21)
    seeds = t(I.vector_seeds(V, 21).astype(np.int64))
    shots = t(np.array([S, 1, 77, S, 250, 3], dtype=np.int32))
    ac = N().load_ac(cuda_ctx, compiled("qaoa4_ring_p1", kind), precision=prec)
    N().set_params(ac, t(angs))
    bits, probs = N().sample_probs(ac, seeds, shots, S)
    bits2 = N().sample(ac, seeds, shots, S)
    bits, probs, bits2 = bits.cpu().numpy(), probs.cpu().numpy(), bits2.cpu().numpy()
    sh = shots.cpu().numpy()
    for v in range(V):
        P = Q.probabilities(c, angs[v])
        Pt = P.reshape((2,) * 4)
        x = bits[v, :sh[v]]
        assert np.array_equal(x, bits2[v, :sh[v]])
        want = P[x]
        pre = np.array([Pt[tuple((int(xx) >> (3 - k)) & 1 for k in range(3))].sum() for xx in x])
        bound = 1e-12 if prec == 64 else 1e-5 * pre
        assert (np.abs(probs[v, :sh[v]] - want) <= bound).all(), v
        assert (probs[v, sh[v]:] == 0).all()  # entries past the shots are left untouched
