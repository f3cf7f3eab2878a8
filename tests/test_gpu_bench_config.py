"""GPU parity at the benchmarked configuration, and on a skewed distribution.

The bench's sampling call, exactly: the 32-qubit noise-free QAOA p=1 (seeded random 3-regular
graph), its light-cone step AC in FP32, the default sampler (mode 1: memoised passes when
estimated cheaper), the default column tile, 64 parameter vectors x 10000 samples.  Checked
  * index for index against the whole density AC's per-group sampler (mode 0): every
    difference must be a decision within the FP32 tie margin, as the FP64 AC oracle decides it;
  * 2000 indices (8 vectors x 250) against the FP64 AC oracle's chain rule (acref), and each
    of their probabilities P(x) as the sampler computed it;
  * p0 / P = P(x_j = 0 | x_<j) on 64 random prefixes against the oracle, relative 1e-5;
  * chi-square of all 496 two-qubit and 100 random three-qubit marginal histograms (each on
    its own 1000 samples) against the oracle's marginals, with a Kolmogorov-Smirnov check that
    the 596 independent p-values look uniform (each single test fails 1% of the time).
The skewed case (angles within a few 1e-3 of 0 on half the qubits: conditionals of 1e-4 to
1e-6) runs the memoised FP32 sampler against the FP64 per-group sampler, whose decisions are
the oracle's: every difference must sit within the tie margin.  It exercises the carried
P(x_<j) of a rare branch and the unscaled tier-A values.
"""
import math

import numpy as np
import pytest

from oracle import acref as R
from oracle import quantum as Q
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TIE32 = 1e-5


def N():
    from paper_2103_17226_gb300 import native
    return native


def t(x):
    return torch.tensor(np.asarray(x), device="cuda")


def _first_diff(g, r, n):
    for j in range(n):
        if ((int(g) >> (n - 1 - j)) & 1) != ((int(r) >> (n - 1 - j)) & 1):
            return j
    return None


def _margins(ref, angles, seed, n, s_idx, got, want):
    """|u P - p0| / P by the FP64 oracle at the first qubit where two indices of sample s differ."""
    out = []
    for s, g, r in zip(s_idx, got, want):
        j = _first_diff(g, r, n)
        prefix = [(int(r) >> (n - 1 - k)) & 1 for k in range(j)]
        ev = prefix + [-1] * (n - j)
        P = ref.up(angles, ev).real
        ev[j] = 0
        p0 = ref.up(angles, ev).real
        out.append(abs(Q.sample_uniform(seed, int(s), j, n) * P - p0) / P)
    return out


@pytest.fixture(scope="module")
def qaoa32():
    c = I.workload("qaoa32_3reg_p1_ideal")
    V, S = 64, 10000
    return dict(c=c, V=V, S=S, angs=I.uniform_angles(V, c.n_angles, seed=5), seeds=I.vector_seeds(V, 5),
                dens=N().compile(c, N().QKC_AC_DENSITY), steps=N().compile(c, N().QKC_AC_DENSITY_STEPS))


@pytest.fixture(scope="module")
def bench_samples(cuda_ctx, qaoa32):
    """The bench's call (light-cone step AC, mode 1, default tile) and the whole density AC's
    per-group sampler on the same inputs."""
    W = qaoa32
    out = {}
    for key, b, mode in (("bench", W["steps"], 1), ("per_group", W["dens"], 0)):
        ac = N().load_ac(cuda_ctx, b, precision=32)
        N().set_sampler(ac, mode)
        N().set_params(ac, t(W["angs"]))
        bits, probs = N().sample_probs(ac, t(W["seeds"].astype(np.int64)), t(np.full(W["V"], W["S"], dtype=np.int32)),
                                       W["S"])
        out[key] = bits.cpu().numpy()
        out[key + "_probs"] = probs.cpu().numpy()
        N().check_status(ac)
        ac.close()
        torch.cuda.empty_cache()
    return out


def test_bench_call_equals_per_group_sampler_up_to_ties(qaoa32, bench_samples):
    W = qaoa32
    a, b = bench_samples["bench"], bench_samples["per_group"]
    assert a.shape == (W["V"], W["S"]) and (a >= 0).all() and (a < 2 ** 32).all()
    ref = R.ACRef(W["dens"])
    diff = 0
    for v in range(W["V"]):
        s_idx = np.nonzero(a[v] != b[v])[0]
        diff += len(s_idx)
        if len(s_idx):
            m = _margins(ref, W["angs"][v], int(W["seeds"][v]), 32, s_idx, a[v, s_idx], b[v, s_idx])
            assert max(m) <= 2 * TIE32, (v, s_idx[:4], m[:4])
    # both are FP32 evaluations of the same probabilities: differences only at near-ties
    assert diff <= 1e-4 * a.size, diff


def test_bench_call_against_oracle_chain_rule(qaoa32, bench_samples):
    """2000 indices (8 vectors x 250 samples) against acref's FP64 chain rule, computed on the
    host cores in spawned processes."""
    W = qaoa32
    vs = [0, 9, 18, 27, 36, 45, 54, 63]
    k = 250
    want = R.run_many(W["dens"], [("sample", W["angs"][v], int(W["seeds"][v]), k) for v in vs])
    ref = R.ACRef(W["dens"])
    mis = 0
    for v, w in zip(vs, want):
        got = bench_samples["bench"][v, :k].astype(np.uint64)
        s_idx = np.nonzero(got != w)[0]
        mis += len(s_idx)
        if len(s_idx):
            m = _margins(ref, W["angs"][v], int(W["seeds"][v]), 32, s_idx, got[s_idx], w[s_idx])
            assert max(m) <= TIE32, (v, m)
    assert mis <= 2, mis


def test_bench_call_sample_probabilities(qaoa32, bench_samples):
    """Each sample's probability P(x) as the bench call computed it (the last step's branch
    probability) against the FP64 oracle, for the 2000 indices above: within the FP32 tie margin of
    the last step, |dP(x)| <= 1e-5 P(x_<n-1)."""
    W = qaoa32
    n, k = 32, 250
    vs = [0, 9, 18, 27, 36, 45, 54, 63]
    tasks = []
    for v in vs:
        for s in range(k):
            x = int(bench_samples["bench"][v, s])
            bits = [(x >> (n - 1 - q)) & 1 for q in range(n)]
            tasks.append(("up", W["angs"][v], bits))
            tasks.append(("up", W["angs"][v], bits[:-1] + [-1]))
    vals = R.run_many(W["dens"], tasks)
    worst = 0.0
    for i, v in enumerate(vs):
        for s in range(k):
            Px, Ppre = vals[2 * (i * k + s)].real, vals[2 * (i * k + s) + 1].real
            err = abs(bench_samples["bench_probs"][v, s] - Px) / Ppre
            worst = max(worst, err)
    assert worst <= TIE32, worst


def test_conditionals_relative_to_oracle(cuda_ctx, qaoa32):
    """p0 / P on 64 random prefixes (lengths 1..31) of random vectors: FP32 upward pass (the
    values the sampler's decisions compare) against the FP64 oracle, relative 1e-5 -- the
    quantity that decides a sample, which an absolute bound cannot check at P ~ 2^-31."""
    W = qaoa32
    n = 32
    ac = N().load_ac(cuda_ctx, W["dens"], precision=32)
    N().set_params(ac, t(W["angs"]))
    rng = I.SplitMix(56)
    cols, vecs = [], []
    for _ in range(64):
        L = 1 + rng.randint(n - 1)
        pre = [rng.randint(2) for _ in range(L)]
        v = rng.randint(W["V"])
        cols.append(pre + [-1] * (n - L))
        cols.append(pre + [0] + [-1] * (n - L - 1))
        vecs += [v, v]
    out = N().evaluate(ac, t(np.array(vecs, dtype=np.int32)), t(np.array(cols, dtype=np.int8))).cpu().numpy()
    ref = R.ACRef(W["dens"])
    worst = 0.0
    for k in range(64):
        v = vecs[2 * k]
        P, p0 = ref.up(W["angs"][v], cols[2 * k]).real, ref.up(W["angs"][v], cols[2 * k + 1]).real
        rel = abs(out[2 * k + 1, 0] / out[2 * k, 0] - p0 / P) / (p0 / P)
        worst = max(worst, rel)
        assert abs(out[2 * k, 0] - P) <= 1e-5 * P and abs(out[2 * k + 1, 0] - p0) <= 1e-5 * p0
    assert worst <= 1e-5, worst


def _chi2_p(counts, exp, S):
    from scipy.stats import chisquare
    keep = exp * S > 5
    e = exp[keep] * S
    o = counts[keep] * e.sum() / counts[keep].sum()
    return float(chisquare(o, e).pvalue)


def test_bench_call_marginal_histograms(qaoa32, bench_samples):
    """All 496 two-qubit and 100 random three-qubit marginal histograms against the oracle's
    marginals.  Each test gets its own 1000 samples -- test k uses vector k % 64, samples
    1000 (k // 64) .. 1000 (k // 64) + 999 -- so the 596 chi-square p-values are independent
    (the same samples shared by all pairs of a qubit would correlate them) and a
    Kolmogorov-Smirnov test of their uniformity is valid.  A single test fails 1% of the time
    by construction; the count below 0.01 and the KS statistic are what is checked."""
    from scipy.stats import kstest
    W = qaoa32
    n, m_per = 32, 1000
    pairs = [(a, b) for a in range(n) for b in range(a + 1, n)]
    rng = I.SplitMix(57)
    triples = set()
    while len(triples) < 100:
        tr = tuple(sorted({rng.randint(n) for _ in range(3)}))
        if len(tr) == 3:
            triples.add(tr)
    subs = pairs + sorted(triples)
    assert len(subs) == 596 and len(subs) <= W["V"] * (W["S"] // m_per)
    tasks = []
    for k, sub in enumerate(subs):
        v = k % W["V"]
        for x in range(2 ** len(sub)):
            ev = [-1] * n
            for i, q in enumerate(sub):
                ev[q] = (x >> (len(sub) - 1 - i)) & 1
            tasks.append(("up", W["angs"][v], ev))
    vals = R.run_many(W["dens"], tasks)
    pv, i = [], 0
    for k, sub in enumerate(subs):
        v, sl = k % W["V"], k // W["V"]
        bits = bench_samples["bench"][v, sl * m_per:(sl + 1) * m_per].astype(np.int64)
        m = 2 ** len(sub)
        exp = np.array([vals[i + x].real for x in range(m)])
        i += m
        assert abs(exp.sum() - 1.0) < 1e-12
        idx = np.zeros(m_per, dtype=np.int64)
        for q in sub:
            idx = idx * 2 + ((bits >> (n - 1 - q)) & 1)
        pv.append(_chi2_p(np.bincount(idx, minlength=m).astype(float), exp, m_per))
    pv = np.array(pv)
    assert (pv < 0.01).sum() <= 16, np.sort(pv)[:20]  # binomial(596, 0.01) tail beyond 16: < 1e-4
    assert kstest(pv, "uniform").pvalue > 0.01


def _skewed_circuit():
    """12 qubits, two HEA-like layers (RY, RZ on every qubit, CZ chain, then RY again): the even
    qubits' RY angles are drawn near 0, so their 1-branches have conditionals of 1e-4 .. 1e-6
    while the odd qubits stay generic."""
    n, layers = 12, 2
    c = I.Circuit(n, 3 * n * layers, name="skewed12")
    a = 0
    for _ in range(layers):
        for q in range(n):
            c.add("RY", q, angle=a)
            a += 1
        for q in range(n):
            c.add("RZ", q, angle=a)
            a += 1
        for q in range(n - 1):
            c.add("CZ", (q, q + 1))
        for q in range(n):
            c.add("RY", q, angle=a)
            a += 1
    return c


def _skewed_angles(c, V, seed):
    ang = I.uniform_angles(V, c.n_angles, seed=seed)
    n = c.n_qubits
    for a in range(c.n_angles):
        q = a % n
        kind = (a // n) % 3  # 0 RY, 1 RZ, 2 RY
        if kind != 1 and q % 2 == 0:
            ang[:, a] = ang[:, a] * 2e-3 / (2 * math.pi) * (1 + q)  # |angle| < 2e-3 (q + 1)
    return ang


@pytest.mark.parametrize("mode", [0, 2])
def test_skewed_distribution_fp32_against_fp64(cuda_ctx, mode):
    """FP32 sampler (per group, mode 0; memoised, mode 2) against the FP64 per-group sampler,
    whose indices equal the oracle's chain rule: each difference must be a near-tie by the FP64
    AC oracle; the count of differences is reported in the assertion message."""
    c = _skewed_circuit()
    n, V, S = c.n_qubits, 64, 10000
    angs = _skewed_angles(c, V, 61)
    seeds = I.vector_seeds(V, 61)
    b = N().compile(c, 1)
    outs = {}
    for prec, m in ((64, 0), (32, mode)):
        ac = N().load_ac(cuda_ctx, b, precision=prec)
        N().set_sampler(ac, m)
        N().set_params(ac, t(angs))
        outs[prec] = N().sample(ac, t(seeds.astype(np.int64)), t(np.full(V, S, dtype=np.int32)), S).cpu().numpy()
        N().check_status(ac)
        ac.close()
    ones = int(sum(((outs[64] >> (n - 1 - q)) & 1).sum() for q in range(0, n, 2)))
    assert ones > 100  # the rare branches are taken often enough to matter
    ref = R.ACRef(b)
    worst, diff = 0.0, 0
    for v in range(V):
        s_idx = np.nonzero(outs[32][v] != outs[64][v])[0]
        diff += len(s_idx)
        if len(s_idx):
            m = _margins(ref, angs[v], int(seeds[v]), n, s_idx, outs[32][v, s_idx], outs[64][v, s_idx])
            worst = max(worst, max(m))
    assert worst <= TIE32, (diff, worst)
    # FP64 per-group = the FP64 oracle's chain rule (checked on two vectors)
    for v in (0, 41):
        want = ref.sample(angs[v], int(seeds[v]), 300)
        assert np.array_equal(outs[64][v, :300].astype(np.uint64), want)
