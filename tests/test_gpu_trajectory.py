"""GPU parity of trajectory sampling (TRAJECTORY ACs) on the 10-qubit noisy QAOA p=2 of the
paper's noisy evaluations (1q depolarising 0.001, 2q depolarising 0.01, a seeded random
3-regular graph; 1024 parameter vectors x 1000 samples at full size).

Every sample draws its noise trajectory r from the channels' branch probabilities (exact for
mixed-unitary channels) and then its outcome by the chain rule on |A(x, r)|^2, the TRAJECTORY
AC's polynomial with r observed.  Checked against oracle/trajectory.py (state vector per
trajectory): FP64 indices bit-exact (a difference only at a tie within 1e-12), FP32 within the
1e-5 tie margin; histograms against the density-matrix oracle's distribution; the AC's values
per trajectory against |psi_r(x)|^2."""
import numpy as np
import pytest

from oracle import quantum as Q
from oracle import trajectory as T
from paper_2103_17226_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
TIE = {64: 1e-12, 32: 1e-5}


def N():
    from paper_2103_17226_gb300 import native
    return native


def t(x):
    return torch.tensor(np.asarray(x), device="cuda")


@pytest.fixture(scope="module")
def cfg2():
    c = I.workload("qaoa10_3reg_p2")
    V = 1024
    return dict(c=c, V=V, angs=I.uniform_angles(V, c.n_angles, seed=2), seeds=I.vector_seeds(V, 2),
                b=N().compile(c, N().QKC_AC_TRAJECTORY))


def _margins(c, angles, seed, got, want):
    """|u P - p0| / P at the first differing qubit of each differing sample, under that sample's
    trajectory (the oracle's)."""
    n = c.n_qubits
    out = []
    for s in np.nonzero(got != want)[0]:
        r = T.draw_trajectory(c, seed, int(s))
        prob = (np.abs(Q.statevector(c, angles, r)) ** 2).reshape((2,) * n)
        g, w = int(got[s]), int(want[s])
        j = next(k for k in range(n) if ((g ^ w) >> (n - 1 - k)) & 1)
        pre = tuple((w >> (n - 1 - k)) & 1 for k in range(j))
        P, p0 = float(prob[pre].sum()), float(prob[pre + (0,)].sum())
        out.append(abs(Q.sample_uniform(seed, int(s), j, n) * P - p0) / P)
    return out


@pytest.mark.parametrize("prec", [64, 32])
def test_trajectory_sampling_against_oracle(cuda_ctx, cfg2, prec):
    """Eight of the 1024 vectors, 150 samples each (tile columns: a group per error trajectory)."""
    W = cfg2
    vs = [0, 131, 262, 393, 524, 655, 786, 1023]
    S = 150
    ac = N().load_ac(cuda_ctx, W["b"], precision=prec)
    N().set_params(ac, t(W["angs"][vs]))
    seeds = W["seeds"][vs]
    bits = N().sample(ac, t(seeds.astype(np.int64)), t(np.full(len(vs), S, dtype=np.int32)), S).cpu().numpy()
    N().check_status(ac)
    mis = 0
    for i, v in enumerate(vs):
        want = T.trajectory_samples(W["c"], W["angs"][v], int(seeds[i]), S)
        got = bits[i].astype(np.uint64)
        m = _margins(W["c"], W["angs"][v], int(seeds[i]), got, want)
        assert all(x <= TIE[prec] for x in m), (v, m)
        mis += len(m)
    assert mis <= (0 if prec == 64 else 3)


def test_trajectory_ac_values_against_statevector(cuda_ctx, cfg2):
    """qkc_evaluate on the TRAJECTORY AC with outputs and noise observed (FP32 and FP64): |psi_r(x)|^2;
    with the outputs free: the trajectory's probability prod p_{r_i}."""
    W = cfg2
    c, n = W["c"], W["c"].n_qubits
    rng = I.SplitMix(91)
    cols, vecs, want = [], [], []
    for k in range(24):
        v = rng.randint(W["V"])
        r = T.draw_trajectory(c, 1000 + k, 0) if k % 3 else [0] * len(T.channels(c))
        if k % 4 == 1:  # a trajectory with a few errors
            r = list(r)
            for _ in range(3):
                i = rng.randint(len(r))
                r[i] = rng.randint(len(T.branch_probabilities(T.channels(c)[i].kind, T.channels(c)[i].p)))
        prob = np.abs(Q.statevector(c, W["angs"][v], r).reshape(-1)) ** 2
        x = rng.randint(2 ** n)
        free = k % 5 == 0
        cols.append(([-1] * n if free else [(x >> (n - 1 - j)) & 1 for j in range(n)]) + list(r))
        vecs.append(v)
        want.append(prob.sum() if free else prob[x])
    for prec in (64, 32):
        ac = N().load_ac(cuda_ctx, W["b"], precision=prec)
        N().set_params(ac, t(W["angs"]))
        out = N().evaluate(ac, t(np.array(vecs, dtype=np.int32)), t(np.array(cols, dtype=np.int8))).cpu().numpy()
        for k in range(len(cols)):
            assert abs(out[k, 0] - want[k]) <= (1e-12 if prec == 64 else 1e-5 * max(want[k], 1e-3)), (prec, k)


def test_trajectory_samples_follow_density_matrix(cuda_ctx, cfg2):
    """Eight vectors x 20000 FP32 samples: outcome histograms against the density-matrix oracle's
    distribution (outcomes expected at least 5 times are bins of their own, the rest one bin):
    chi-square of each vector p > 1e-3 and of the eight together (summed statistics) p > 0.01."""
    from scipy.stats import chi2
    W = cfg2
    vs = [3, 77, 200, 341, 512, 640, 901, 1000]
    S = 20000
    ac = N().load_ac(cuda_ctx, W["b"], precision=32)
    N().set_params(ac, t(W["angs"][vs]))
    bits = N().sample(ac, t(W["seeds"][vs].astype(np.int64)), t(np.full(len(vs), S, dtype=np.int32)), S).cpu().numpy()
    N().check_status(ac)
    Ps = Q.probabilities_many(W["c"], [W["angs"][v] for v in vs])
    tot, dof = 0.0, 0
    for i, P in enumerate(Ps):
        assert abs(P.sum() - 1) < 1e-12
        cnt = np.bincount(bits[i].astype(np.int64), minlength=P.size).astype(float)
        keep = P * S >= 5
        e = np.append(P[keep] * S, P[~keep].sum() * S)
        o = np.append(cnt[keep], cnt[~keep].sum())
        if e[-1] < 5:
            e, o = e[:-1], o[:-1]
        stat = float(((o - e) ** 2 / e).sum())
        assert chi2.sf(stat, len(e) - 1) > 1e-3, (vs[i], stat, len(e))
        tot += stat
        dof += len(e) - 1
    assert chi2.sf(tot, dof) > 0.01, (tot, dof)


def test_trajectory_full_batch_sampled(cuda_ctx, cfg2):
    """The full configuration -- 1024 vectors x 1000 samples, FP32 -- runs through (status clear),
    and the first 100 samples of two vectors match the oracle within the tie margin."""
    W = cfg2
    ac = N().load_ac(cuda_ctx, W["b"], precision=32)
    N().set_params(ac, t(W["angs"]))
    S = 1000
    bits, probs = N().sample_probs(ac, t(W["seeds"].astype(np.int64)), t(np.full(W["V"], S, dtype=np.int32)), S)
    N().check_status(ac)
    bits, probs = bits.cpu().numpy(), probs.cpu().numpy()
    assert (bits >= 0).all() and (bits < 1024).all() and (probs > 0).all()
    for v in (0, 1023):
        want = T.trajectory_samples(W["c"], W["angs"][v], int(W["seeds"][v]), 100)
        m = _margins(W["c"], W["angs"][v], int(W["seeds"][v]), bits[v, :100].astype(np.uint64), want)
        assert all(x <= TIE[32] for x in m) and len(m) <= 1, m


def test_trajectory_edge_cases(cuda_ctx):
    """A circuit without channels compiled as a TRAJECTORY AC has no noise variables: every sample is
    error-free, and its samples equal the density AC's bit for bit (FP64, same uniforms).  Ragged shot
    counts leave the tail untouched; an understated shot total is reported, never read out of range."""
    c0 = I.qaoa_maxcut(6, I.random_regular_graph(6, 3, seed=6), 2, None)
    V = 4
    angs = I.uniform_angles(V, c0.n_angles, seed=8)
    seeds = t(I.vector_seeds(V, 8).astype(np.int64))
    shots = t(np.array([300, 0, 17, 300], dtype=np.int32))
    outs = []
    for kind in (N().QKC_AC_DENSITY, N().QKC_AC_TRAJECTORY):
        ac = N().load_ac(cuda_ctx, N().compile(c0, kind), precision=64)
        assert ac.n_vars == 6
        N().set_params(ac, t(angs))
        out = torch.full((V, 300), -7, dtype=torch.int64, device="cuda")
        N().sample(ac, seeds, shots, 300, out=out)
        N().check_status(ac)
        outs.append(out.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
    assert (outs[1][1] == -7).all() and (outs[1][2, 17:] == -7).all()
    # noisy: an understated total is caught by the status check
    c = I.qaoa_maxcut(6, I.random_regular_graph(6, 3, seed=6), 1, I.NOISE_CFG2)
    ac = N().load_ac(cuda_ctx, N().compile(c, N().QKC_AC_TRAJECTORY), precision=32)
    N().set_params(ac, t(I.uniform_angles(V, c.n_angles, seed=8)))
    N().sample(ac, seeds, shots, 300, total_shots=int(shots.sum().item()))
    N().check_status(ac)
    N().sample(ac, seeds, shots, 300, total_shots=50)
    with pytest.raises(N().QKCError):
        N().check_status(ac)
